// FP64 grouped / segmented / batched GEMM and GEMV on the SIMT DFMA pipe.
//
// Every mode product of the Kronecker matvec (Eq. kronecker-structure), every
// PDE <-> point-set block product and the trailing updates of the IC/BC
// Cholesky reduce to  C = sum_s alpha_s A_s B_s (+ beta C + gamma D).  GB300's
// FP64 rate is low relative to its memory system, so these kernels are bound
// by the DFMA pipe: a 64x64 (or 32x64, 16x64) output tile per CTA, a 4x4 (or
// smaller) register tile per thread, operands staged through shared memory in
// K-chunks of 16, and no more than a few bytes of shared-memory traffic per
// DFMA.
#include "kernels.cuh"

namespace gpfvm {

template <typename T, int BM>
__global__ void __launch_bounds__(256) gemm64_kernel(GemmDesc g) {
  constexpr int BN = 64, BK = 16;
  constexpr int RM = BM / 16;  // rows per thread (4, 2, 1)
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int j0 = blockIdx.x * BN, i0 = blockIdx.y * BM;
  if ((g.tri & TRI_C_LOWER) && j0 > i0 + BM - 1) return;
  if (g.skip && *g.skip) return;
  for (i64 zb = blockIdx.z; zb < (i64)g.batch * g.n_groups; zb += gridDim.z) {
  const int grp = (int)(zb % g.n_groups);
  const int b = (int)(zb / g.n_groups);
  const GemmGroup G = g.groups[grp];

  int k_lo = 0, k_hi = g.k;
  if (g.tri & TRI_A_LOWER) k_hi = min(k_hi, i0 + BM);
  if (g.tri & TRI_A_UPPER) k_lo = max(k_lo, i0);
  if (g.tri & TRI_B_UPPER) k_hi = min(k_hi, j0 + BN);
  if (g.tri & TRI_B_LOWER) k_lo = max(k_lo, j0);

  T acc[RM][4];
#pragma unroll
  for (int r = 0; r < RM; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = T(0);

  const bool a_kfast = (g.a_cs == 1);
  const bool b_jfast = (g.b_cs == 1);

  for (int s = 0; s < G.nseg; ++s) {
    const GemmSeg S = g.segs[G.seg0 + s];
    const T* __restrict__ A = reinterpret_cast<const T*>(S.A) + (i64)b * g.a_bs;
    const T* __restrict__ B = reinterpret_cast<const T*>(S.B) + (i64)b * g.b_bs;
    const T alpha = (T)S.alpha;
    T part[RM][4];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) part[r][c] = T(0);

    for (int k0 = k_lo; k0 < k_hi; k0 += BK) {
      // stage A tile (BM x BK)
      for (int e = tid; e < BM * BK; e += 256) {
        int ii, kk;
        if (a_kfast) { ii = e / BK; kk = e % BK; } else { ii = e % BM; kk = e / BM; }
        const int gi = i0 + ii, gk = k0 + kk;
        As[kk][ii] = (gi < g.m && gk < k_hi) ? A[(i64)gi * g.a_rs + (i64)gk * g.a_cs] : T(0);
      }
      // stage B tile (BK x BN)
      for (int e = tid; e < BK * BN; e += 256) {
        int kk, jj;
        if (b_jfast) { kk = e / BN; jj = e % BN; } else { kk = e % BK; jj = e / BK; }
        const int gk = k0 + kk, gj = j0 + jj;
        Bs[kk][jj] = (gj < g.n && gk < k_hi) ? B[(i64)gk * g.b_rs + (i64)gj * g.b_cs] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[RM], bb[4];
#pragma unroll
        for (int r = 0; r < RM; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bb[c] = Bs[kk][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < RM; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) part[r][c] = fma(a[r], bb[c], part[r][c]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = fma(alpha, part[r][c], acc[r][c]);
  }

  T* __restrict__ C = reinterpret_cast<T*>(G.C) + (i64)b * g.c_bs;
  const T* __restrict__ D = G.D ? reinterpret_cast<const T*>(G.D) + (i64)b * g.d_bs : nullptr;
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    const int gi = i0 + ty + 16 * r;
    if (gi >= g.m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = j0 + tx + 16 * c;
      if (gj >= g.n) continue;
      T v = acc[r][c];
      if (G.beta != 0.0) v += (T)G.beta * C[(i64)gi * g.c_rs + gj];
      if (D) v += (T)G.gamma * D[(i64)gi * g.d_rs + gj];
      C[(i64)gi * g.c_rs + gj] = v;
    }
  }
  }  // zb
}

void launch_gemm64(const GemmDesc& g, cudaStream_t st) {
  if (g.m <= 0 || g.n <= 0 || g.batch <= 0 || g.n_groups <= 0) return;
  const int BM = g.tile == 2 ? 16 : (g.tile == 1 ? 32 : 64);
  i64 z = (i64)g.batch * g.n_groups;
  if (z > 65535) z = 65535;  // the kernel strides over the remaining (batch, group) pairs
  dim3 grid(ceil_div(g.n, 64), ceil_div(g.m, BM), (unsigned)z);
  if (g.f32) {
    if (BM == 64) gemm64_kernel<float, 64><<<grid, 256, 0, st>>>(g);
    else if (BM == 32) gemm64_kernel<float, 32><<<grid, 256, 0, st>>>(g);
    else gemm64_kernel<float, 16><<<grid, 256, 0, st>>>(g);
  } else {
    if (BM == 64) gemm64_kernel<double, 64><<<grid, 256, 0, st>>>(g);
    else if (BM == 32) gemm64_kernel<double, 32><<<grid, 256, 0, st>>>(g);
    else gemm64_kernel<double, 16><<<grid, 256, 0, st>>>(g);
  }
  GPFVM_LAUNCH_CHECK();
}

// One warp per row: y(i) = alpha * sum_j A(i,j) x(j) + beta y(i).
template <typename T>
__global__ void __launch_bounds__(256) gemv_kernel(int m, int n, const T* __restrict__ A, i64 lda,
                                                   const T* __restrict__ x, T* __restrict__ y, T alpha, T beta,
                                                   int tri, const int* skip) {
  if (skip && *skip) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  const int i = warp;
  int lo = 0, hi = n;
  if (tri == 1) hi = min(n, i + 1);
  if (tri == 2) lo = i;
  const T* row = A + (i64)i * lda;
  T s0 = T(0), s1 = T(0);
  int j = lo + lane;
  for (; j + 32 < hi; j += 64) {
    s0 = fma(row[j], x[j], s0);
    s1 = fma(row[j + 32], x[j + 32], s1);
  }
  if (j < hi) s0 = fma(row[j], x[j], s0);
  T s = s0 + s1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[i] = alpha * s + (beta != T(0) ? beta * y[i] : T(0));
}

void launch_gemv64(int m, int n, const double* A, i64 lda, const double* x, double* y, double alpha,
                   double beta, int tri, cudaStream_t st, const int* skip) {
  if (m <= 0) return;
  gemv_kernel<double><<<ceil_div((i64)m * 32, 256), 256, 0, st>>>(m, n, A, lda, x, y, alpha, beta, tri, skip);
  GPFVM_LAUNCH_CHECK();
}

void launch_gemv32(int m, int n, const float* A, i64 lda, const float* x, float* y, float alpha, float beta, int tri,
                   cudaStream_t st, const int* skip) {
  if (m <= 0) return;
  gemv_kernel<float><<<ceil_div((i64)m * 32, 256), 256, 0, st>>>(m, n, A, lda, x, y, alpha, beta, tri, skip);
  GPFVM_LAUNCH_CHECK();
}

__global__ void k_d2f(const double* __restrict__ in, float* __restrict__ out, i64 n) {
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
void convert_d2f(const double* in, float* out, i64 n, cudaStream_t st) {
  if (n <= 0) return;
  int g = ceil_div(n, 256);
  if (g > 8192) g = 8192;
  k_d2f<<<g, 256, 0, st>>>(in, out, n);
  GPFVM_LAUNCH_CHECK();
}

}  // namespace gpfvm
