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
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "kernels.cuh"

namespace gpfvm {

// cp.async (global -> shared, bypassing registers) of one element; src_bytes
// = 0 zero-fills the destination without reading the source.
template <typename T>
__device__ __forceinline__ void cp_async_el(T* dst, const T* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// pipeline depth: shared memory per CTA stays below the 48 KB static limit
template <typename T, int BM>
struct GemmStages {
  static constexpr int value = sizeof(T) == 8 ? (BM == 64 ? 2 : (BM == 32 ? 3 : 4)) : 4;
};

// One output tile (BM x 64) of one (batch, group) entry; all threads of the
// CTA must call it together (it synchronises through shared memory).  The
// (segment, 16-wide K chunk) pairs form one sequence of stages that cp.async
// streams into a ring of STAGES shared-memory buffers, so up to STAGES - 1
// chunks are in flight while one is multiplied: a short tile pays the
// global-load latency about once instead of once per chunk.  The arithmetic
// order (per segment: chunks in K order, then acc += alpha * part) is fixed.
template <typename T, int BM>
__device__ __forceinline__ void gemm_tile(const GemmDesc& g, int bx, int by, i64 zb, T (*As)[16][BM + 1],
                                          T (*Bs)[16][65]) {
  constexpr int BN = 64, BK = 16;
  constexpr int RM = BM / 16;  // rows per thread (4, 2, 1)
  constexpr int STAGES = GemmStages<T, BM>::value;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int j0 = bx * BN, i0 = by * BM;
  if ((g.tri & TRI_C_LOWER) && j0 > i0 + BM - 1) return;
  const int grp = (int)(zb % g.n_groups);
  const int b = (int)(zb / g.n_groups);
  const GemmGroup G = g.groups[grp];

  int k_lo = 0, k_hi = g.k;
  if (g.tri & TRI_A_LOWER) k_hi = min(k_hi, i0 + BM);
  if (g.tri & TRI_A_UPPER) k_lo = max(k_lo, i0);
  if (g.tri & TRI_B_UPPER) k_hi = min(k_hi, j0 + BN);
  if (g.tri & TRI_B_LOWER) k_lo = max(k_lo, j0);
  const int nkc = k_hi > k_lo ? (k_hi - k_lo + BK - 1) / BK : 0;
  const int nst = G.nseg * nkc;

  const bool a_kfast = (g.a_cs == 1);
  const bool b_jfast = (g.b_cs == 1);

  // issue the copies of stage st into ring buffer buf
  auto issue = [&](int st, int buf) {
    const int sg = st / nkc, k0 = k_lo + (st % nkc) * BK;
    const GemmSeg S = g.segs[G.seg0 + sg];
    const T* __restrict__ A = reinterpret_cast<const T*>(S.A) + (i64)b * g.a_bs;
    const T* __restrict__ B = reinterpret_cast<const T*>(S.B) + (i64)b * g.b_bs;
    for (int e = tid; e < BM * BK; e += 256) {
      int ii, kk;
      if (a_kfast) { ii = e / BK; kk = e % BK; } else { ii = e % BM; kk = e / BM; }
      const int gi = i0 + ii, gk = k0 + kk;
      const bool ok = gi < g.m && gk < k_hi;
      cp_async_el(&As[buf][kk][ii], ok ? A + (i64)gi * g.a_rs + (i64)gk * g.a_cs : A, ok);
    }
    for (int e = tid; e < BK * BN; e += 256) {
      int kk, jj;
      if (b_jfast) { kk = e / BN; jj = e % BN; } else { kk = e % BK; jj = e / BK; }
      const int gk = k0 + kk, gj = j0 + jj;
      const bool ok = gj < g.n && gk < k_hi;
      cp_async_el(&Bs[buf][kk][jj], ok ? B + (i64)gk * g.b_rs + (i64)gj * g.b_cs : B, ok);
    }
  };

  T acc[RM][4], part[RM][4];
#pragma unroll
  for (int r = 0; r < RM; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = part[r][c] = T(0);

#pragma unroll
  for (int st = 0; st < STAGES - 1; ++st) {
    if (st < nst) issue(st, st);
    cp_async_commit();
  }
  for (int st = 0; st < nst; ++st) {
    cp_async_wait<STAGES - 2>();  // stage st has landed (for this thread)
    __syncthreads();              // ... for all threads; buffer (st - 1) % STAGES is free again
    if (st + STAGES - 1 < nst) issue(st + STAGES - 1, (st + STAGES - 1) % STAGES);
    cp_async_commit();
    const int buf = st % STAGES;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[RM], bb[4];
#pragma unroll
      for (int r = 0; r < RM; ++r) a[r] = As[buf][kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bb[c] = Bs[buf][kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) part[r][c] = fma(a[r], bb[c], part[r][c]);
    }
    if (st % nkc == nkc - 1) {  // last chunk of segment st / nkc
      const T alpha = (T)g.segs[G.seg0 + st / nkc].alpha;
#pragma unroll
      for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[r][c] = fma(alpha, part[r][c], acc[r][c]);
          part[r][c] = T(0);
        }
    }
  }
  cp_async_wait<0>();
  __syncthreads();  // the ring is reused by the CTA's next tile

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
}

template <typename T, int BM>
__global__ void __launch_bounds__(256) gemm64_kernel(GemmDesc g) {
  pdl_wait();
  __shared__ T As[GemmStages<T, BM>::value][16][BM + 1];
  __shared__ T Bs[GemmStages<T, BM>::value][16][65];
  if (g.skip && *g.skip) return;
  for (i64 zb = blockIdx.z; zb < (i64)g.batch * g.n_groups; zb += gridDim.z)
    gemm_tile<T, BM>(g, blockIdx.x, blockIdx.y, zb, As, Bs);
}

// Many GEMM ops (different shapes and operands, same element type and row
// tile) in one launch: CTA t works on tile t - ops[o].tile_begin of op o.
template <typename T, int BM>
__global__ void __launch_bounds__(256) multi_gemm_kernel(const MOp* __restrict__ ops, int nops, i64 total) {
  __shared__ T As[GemmStages<T, BM>::value][16][BM + 1];
  __shared__ T Bs[GemmStages<T, BM>::value][16][65];
  bool waited = false;
  for (i64 t = blockIdx.x; t < total; t += gridDim.x) {
    // the op tables are written at plan build time: look them up before waiting
    int lo = 0, hi = nops - 1;
    while (lo < hi) {  // last op with tile_begin <= t
      const int mid = (lo + hi + 1) >> 1;
      if (ops[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    const MOp& op = ops[lo];
    const i64 r = t - op.tile_begin;
    const int bx = (int)(r % op.tiles_x);
    const int by = (int)((r / op.tiles_x) % op.tiles_y);
    const i64 zb = r / ((i64)op.tiles_x * op.tiles_y);
    if (!waited) {
      pdl_wait();
      waited = true;
    }
    if (op.g.skip && *op.g.skip) continue;
    gemm_tile<T, BM>(op.g, bx, by, zb, As, Bs);
  }
  if (!waited) pdl_wait();
}

void launch_multi_gemm(const MOp* d_ops, int nops, i64 total, int f32, int bm, cudaStream_t st) {
  if (nops <= 0 || total <= 0) return;
  const int grid = (int)std::min<i64>(total, 152 * 16);
  if (f32) {
    if (bm == 64) launch_pdl(multi_gemm_kernel<float, 64>, grid, 256, 0, st, d_ops, nops, total);
    else if (bm == 32) launch_pdl(multi_gemm_kernel<float, 32>, grid, 256, 0, st, d_ops, nops, total);
    else launch_pdl(multi_gemm_kernel<float, 16>, grid, 256, 0, st, d_ops, nops, total);
  } else {
    if (bm == 64) launch_pdl(multi_gemm_kernel<double, 64>, grid, 256, 0, st, d_ops, nops, total);
    else if (bm == 32) launch_pdl(multi_gemm_kernel<double, 32>, grid, 256, 0, st, d_ops, nops, total);
    else launch_pdl(multi_gemm_kernel<double, 16>, grid, 256, 0, st, d_ops, nops, total);
  }
}

// sum_{j in [jlo, jhi)} row[j] x[j] over one warp (result in every lane):
// 16-byte vector loads over the aligned interior (four independent
// accumulators, so that many loads are in flight), scalar head and tail.
template <typename T>
__device__ __forceinline__ T warp_row_dot(const T* __restrict__ row, const T* __restrict__ x, int jlo, int jhi,
                                          int lane) {
  constexpr int W = 16 / sizeof(T);
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V;
  T acc0 = T(0), acc1 = T(0), acc2 = T(0), acc3 = T(0);
  const bool vec = (((uintptr_t)row | (uintptr_t)x) & 15) == 0;
  const int va = vec ? min(jhi, (jlo + W - 1) / W * W) : jhi;
  const int vb = vec ? max(va, jhi / W * W) : jhi;
  for (int j = jlo + lane; j < va; j += 32) acc0 = fma(row[j], x[j], acc0);
  for (int j = vb + lane; j < jhi; j += 32) acc1 = fma(row[j], x[j], acc1);
  const int nv = (vb - va) / W;
  const V* __restrict__ rv = reinterpret_cast<const V*>(row + va);
  const V* __restrict__ xv = reinterpret_cast<const V*>(x + va);
  auto dot = [](const V& a, const V& b, T acc) {
    if constexpr (sizeof(T) == 4) {
      acc = fma(a.x, b.x, acc);
      acc = fma(a.y, b.y, acc);
      acc = fma(a.z, b.z, acc);
      return fma(a.w, b.w, acc);
    } else {
      acc = fma(a.x, b.x, acc);
      return fma(a.y, b.y, acc);
    }
  };
  int v = lane;
  for (; v + 96 < nv; v += 128) {
    const V a0 = rv[v], a1 = rv[v + 32], a2 = rv[v + 64], a3 = rv[v + 96];
    const V b0 = xv[v], b1 = xv[v + 32], b2 = xv[v + 64], b3 = xv[v + 96];
    acc0 = dot(a0, b0, acc0);
    acc1 = dot(a1, b1, acc1);
    acc2 = dot(a2, b2, acc2);
    acc3 = dot(a3, b3, acc3);
  }
  for (; v < nv; v += 32) acc2 = dot(rv[v], xv[v], acc2);
  T s = (acc0 + acc1) + (acc2 + acc3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Many GEMV ops in one launch, one warp per output row over all ops:
// y = alpha * A x + beta * z  (z may alias y).
template <typename T>
__global__ void __launch_bounds__(256) multi_gemv_kernel(const MGemv* __restrict__ ops, int nops, i64 total_rows) {
  const i64 w = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= total_rows) return;
  int lo = 0, hi = nops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ops[mid].row_begin <= w) lo = mid; else hi = mid - 1;
  }
  const MGemv op = ops[lo];  // copied to registers before the wait
  pdl_wait();
  if (op.skip && *op.skip) return;
  const int i = (int)(w - op.row_begin);
  int jlo = 0, jhi = op.n;
  if (op.tri == 1) jhi = min(op.n, i + 1);
  if (op.tri == 2) jlo = i;
  const T* row = reinterpret_cast<const T*>(op.A) + (i64)i * op.lda;
  const T* x = reinterpret_cast<const T*>(op.x);
  const T s = warp_row_dot(row, x, jlo, jhi, lane);
  if (lane == 0) {
    T v = (T)op.alpha * s;
    if (op.beta != 0.0) v += (T)op.beta * reinterpret_cast<const T*>(op.z)[i];
    reinterpret_cast<T*>(op.y)[i] = v;
  }
}

void launch_multi_gemv(const MGemv* d_ops, int nops, i64 total_rows, int f32, cudaStream_t st) {
  if (nops <= 0 || total_rows <= 0) return;
  const int grid = ceil_div(total_rows * 32, 256);
  if (f32) launch_pdl(multi_gemv_kernel<float>, grid, 256, 0, st, d_ops, nops, total_rows);
  else launch_pdl(multi_gemv_kernel<double>, grid, 256, 0, st, d_ops, nops, total_rows);
}

void launch_gemm64(const GemmDesc& g, cudaStream_t st) {
  if (g.m <= 0 || g.n <= 0 || g.batch <= 0 || g.n_groups <= 0) return;
  const int BM = g.tile == 2 ? 16 : (g.tile == 1 ? 32 : 64);
  i64 z = (i64)g.batch * g.n_groups;
  if (z > 65535) z = 65535;  // the kernel strides over the remaining (batch, group) pairs
  dim3 grid(ceil_div(g.n, 64), ceil_div(g.m, BM), (unsigned)z);
  if (g.f32) {
    if (BM == 64) launch_pdl(gemm64_kernel<float, 64>, grid, 256, 0, st, g);
    else if (BM == 32) launch_pdl(gemm64_kernel<float, 32>, grid, 256, 0, st, g);
    else launch_pdl(gemm64_kernel<float, 16>, grid, 256, 0, st, g);
  } else {
    if (BM == 64) launch_pdl(gemm64_kernel<double, 64>, grid, 256, 0, st, g);
    else if (BM == 32) launch_pdl(gemm64_kernel<double, 32>, grid, 256, 0, st, g);
    else launch_pdl(gemm64_kernel<double, 16>, grid, 256, 0, st, g);
  }
}

// One warp per row: y(i) = alpha * sum_j A(i,j) x(j) + beta y(i).
template <typename T>
__global__ void __launch_bounds__(256) gemv_kernel(int m, int n, const T* __restrict__ A, i64 lda,
                                                   const T* __restrict__ x, T* __restrict__ y, T alpha, T beta,
                                                   int tri, const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  const int i = warp;
  int lo = 0, hi = n;
  if (tri == 1) hi = min(n, i + 1);
  if (tri == 2) lo = i;
  const T* row = A + (i64)i * lda;
  const T s = warp_row_dot(row, x, lo, hi, lane);
  if (lane == 0) y[i] = alpha * s + (beta != T(0) ? beta * y[i] : T(0));
}

void launch_gemv64(int m, int n, const double* A, i64 lda, const double* x, double* y, double alpha,
                   double beta, int tri, cudaStream_t st, const int* skip) {
  if (m <= 0) return;
  launch_pdl(gemv_kernel<double>, ceil_div((i64)m * 32, 256), 256, 0, st, m, n, A, lda, x, y, alpha, beta, tri, skip);
}

void launch_gemv32(int m, int n, const float* A, i64 lda, const float* x, float* y, float alpha, float beta, int tri,
                   cudaStream_t st, const int* skip) {
  if (m <= 0) return;
  launch_pdl(gemv_kernel<float>, ceil_div((i64)m * 32, 256), 256, 0, st, m, n, A, lda, x, y, alpha, beta, tri, skip);
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
