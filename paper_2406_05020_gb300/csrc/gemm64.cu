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

#include "gemm_tiles.cuh"

namespace gpfvm {

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

// Many GEMV ops in one launch (mgemv_item): S warps per output row.
template <typename T>
__global__ void __launch_bounds__(256) multi_gemv_kernel(const MGemv* __restrict__ ops, int nops, i64 total_rows,
                                                         int S) {
  __shared__ T part[8];
  mgemv_item<T, true>(ops, nops, total_rows, S, blockIdx.x, part);
}

void launch_multi_gemv(const MGemv* d_ops, int nops, i64 total_rows, int f32, int S, cudaStream_t st) {
  if (nops <= 0 || total_rows <= 0) return;
  const int grid = ceil_div(total_rows * S, 8);
  if (f32) launch_pdl(multi_gemv_kernel<float>, grid, 256, 0, st, d_ops, nops, total_rows, S);
  else launch_pdl(multi_gemv_kernel<double>, grid, 256, 0, st, d_ops, nops, total_rows, S);
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
