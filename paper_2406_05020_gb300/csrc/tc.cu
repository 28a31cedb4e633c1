// Kronecker mode products on the 5th-generation tensor cores (tcgen05, TMEM).
//
// A mode product along the contiguous (last) axis of a tensor is the GEMM
//   out[j][r] = sum_s sum_k A_s[r][k] * B_s[j][k]
// with A_s the tensor viewed as (rows x K) and B_s = alpha_s * F_s the (N x K)
// 1D factor.  Writing the output with the new axis first ("rotating" the
// axes) makes the next axis contiguous, so the three levels of the shared
// Kronecker matvec (Eq. kronecker-structure) are all K-major x K-major GEMMs
// and the third level returns the tensor to its original (t, x, y) order.
//
// Precision: split TF32.  Each operand x = x_hi + x_lo with x_hi = tf32(x)
// (round to nearest) and x_lo = x - x_hi; the product is accumulated in FP32
// TMEM as A_hi B_hi + A_hi B_lo + A_lo B_hi, about FP32 accuracy.  Factors are
// pre-scaled and pre-split once per assembly; tensor data is split while it
// is staged into shared memory.  The bf16 forms (kind::f16) split into
// bf16(x) and bf16(x - bf16(x)) (three products, about 2^-16 relative) or
// keep bf16(x) alone (one product, 2^-8), staged in 64-byte-swizzled rows.
//
// Per CTA (128 threads): one 128-row output tile at a time; for every segment
// and 32-wide K block the A and B slices are written to shared memory in the
// 128-byte-swizzled K-major layout the UMMA descriptors describe, thread 0
// issues tcgen05.mma (kind::tf32, M = 128, N = padded output size) and
// commits to an mbarrier; the epilogue reads the FP32 accumulator with
// tcgen05.ld (one row per thread) and stores it transposed (coalesced).
// All mbarrier waits are bounded; a timeout sets *status and the kernel
// drains and frees its TMEM before returning.
#include <cstdlib>

#include "tc_tile.cuh"

namespace gpfvm {

__global__ void __launch_bounds__(128, 1) tc_mode_kernel(const TcOp* __restrict__ ops, int nops, i64 total,
                                                         int ncols, int nbuf, int* status) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  // carve, twice: A_hi, A_lo (16 KB each), B_hi, B_lo (ncols x 128 B each), aligned to 1024
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
  const int set_bytes = 2 * TC_A_BYTES + 2 * ncols * 128;
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])) : "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  TcCtx cx{};
  for (int b = 0; b < 2; ++b) {
    unsigned char* sb = base + (nbuf == 2 ? b : 0) * set_bytes;
    cx.sAhi[b] = sb;
    cx.sAlo[b] = sb + TC_A_BYTES;
    cx.sBhi[b] = sb + 2 * TC_A_BYTES;
    cx.sBlo[b] = sb + 2 * TC_A_BYTES + ncols * 128;
    cx.bar[b] = &bar[b];
    cx.phase[b] = 0u;
  }
  cx.nbuf = nbuf;
  cx.tmem = tmem_slot;
  cx.abort_flag = &abort_flag;
  cx.status = status;
  pdl_wait();  // TMEM and the barrier are set up while the previous kernel drains
  for (i64 t = blockIdx.x; t < total && !abort_flag; t += gridDim.x) tc_tile(ops, nops, t, cx);
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(cx.tmem), "r"(ncols) : "memory");
  }
}

// out = sum_g part[g] (groups in order) + gamma D + beta out, for the split ops
__global__ void __launch_bounds__(256) tc_sum_kernel(const TcOp* __restrict__ ops) {
  pdl_wait();
  const TcOp& op = ops[blockIdx.y];
  if (op.sgroups <= 1 || (op.skip && *op.skip)) return;
  const i64 n = (i64)op.N * op.R;
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x) {
    float v = 0.0f;
    for (int g = 0; g < op.sgroups; ++g) v += op.part[(i64)g * n + e];
    if (op.D) v += op.gamma * op.D[e];
    if (op.beta != 0.0f) v += op.beta * op.out[e];
    op.out[e] = v;
  }
}

int tc_smem_bytes(int ncols, int nbuf) { return nbuf * (2 * TC_A_BYTES + 2 * ncols * 128) + 1024; }

// GPFVM_TC_NBUF=1 or 2 forces the number of operand sets (for timing both).
static int tc_env_nbuf() {
  static const int v = [] {
    const char* e = std::getenv("GPFVM_TC_NBUF");
    const int n = e ? std::atoi(e) : 0;
    return (n == 1 || n == 2) ? n : 0;
  }();
  return v;
}

// Two operand sets (staging overlapped with the MMAs of the previous stage)
// where two CTAs still fit on an SM with them; one set otherwise, so that
// two CTAs overlap each other instead.
static int tc_nbuf(int ncols) { return 2 * tc_smem_bytes(ncols, 2) <= 227 * 1024 ? 2 : 1; }

void launch_tc_modes(const TcOp* d_ops, int nops, i64 total_tiles, int max_n, int* status, cudaStream_t st,
                     int any_split) {
  if (nops <= 0 || total_tiles <= 0) return;
  const int npad = (max_n + 15) & ~15;
  int ncols = 32;
  while (ncols < npad) ncols <<= 1;
  if (npad > 4 * TC_BREG) throw CudaError{cudaErrorInvalidValue, "tc: output size above 128"};
  const int nbuf = tc_env_nbuf() ? tc_env_nbuf() : tc_nbuf(ncols);
  const int smem = tc_smem_bytes(ncols, nbuf);
  static int attr_set = 0;
  if (attr_set < smem) {
    GPFVM_CUDA(cudaFuncSetAttribute(tc_mode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes(128, 2)));
    attr_set = tc_smem_bytes(128, 2);
  }
  const int grid = (int)std::min<i64>(total_tiles, 2 * 152);
  launch_pdl(tc_mode_kernel, grid, 128, smem, st, d_ops, nops, total_tiles, ncols, nbuf, status);
  if (any_split) launch_pdl(tc_sum_kernel, dim3(2 * 152, nops), 256, 0, st, d_ops);
}

// hi / lo parts of alpha * F (n entries) for the operand format `mode`:
// TF32X3 hi = tf32(v), lo = v - hi; BF16X3 hi = bf16(v), lo = bf16(v - hi);
// BF16 hi = bf16(v), lo = 0
__global__ void k_tc_split(const float* __restrict__ F, i64 n, float alpha, float* __restrict__ hi,
                           float* __restrict__ lo, int mode) {
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x) {
    const float v = alpha * F[e];
    const float h = mode == TC_TF32X3 ? tf32_rna(v) : bf16_rn(v);
    hi[e] = h;
    lo[e] = mode == TC_TF32X3 ? v - h : (mode == TC_BF16X3 ? bf16_rn(v - h) : 0.0f);
  }
}
void tc_split(const float* F, i64 n, float alpha, float* hi, float* lo, cudaStream_t st, int mode) {
  if (n <= 0) return;
  int g = ceil_div(n, 256);
  if (g > 1024) g = 1024;
  k_tc_split<<<g, 256, 0, st>>>(F, n, alpha, hi, lo, mode);
  GPFVM_LAUNCH_CHECK();
}

}  // namespace gpfvm
