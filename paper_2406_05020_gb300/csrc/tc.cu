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
// is staged into shared memory.
//
// Per CTA (128 threads): one 128-row output tile at a time; for every segment
// and 32-wide K block the A and B slices are written to shared memory in the
// 128-byte-swizzled K-major layout the UMMA descriptors describe, thread 0
// issues tcgen05.mma (kind::tf32, M = 128, N = padded output size) and
// commits to an mbarrier; the epilogue reads the FP32 accumulator with
// tcgen05.ld (one row per thread) and stores it transposed (coalesced).
// All mbarrier waits are bounded; a timeout sets *status and the kernel
// drains and frees its TMEM before returning.
#include "tc.cuh"

namespace gpfvm {

constexpr int TC_ROWS = 128;
constexpr int TC_KB = 32;                    // floats per K block (128 bytes)
constexpr int TC_A_BYTES = TC_ROWS * 128;    // 16 KB per A slice
constexpr int TC_BREG = 32;                  // B rows per thread / 4: npad <= 128 in registers
constexpr long long TC_SPIN_LIMIT = 1LL << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, c) (c < 32) in a K-major, 128-byte-swizzled slice
__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((c >> 2) ^ (r & 7)) & 7) << 4) + (c & 3) * 4);
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address (16-byte units)
  d |= (uint64_t)1 << 16;                    // leading byte offset: unused for swizzled K-major
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8-row groups 1024 B apart
  d |= (uint64_t)1 << 46;                    // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                    // layout: 128-byte swizzle
  return d;
}

// kind::tf32 instruction descriptor: D f32, A/B tf32, both K-major, M = 128.
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_ROWS >> 4) << 24);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < TC_SPIN_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__global__ void __launch_bounds__(128, 1) tc_mode_kernel(const TcOp* __restrict__ ops, int nops, i64 total,
                                                         int ncols, int* status) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  // carve: A_hi, A_lo (16 KB each), B_hi, B_lo (npad x 128 B each), aligned to 1024
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
  unsigned char* sAhi = base;
  unsigned char* sAlo = base + TC_A_BYTES;
  unsigned char* sBhi = base + 2 * TC_A_BYTES;
  unsigned char* sBlo = sBhi + ncols * 128;
  __shared__ uint64_t bar;
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
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  uint32_t phase = 0;
  pdl_wait();  // TMEM and the barrier are set up while the previous kernel drains

  for (i64 t = blockIdx.x; t < total && !abort_flag; t += gridDim.x) {
    int lo = 0, hi = nops - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ops[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    const TcOp& op = ops[lo];
    if (op.skip && *op.skip) continue;
    const int row0 = (int)(t - op.tile_begin) * TC_ROWS;
    const int K = op.K, N = op.N, R = op.R;
    const int npad = (N + 15) & ~15;
    const uint32_t idesc = idesc_tf32(npad);
    uint32_t acc = 0;
    // Stage (segment, K block) pairs in order; the next pair's global loads
    // are issued into registers while the tensor cores work on the current one.
    const int nkb = (K + TC_KB - 1) / TC_KB;
    const int nstage = op.nseg * nkb;
    float ra[TC_ROWS * TC_KB / 128];  // 32 A values per thread
    float rbh[TC_BREG], rbl[TC_BREG];  // B slice (npad <= 128 rows)
    auto load_stage = [&](int st) {
      const int s = st / nkb, k0 = (st % nkb) * TC_KB;
      const float* __restrict__ A = op.A[s];
      const float* __restrict__ Bh = op.Bhi[s];
      const float* __restrict__ Bl = op.Blo[s];
      const int c = tid & 31, rb = tid >> 5;
      const int gc = k0 + c;
#pragma unroll
      for (int q = 0; q < TC_ROWS * TC_KB / 128; ++q) {
        const int gr = row0 + rb + 4 * q;
        ra[q] = (gr < R && gc < K) ? __ldg(&A[(i64)gr * K + gc]) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < TC_BREG; ++q) {
        const int r = rb + 4 * q;
        const bool in = (r < N && gc < K && r < npad);
        rbh[q] = in ? __ldg(&Bh[(i64)r * K + gc]) : 0.0f;
        rbl[q] = in ? __ldg(&Bl[(i64)r * K + gc]) : 0.0f;
      }
    };
    load_stage(0);
    for (int st = 0; st < nstage && !abort_flag; ++st) {
      const int k0 = (st % nkb) * TC_KB;
      const int c = tid & 31, rb = tid >> 5;
      // registers -> shared (split A into hi / lo), previous MMAs have completed
#pragma unroll
      for (int q = 0; q < TC_ROWS * TC_KB / 128; ++q) {
        const int r = rb + 4 * q;
        const float v = ra[q], vh = tf32_rna(v);
        const uint32_t off = sw128(r, c);
        *(float*)(sAhi + off) = vh;
        *(float*)(sAlo + off) = v - vh;
      }
#pragma unroll
      for (int q = 0; q < TC_BREG; ++q) {
        const int r = rb + 4 * q;
        if (r < npad) {
          const uint32_t off = sw128(r, c);
          *(float*)(sBhi + off) = rbh[q];
          *(float*)(sBlo + off) = rbl[q];
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int kk = min(TC_KB, K - k0);
        const int ksteps = (kk + 7) / 8;
        for (int ks = 0; ks < ksteps; ++ks) {
          const uint32_t koff = ks * 32;  // 8 tf32 = 32 bytes inside the 128-byte row
          const uint64_t ah = desc_sw128(smem_u32(sAhi) + koff), al = desc_sw128(smem_u32(sAlo) + koff);
          const uint64_t bh = desc_sw128(smem_u32(sBhi) + koff), bl = desc_sw128(smem_u32(sBlo) + koff);
          mma_tf32(tmem, ah, bh, idesc, acc);
          acc = 1;
          mma_tf32(tmem, ah, bl, idesc, 1);
          mma_tf32(tmem, al, bh, idesc, 1);
        }
        mma_commit(&bar);
      }
      if (st + 1 < nstage) load_stage(st + 1);  // overlaps the MMAs
      const bool ok = mbar_wait(&bar, phase);
      phase ^= 1;
      if (!ok && tid == 0) {
        atomicOr(status, (int)DEV_TIMEOUT);
        abort_flag = 1;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      __syncthreads();
    }
    if (abort_flag) break;
    // epilogue: row = row0 + tid, columns j < N, rotated store out[j * R + row]
    const int row = row0 + tid;
    for (int j0 = 0; j0 < npad; j0 += 8) {
      uint32_t v[8];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < R) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = j0 + q;
          if (j >= N) break;
          const i64 o = (i64)j * R + row;
          float val = __uint_as_float(v[q]);
          if (op.D) val += op.gamma * op.D[o];
          if (op.beta != 0.0f) val += op.beta * op.out[o];
          op.out[o] = val;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

int tc_smem_bytes(int ncols) { return 2 * TC_A_BYTES + 2 * ncols * 128 + 1024; }

void launch_tc_modes(const TcOp* d_ops, int nops, i64 total_tiles, int max_n, int* status, cudaStream_t st) {
  if (nops <= 0 || total_tiles <= 0) return;
  const int npad = (max_n + 15) & ~15;
  int ncols = 32;
  while (ncols < npad) ncols <<= 1;
  if (npad > 4 * TC_BREG) throw CudaError{cudaErrorInvalidValue, "tc: output size above 128"};
  const int smem = tc_smem_bytes(ncols);
  static int attr_set = 0;
  if (attr_set < smem) {
    GPFVM_CUDA(cudaFuncSetAttribute(tc_mode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes(256)));
    attr_set = tc_smem_bytes(256);
  }
  const int grid = (int)std::min<i64>(total_tiles, 2 * 152);
  launch_pdl(tc_mode_kernel, grid, 128, smem, st, d_ops, nops, total_tiles, ncols, status);
}

// hi = tf32(alpha * F), lo = alpha * F - hi for an n x k row-major factor
__global__ void k_tc_split(const float* __restrict__ F, i64 n, float alpha, float* __restrict__ hi,
                           float* __restrict__ lo) {
  for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x) {
    const float v = alpha * F[e];
    const float h = tf32_rna(v);
    hi[e] = h;
    lo[e] = v - h;
  }
}
void tc_split(const float* F, i64 n, float alpha, float* hi, float* lo, cudaStream_t st) {
  if (n <= 0) return;
  int g = ceil_div(n, 256);
  if (g > 1024) g = 1024;
  k_tc_split<<<g, 256, 0, st>>>(F, n, alpha, hi, lo);
  GPFVM_LAUNCH_CHECK();
}

}  // namespace gpfvm
