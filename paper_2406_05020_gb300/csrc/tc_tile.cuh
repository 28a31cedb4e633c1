// Device building blocks of the tcgen05 mode-product kernel (tc.cu), shared
// with the persistent plan kernel (persist.cu).  See tc.cu for the method.
#pragma once
#include <cuda_bf16.h>

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

// byte offset of bf16 element (r, c) (c < 32) in a K-major, 64-byte-swizzled
// slice: 64-byte rows, 8-row atoms of 512 bytes, the 16-byte chunk index
// XOR-ed with address bits 7-8 (= (r >> 1) & 3)
__device__ __forceinline__ uint32_t sw64(int r, int c) {
  return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((((c >> 3) ^ (r >> 1)) & 3) << 4) + (c & 7) * 2);
}

__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address (16-byte units)
  d |= (uint64_t)1 << 16;                    // leading byte offset: unused for swizzled K-major
  d |= (uint64_t)(512 >> 4) << 32;           // stride byte offset: 8-row groups 512 B apart
  d |= (uint64_t)1 << 46;                    // descriptor version (sm_100 family)
  d |= (uint64_t)4 << 61;                    // layout: 64-byte swizzle
  return d;
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

// kind::f16 instruction descriptor with bf16 A and B: D f32, both K-major, M = 128.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_ROWS >> 4) << 24);
}

__device__ __forceinline__ unsigned short bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float bf16_rn(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

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

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
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

// Per-CTA state for running tensor-core tiles (set up by the kernel: one or
// two sets of shared operand buffers, one MMA-completion mbarrier per set,
// the TMEM accumulator, the barrier phases, an abort flag in shared memory
// and the status word).  With two sets, stage s + 1 is written into the other
// set while the MMAs of stage s run; a set is rewritten only after its own
// MMAs have completed.
struct TcCtx {
  unsigned char *sAhi[2], *sAlo[2], *sBhi[2], *sBlo[2];
  uint64_t* bar[2];
  uint32_t tmem;
  uint32_t phase[2];
  int nbuf;
  int* abort_flag;
  int* status;
};

// Waits for the MMAs committed to operand set b (bounded; a timeout sets the
// status and the CTA's abort flag) and flips that set's barrier phase.
__device__ __forceinline__ void tc_wait_set(TcCtx& cx, int b) {
  const bool ok = b ? mbar_wait(cx.bar[1], cx.phase[1]) : mbar_wait(cx.bar[0], cx.phase[0]);
  if (b) cx.phase[1] ^= 1u; else cx.phase[0] ^= 1u;
  if (!ok) {
    atomicOr(cx.status, (int)DEV_TIMEOUT);
    *cx.abort_flag = 1;
  }
}

// One 128-row output tile t of the op table.  Every thread of the CTA calls
// it (it synchronises the CTA); threads 0..127 stage the operands and read
// the accumulator (one row each), the others only join the barriers.
__device__ __forceinline__ void tc_tile(const TcOp* __restrict__ ops, int nops, i64 t, TcCtx& cx) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool act = tid < 128;
  int lo = 0, hi = nops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ops[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  const TcOp& op = ops[lo];
  if (op.skip && *op.skip) return;
  const int sg = op.sgroups;
  const i64 local = t - op.tile_begin;
  const int grp = (int)(local % sg);
  const int row0 = (int)(local / sg) * TC_ROWS;
  const int s_lo = grp * op.nseg / sg;
  const int K = op.K, N = op.N, R = op.R;
  const int npad = (N + 15) & ~15;
  const int mode = op.mode;
  const uint32_t idesc = mode == TC_TF32X3 ? idesc_tf32(npad) : idesc_bf16(npad);
  uint32_t acc = 0;
  // Stage (segment, K block) pairs in order; the next pair's global loads
  // are issued into registers while the tensor cores work on the current one.
  const int nkb = (K + TC_KB - 1) / TC_KB;
  const int nstage = ((grp + 1) * op.nseg / sg - s_lo) * nkb;
  float ra[TC_ROWS * TC_KB / 128];  // 32 A values per thread
  float rbh[TC_BREG], rbl[TC_BREG];  // B slice (npad <= 128 rows)
  const int c = tid & 31, rb = (tid >> 5) & 3;
  auto load_stage = [&](int st) {
    if (!act) return;
    const int s = s_lo + st / nkb, k0 = (st % nkb) * TC_KB;
    const float* __restrict__ A = op.A[s];
    const float* __restrict__ Bh = op.Bhi[s];
    const float* __restrict__ Bl = op.Blo[s];
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
  int st = 0;
  for (; st < nstage; ++st) {
    const int b = cx.nbuf == 2 ? (st & 1) : 0;
    const int k0 = (st % nkb) * TC_KB;
    // the set's previous MMAs (stage st - nbuf) must be done before it is rewritten
    if (st >= cx.nbuf) {
      tc_wait_set(cx, b);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    unsigned char* sAhi = b ? cx.sAhi[1] : cx.sAhi[0];
    unsigned char* sAlo = b ? cx.sAlo[1] : cx.sAlo[0];
    unsigned char* sBhi = b ? cx.sBhi[1] : cx.sBhi[0];
    unsigned char* sBlo = b ? cx.sBlo[1] : cx.sBlo[0];
    // registers -> shared (split A into hi / lo)
    if (act && mode == TC_TF32X3) {
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
    } else if (act) {  // bf16 operands in 64-byte rows (the B parts are exact bf16 values)
#pragma unroll
      for (int q = 0; q < TC_ROWS * TC_KB / 128; ++q) {
        const int r = rb + 4 * q;
        const float v = ra[q], vh = bf16_rn(v);
        const uint32_t off = sw64(r, c);
        *(unsigned short*)(sAhi + off) = bf16_bits(vh);
        if (mode == TC_BF16X3) *(unsigned short*)(sAlo + off) = bf16_bits(v - vh);
      }
#pragma unroll
      for (int q = 0; q < TC_BREG; ++q) {
        const int r = rb + 4 * q;
        if (r < npad) {
          const uint32_t off = sw64(r, c);
          *(unsigned short*)(sBhi + off) = bf16_bits(rbh[q]);
          if (mode == TC_BF16X3) *(unsigned short*)(sBlo + off) = bf16_bits(rbl[q]);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (*cx.abort_flag) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int kk = min(TC_KB, K - k0);
      if (mode == TC_TF32X3) {
        const int ksteps = (kk + 7) / 8;
        for (int ks = 0; ks < ksteps; ++ks) {
          const uint32_t koff = ks * 32;  // 8 tf32 = 32 bytes inside the 128-byte row
          const uint64_t ah = desc_sw128(smem_u32(sAhi) + koff), al = desc_sw128(smem_u32(sAlo) + koff);
          const uint64_t bh = desc_sw128(smem_u32(sBhi) + koff), bl = desc_sw128(smem_u32(sBlo) + koff);
          mma_tf32(cx.tmem, ah, bh, idesc, acc);
          acc = 1;
          mma_tf32(cx.tmem, ah, bl, idesc, 1);
          mma_tf32(cx.tmem, al, bh, idesc, 1);
        }
      } else {
        const int ksteps = (kk + 15) / 16;
        for (int ks = 0; ks < ksteps; ++ks) {
          const uint32_t koff = ks * 32;  // 16 bf16 = 32 bytes inside the 64-byte row
          const uint64_t ah = desc_sw64(smem_u32(sAhi) + koff), bh = desc_sw64(smem_u32(sBhi) + koff);
          mma_bf16(cx.tmem, ah, bh, idesc, acc);
          acc = 1;
          if (mode == TC_BF16X3) {
            const uint64_t al = desc_sw64(smem_u32(sAlo) + koff), bl = desc_sw64(smem_u32(sBlo) + koff);
            mma_bf16(cx.tmem, ah, bl, idesc, 1);
            mma_bf16(cx.tmem, al, bh, idesc, 1);
          }
        }
      }
      mma_commit(b ? cx.bar[1] : cx.bar[0]);
    }
    if (st + 1 < nstage) load_stage(st + 1);  // overlaps the MMAs
  }
  if (!*cx.abort_flag) {
    // drain: the last nbuf stages have not been waited for
    for (int s2 = max(0, nstage - cx.nbuf); s2 < nstage; ++s2) tc_wait_set(cx, cx.nbuf == 2 ? (s2 & 1) : 0);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (*cx.abort_flag) return;
  // epilogue: row = row0 + tid, columns j < N, rotated store out[j * R + row]
  // (a partial sum of a segment group goes to its slice of op.part)
  if (act) {
    const bool fin = sg == 1;
    float* __restrict__ dst = fin ? op.out : op.part + (i64)grp * N * R;
    const int row = row0 + tid;
    for (int j0 = 0; j0 < npad; j0 += 8) {
      uint32_t v[8];
      const uint32_t taddr = cx.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0;
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
          if (fin) {
            if (op.D) val += op.gamma * op.D[o];
            if (op.beta != 0.0f) val += op.beta * op.out[o];
          }
          dst[o] = val;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

}  // namespace gpfvm
