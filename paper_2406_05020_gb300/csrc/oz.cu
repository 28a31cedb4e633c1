// FP64 Kronecker mode products on the 5th-generation tensor cores by exact
// digit products.
//
// Method: the error-free splitting of a matrix product into exactly computed
// partial products (Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012),
// in the fixed-point form of its integer-unit variant (Ootomo, Ozaki and
// Yokota, IJHPCA 2024).  Every row of an FP64 operand is scaled by a power of
// two, taken from the row's largest exponent, into a 55-bit integer
//   X = sum_j d_j 2^(49 - 7 j),   j = 0..7,
// with balanced digits d_j in [-64, 64].  A digit is exact in bf16, a product
// of two digits is exact in FP32 (|d d'| <= 2^12), and for K <= 128 each of
// the 8 "diagonals"
//   acc_d[r][c] = sum_k sum_{a + b = d} dA_a[r][k] dB_b[c][k]        (d = 0..7)
// (at most 8 products per k) stays within 2^22, so tcgen05.mma (kind::f16,
// bf16 inputs, FP32 accumulators in TMEM) computes it exactly.  The diagonals
// are recombined in 64-bit fixed point (the least significant through
// truncating shifts), the segments of a sum are aligned on the grid of the
// largest segment scale max_s 2^(E_s + F_s) of each output (row and column
// exponents of different segments do not add up), and the total is rounded
// once to FP64.  Pairs with a + b >= 8 are dropped;
// with the digit truncation the error of one output stays near 2^-54 of
// K max_k|A[r][k]| max_k|B[c][k]| summed over the segments (FP64
// matrix-product accuracy).  The FP64 FMA rate of this part is about 1/70 of
// its dense bf16 tensor rate.
//
// Per CTA (512 threads; one CTA per SM: its 512 TMEM columns hold 8 diagonals
// x 64 columns): one tile = 128 tensor rows x 64 output columns of one
// op.  For every (segment, 32-wide K block) stage, thread 0 starts a bulk copy
// (cp.async.bulk, mbarrier transaction count) of the stage's pre-sliced factor
// digit planes into shared memory, all threads slice the FP64 tensor rows into
// 8 bf16 digit planes (64-byte-swizzled K-major rows), and thread 0 issues
// 2 x 36 MMAs (M = 128, N = 64, K = 16) into the 8 diagonal accumulators.  Two
// operand sets: the next stage is sliced while the MMAs of the current one
// run; the warps hand a stage to the issuing thread through an mbarrier (no
// CTA barrier per stage).  After the last K block of a segment the
// accumulators are drained into per-thread 64-bit sums.  All waits are bounded; a timeout sets *status and
// the kernel returns after its outstanding copies and MMAs and freeing TMEM.
#include <algorithm>

#include "oz.cuh"
#include "tc_tile.cuh"

namespace gpfvm {

constexpr int OZ_THREADS = 256;   // the long-K GEMM kernel
constexpr int OZ_MTHREADS = 512;  // the mode-product kernel: 16 warps, 4 per TMEM lane quadrant
constexpr int OZ_G = 43;  // binary point of one segment's 64-bit sum (see the drain)
constexpr int OZ_NONFINITE = 0x7fffffff;  // block exponent of a sum that met a NaN or infinity
constexpr int OZ_SET = OZ_DIGITS * OZ_A_PLANE + OZ_IMG_STAGE;  // 96 KB: one operand set
constexpr int OZ_DYN_SMEM = 2 * OZ_SET + 1024;
constexpr int OZ_SOPS = 16;  // op tables up to this size are read from shared memory
static_assert(sizeof(OzOp) % 16 == 0, "op table copied in 16-byte words");

// Outputs of 64 < N <= 128 take the "tall" tiling: the factor (128 rows, all
// outputs) is the MMA's M side and 64 tensor rows its N side, so every tensor
// element is sliced once; otherwise the factor is the N side (64 outputs per
// tile) and 128 tensor rows the M side.
bool oz_tall(int N) { return N > OZ_COLS && N <= 2 * OZ_COLS; }

// rows of one factor digit-image block: 128 for the tall tiling, else 64
static int oz_img_rows(int N) { return oz_tall(N) ? 2 * OZ_COLS : OZ_COLS; }

i64 oz_image_bytes(int N, int K) {
  const int rb = oz_img_rows(N);
  const int nh = (N + rb - 1) / rb, nkb = (K + OZ_KB - 1) / OZ_KB;
  return (i64)nkb * nh * OZ_DIGITS * rb * 64;
}

i64 oz_tiles(int R, int N) {
  if (oz_tall(N)) return (R + OZ_COLS - 1) / OZ_COLS;
  return (i64)((R + OZ_ROWS - 1) / OZ_ROWS) * ((N + OZ_COLS - 1) / OZ_COLS);
}

__device__ __forceinline__ int oz_field(unsigned long long bits) { return (int)((bits >> 52) & 0x7ff); }

// |a| (bit pattern `bits`) as a 55-bit integer on the grid of a row whose
// largest exponent field is emax (zero, subnormal and tiny values give 0)
__device__ __forceinline__ unsigned long long oz_fix(unsigned long long bits, int emax) {
  const int e = oz_field(bits);
  const int sh = max(emax - e, 0);
  if (e == 0 || sh > 54) return 0ull;
  return (((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 2) >> sh;
}

// Balanced digits by an offset: with C = 64 sum_j 2^(49 - 7 j), the plain
// base-128 digits e_j of Y = X + C (X < 2^55, so e_0 <= 128) give
// X = sum_j (e_j - 64) 2^(49 - 7 j): d_j = e_j - 64 in [-64, 64], no carries.
constexpr unsigned long long OZ_C = 64ull * ((1ull << 49) + (1ull << 42) + (1ull << 35) + (1ull << 28) +
                                             (1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);

// digit field j of Y, or-ed into the FP32 pattern of 1.5 * 2^23 (the value 12582912 + e_j)
template <int J>
__device__ __forceinline__ uint32_t oz_field_f32(uint32_t yhi, uint32_t ylo) {
  uint32_t e;
  if (J == 0) e = yhi >> 17;
  else if (J == 1) e = (yhi >> 10) & 127u;
  else if (J == 2) e = (yhi >> 3) & 127u;
  else if (J == 3) e = __funnelshift_r(ylo, yhi, 28) & 127u;
  else if (J == 4) e = (ylo >> 21) & 127u;
  else if (J == 5) e = (ylo >> 14) & 127u;
  else if (J == 6) e = (ylo >> 7) & 127u;
  else e = ylo & 127u;
  return 0x4B400000u | e;
}

// FP32 bit pattern of sgn * d_j (sgn = +-1, the element's sign): its upper
// half is the bf16 pattern of the same integer
template <int J>
__device__ __forceinline__ uint32_t oz_digit_f32(uint32_t yhi, uint32_t ylo, float sgn, float off) {
  return __float_as_uint(fmaf(__uint_as_float(oz_field_f32<J>(yhi, ylo)), sgn, off));
}

// (hi, lo) words of Y = X + C for the element with bit pattern `bits`, and
// its sign factor / offset for oz_digit_f32 (off = -sgn (12582912 + 64))
__device__ __forceinline__ void oz_prep(unsigned long long bits, int emax, uint32_t& yhi, uint32_t& ylo, float& sgn,
                                        float& off) {
  const unsigned long long Y = oz_fix(bits, emax) + OZ_C;
  yhi = (uint32_t)(Y >> 32);
  ylo = (uint32_t)Y;
  sgn = (bits >> 63) ? -1.0f : 1.0f;
  off = (bits >> 63) ? 12582976.0f : -12582976.0f;
}

// acc_a 2^7 + acc_b for two FP32 accumulators holding integers of magnitude
// <= 2^22 (< 2^30: exact in 32 bits).  Adding 1.5 * 2^23 puts an integer into
// the low mantissa bits (offset 0x4B400000 in the bit pattern); the two
// offsets are removed as one constant, mod 2^32.
__device__ __forceinline__ int oz_pair(uint32_t fa, uint32_t fb) {
  const uint32_t ia = __float_as_uint(__uint_as_float(fa) + 12582912.0f);
  const uint32_t ib = __float_as_uint(__uint_as_float(fb) + 12582912.0f);
  return (int)(ia * 128u + ib - 129u * 0x4B400000u);
}

// sum_d acc_d 2^(OZ_G - 7 d) of the 8 diagonals, the last through a
// truncating shift: pairs (2e, 2e + 1) are formed in 32 bits and weighted
// 2^(OZ_G - 14 e - 7); truncating the last pair by 49 - OZ_G bits gives the
// same value as truncating acc_7 alone (acc_6 2^7 is a multiple of 2^(49 - OZ_G))
__device__ __forceinline__ long long oz_diagonals(const uint32_t (&v)[OZ_DIGITS][8], int i) {
  static_assert(OZ_G >= 35 && OZ_G <= 49, "pair weights need 35 <= OZ_G <= 49");
  const int p0 = oz_pair(v[0][i], v[1][i]), p1 = oz_pair(v[2][i], v[3][i]);
  const int p2 = oz_pair(v[4][i], v[5][i]), p3 = oz_pair(v[6][i], v[7][i]);
  return ((long long)p0 << (OZ_G - 7)) + ((long long)p1 << (OZ_G - 21)) + ((long long)p2 << (OZ_G - 35)) +
         (long long)(p3 >> (49 - OZ_G));
}

// S * 2^T rounded to nearest FP64 (S != 0 assumed small enough: |S| < 2^62)
__device__ __forceinline__ double oz_to_double(long long S, int T) {
  if (S == 0) return 0.0;
  const unsigned long long neg = S < 0 ? 1ull : 0ull;
  const unsigned long long u = neg ? (unsigned long long)(-S) : (unsigned long long)S;
  const int p = 63 - __clzll((long long)u);
  unsigned long long mant;
  int ex = p + T;
  if (p <= 52) {
    mant = u << (52 - p);
  } else {
    const int sh = p - 52;
    mant = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++ex;
      }
    }
  }
  const int biased = ex + 1023;
  if (biased <= 0) return neg ? -0.0 : 0.0;  // below the normal range
  if (biased >= 2047) return __longlong_as_double((long long)((neg << 63) | (0x7FFull << 52)));
  return __longlong_as_double((long long)((neg << 63) | ((unsigned long long)biased << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ void oz_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void oz_bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// ---------------------------------------------------------------------------
// largest exponent field of every row of the jobs' R x K tensors (one warp per row)
__global__ void __launch_bounds__(256) oz_rowexp_kernel(const __grid_constant__ OzExpJobs J) {
  pdl_wait();
  if (J.skip && *J.skip) return;
  const int lane = threadIdx.x & 31;
  const i64 total = (i64)J.n * J.R, nwarps = (i64)gridDim.x * 8;
  for (i64 w = (i64)blockIdx.x * 8 + (threadIdx.x >> 5); w < total; w += nwarps) {
    const int job = (int)(w / J.R);
    const i64 r = w - (i64)job * J.R;
    const double* __restrict__ row = J.A[job] + r * J.K;
    int e = 0;
    for (int k = lane; k < J.K; k += 32) e = max(e, oz_field((unsigned long long)__double_as_longlong(__ldg(row + k))));
    e = __reduce_max_sync(0xffffffffu, e);
    if (lane == 0) J.ex[job][r] = e;
  }
}

void oz_row_exponents(const OzExpJobs& jobs, cudaStream_t st) {
  const i64 rows = (i64)jobs.n * jobs.R;
  if (rows <= 0) return;
  const int grid = (int)std::min<i64>((rows + 7) / 8, 8 * 152);
  launch_pdl(oz_rowexp_kernel, grid, 256, 0, st, jobs);
}

// digit image of alpha F (one warp per row j): plane l of (K block kb, row
// block h of rb rows) at img + ((kb * nh + h) * 8 + l) * rb * 64, 64-byte-swizzled rows
__global__ void __launch_bounds__(256) oz_split_kernel(const double* __restrict__ F, i64 rs, i64 cs, int N, int K,
                                                       int rb, double alpha, unsigned char* __restrict__ img,
                                                       int* __restrict__ fexp) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= N) return;  // whole warps
  const int nh = (N + rb - 1) / rb;
  int e = 0;
  for (int k = lane; k < K; k += 32) e = max(e, oz_field((unsigned long long)__double_as_longlong(alpha * F[j * rs + k * cs])));
  e = __reduce_max_sync(0xffffffffu, e);
  if (lane == 0) fexp[j] = e;
  for (int k = lane; k < K; k += 32) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(alpha * F[j * rs + k * cs]);
    uint32_t yh, yl;
    float sg, of;
    oz_prep(bits, e, yh, yl, sg, of);
    uint32_t f[OZ_DIGITS];
    f[0] = oz_digit_f32<0>(yh, yl, sg, of);
    f[1] = oz_digit_f32<1>(yh, yl, sg, of);
    f[2] = oz_digit_f32<2>(yh, yl, sg, of);
    f[3] = oz_digit_f32<3>(yh, yl, sg, of);
    f[4] = oz_digit_f32<4>(yh, yl, sg, of);
    f[5] = oz_digit_f32<5>(yh, yl, sg, of);
    f[6] = oz_digit_f32<6>(yh, yl, sg, of);
    f[7] = oz_digit_f32<7>(yh, yl, sg, of);
    unsigned char* blk = img + ((i64)(k / OZ_KB) * nh + j / rb) * (OZ_DIGITS * rb * 64);
    const uint32_t off = sw64(j % rb, k % OZ_KB);
#pragma unroll
    for (int l = 0; l < OZ_DIGITS; ++l) *(unsigned short*)(blk + l * rb * 64 + off) = (unsigned short)(f[l] >> 16);
  }
}

void oz_split_factor(const double* F, i64 rs, i64 cs, int N, int K, double alpha, unsigned char* img, int* fexp,
                     cudaStream_t st) {
  if (N <= 0 || K <= 0) return;
  GPFVM_CUDA(cudaMemsetAsync(img, 0, oz_image_bytes(N, K), st));
  oz_split_kernel<<<(N + 7) / 8, 256, 0, st>>>(F, rs, cs, N, K, oz_img_rows(N), alpha, img, fexp);
  GPFVM_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// TALL: see oz_tall.  TR tensor rows and TC outputs per tile; the M side of
// the MMA (128 rows: TMEM lanes) is the factor when TALL, else the tensor.
template <bool TALL>
__global__ void __launch_bounds__(OZ_MTHREADS, 1) oz_mode_kernel(const OzOp* __restrict__ ops, int nops, i64 total,
                                                               int* status) {
  constexpr int TR = TALL ? OZ_COLS : OZ_ROWS, TC = TALL ? 2 * OZ_COLS : OZ_COLS;
  constexpr int TPLANE = TR * 64, FPLANE = TC * 64;      // digit plane bytes: tensor, factor
  constexpr int FIMG = OZ_DIGITS * FPLANE;               // one factor image block
  constexpr int EPT = TALL ? 4 : 8, PARTS = OZ_KB / EPT;  // tensor elements per thread and stage
  constexpr int CW = EPT < 8 ? EPT : 8, NCH = EPT / CW;   // elements per smem store, stores per plane
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  unsigned char* base = (unsigned char*)(((uintptr_t)oz_smem + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t mma_bar[2], full_bar[2], ready_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int s_es[OZ_MAXSEG][TR], s_fs[OZ_MAXSEG][TC];
  __shared__ int s_emax[TR], s_fmax[TC];
  __shared__ __align__(16) OzOp s_ops[OZ_SOPS];  // the op table (nops <= OZ_SOPS)
  __shared__ int s_skip[OZ_SOPS];                // ... and the ops' skip flags
  // per output: how far the largest segment scale 2^(E_s + F_s) lies below 2^(emax + fmax)
  __shared__ unsigned char s_del[TR][TC];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(OZ_DIGITS * OZ_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[b])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[b])) : "memory");
      // every warp arrives once its part of a stage's digit planes is written
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&ready_bar[b])), "r"(OZ_MTHREADS / 32)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  pdl_wait();  // TMEM and the barriers are set up while the previous kernel drains
  // small op tables (and their skip flags, fixed for the launch) go to shared
  // memory once, so a tile's prologue reads no op field from global memory
  const bool stab = nops <= OZ_SOPS;
  if (stab) {
    const int words = nops * (int)(sizeof(OzOp) / 16);
    for (int i = tid; i < words; i += OZ_MTHREADS) ((uint4*)s_ops)[i] = ((const uint4*)ops)[i];
    __syncthreads();
    if (tid < nops) s_skip[tid] = s_ops[tid].skip ? *s_ops[tid].skip : 0;
    __syncthreads();
  }
  const OzOp* tab = stab ? s_ops : ops;

  // per-set pipeline state (the same in every thread)
  uint32_t mph0 = 0, mph1 = 0, fph0 = 0, fph1 = 0, rph0 = 0, rph1 = 0;
  int mpend0 = 0, mpend1 = 0, fpend0 = 0, fpend1 = 0;
  auto wait_mma = [&](int b) {
    const bool ok = b ? mbar_wait(&mma_bar[1], mph1) : mbar_wait(&mma_bar[0], mph0);
    if (b) { mph1 ^= 1u; mpend1 = 0; } else { mph0 ^= 1u; mpend0 = 0; }
    if (!ok) {
      atomicOr(status, (int)DEV_TIMEOUT);
      abort_flag = 1;
    }
  };
  const uint32_t idesc = idesc_bf16(OZ_COLS);
  const int q = warp & 3, ch = warp >> 2;     // drain / epilogue: TMEM lane quadrant, 16-column quarter
  const int srow = tid / PARTS, kh = tid % PARTS;  // staging: tensor row, EPT-wide part of the K block

  for (i64 t = blockIdx.x; t < total; t += gridDim.x) {
    if (abort_flag) break;
    int lo = 0, hi = nops - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tab[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    const OzOp& op = tab[lo];
    if (stab ? s_skip[lo] != 0 : (op.skip && *op.skip)) continue;
    const int R = op.R, K = op.K, N = op.N, nseg = op.nseg;
    const int nh = TALL ? 1 : (N + TC - 1) / TC;
    const i64 local = t - op.tile_begin;
    const int h = (int)(local % nh);
    const int row0 = (int)(local / nh) * TR;
    const int nkb = (K + OZ_KB - 1) / OZ_KB;
    const int nstage = nseg * nkb;
    double ra[EPT];
    auto load_stage = [&](int st2) {
      const int s = st2 / nkb, k0 = (st2 % nkb) * OZ_KB + kh * EPT;
      const double* __restrict__ A = op.A[s];
      const int gr = row0 + srow;
      if (gr < R && (K & 1) == 0 && k0 + EPT <= K) {  // 16-byte aligned pairs
        const double2* src = (const double2*)(A + (i64)gr * K + k0);
#pragma unroll
        for (int i = 0; i < EPT / 2; ++i) {
          const double2 t2 = __ldg(src + i);
          ra[2 * i] = t2.x;
          ra[2 * i + 1] = t2.y;
        }
      } else {
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
          const int k = k0 + i;
          ra[i] = (gr < R && k < K) ? __ldg(A + (i64)gr * K + k) : 0.0;
        }
      }
    };
    load_stage(0);  // in flight during the exponent prologue
    for (int i = tid; i < nseg * TR; i += OZ_MTHREADS) {
      const int s = i / TR, r = i % TR;
      s_es[s][r] = (row0 + r < R) ? op.Aexp[s][row0 + r] : 0;
    }
    for (int i = tid; i < nseg * TC; i += OZ_MTHREADS) {
      const int s = i / TC, c = i % TC, j = h * TC + c;
      s_fs[s][c] = (j < N) ? op.Bexp[s][j] : 0;
    }
    __syncthreads();
    if (tid < TR) {
      int m = 0;
      for (int s = 0; s < nseg; ++s) m = max(m, s_es[s][tid]);
      s_emax[tid] = m;
    } else if (tid < TR + TC) {
      int m = 0;
      for (int s = 0; s < nseg; ++s) m = max(m, s_fs[s][tid - TR]);
      s_fmax[tid - TR] = m;
    }
    if (nseg > 1) {
      // the sums are kept on the grid of max_s (E_s + F_s), not of emax + fmax:
      // segments with the largest row and column exponents need not coincide
      __syncthreads();
      for (int i = tid; i < TR * TC; i += OZ_MTHREADS) {
        const int r = i / TC, c = i % TC;
        int tmax = 0;
        for (int s = 0; s < nseg; ++s) tmax = max(tmax, s_es[s][r] + s_fs[s][c]);
        s_del[r][c] = (unsigned char)min(s_emax[r] + s_fmax[c] - tmax, 255);
      }
    }
    // fixed point: one segment's sum V = sum_d acc_d 2^(OZ_G - 7 d) stays below
    // 1.02 * 2^(19 + OZ_G) = 2^62.03 (one unit: 2^-55 of max|a| max|b|); with
    // more segments each is shifted down by guard = ceil(log2 nseg) bits, so
    // |S| < 2^62.03 and value = S * 2^(E + F - 2056 - OZ_G + guard)
    const int guard = nseg > 1 ? 32 - __clz(nseg - 1) : 0;
    long long S[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) S[i] = 0;
    for (int st = 0; st < nstage; ++st) {
      const int s = st / nkb, kb = st % nkb, b = st & 1;
      if (b ? mpend1 : mpend0) wait_mma(b);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* sA = base + b * OZ_SET;            // tensor digit planes
      unsigned char* sB = sA + OZ_DIGITS * TPLANE;       // factor digit planes
      if (tid == 0) {
        uint64_t* fb = b ? &full_bar[1] : &full_bar[0];
        oz_expect_tx(fb, FIMG);
        oz_bulk_copy(sB, op.Bimg[s] + ((i64)kb * nh + h) * FIMG, FIMG, fb);
      }
      if (b) fpend1 = 1; else fpend0 = 1;
      // slice this thread's EPT values of its row into the 8 digit planes
      const int emax = s_es[s][srow];
#pragma unroll
      for (int q2 = 0; q2 < NCH; ++q2) {
        uint32_t w[OZ_DIGITS][CW / 2];
#pragma unroll
        for (int p2 = 0; p2 < CW / 2; ++p2) {
          uint32_t h0, l0, h1, l1;
          float s0, o0, s1, o1;
          oz_prep((unsigned long long)__double_as_longlong(ra[q2 * CW + 2 * p2]), emax, h0, l0, s0, o0);
          oz_prep((unsigned long long)__double_as_longlong(ra[q2 * CW + 2 * p2 + 1]), emax, h1, l1, s1, o1);
#define OZ_PAIR(J) w[J][p2] = __byte_perm(oz_digit_f32<J>(h0, l0, s0, o0), oz_digit_f32<J>(h1, l1, s1, o1), 0x7632)
          OZ_PAIR(0); OZ_PAIR(1); OZ_PAIR(2); OZ_PAIR(3); OZ_PAIR(4); OZ_PAIR(5); OZ_PAIR(6); OZ_PAIR(7);
#undef OZ_PAIR
        }
        const uint32_t off = sw64(srow, kh * EPT + q2 * CW);
#pragma unroll
        for (int j = 0; j < OZ_DIGITS; ++j) {
          if constexpr (CW == 8)
            *(uint4*)(sA + j * TPLANE + off) = make_uint4(w[j][0], w[j][CW / 2 - 3], w[j][CW / 2 - 2], w[j][CW / 2 - 1]);
          else
            *(uint2*)(sA + j * TPLANE + off) = make_uint2(w[j][0], w[j][CW / 2 - 1]);
        }
      }
      // hand the stage to the MMA issuer without a CTA barrier: the other warps
      // go on to the next stage's loads while thread 0 issues this one
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b ? &ready_bar[1] : &ready_bar[0]))
                     : "memory");
      if (tid == 0) {
        const bool ok = (b ? mbar_wait(&ready_bar[1], rph1) : mbar_wait(&ready_bar[0], rph0)) &&
                        (b ? mbar_wait(&full_bar[1], fph1) : mbar_wait(&full_bar[0], fph0));
        if (!ok) {
          atomicOr(status, (int)DEV_TIMEOUT);
          abort_flag = 1;
        } else {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int ksteps = (min(OZ_KB, K - kb * OZ_KB) + 15) / 16;
          // descriptors differ only in the start address field (16-byte units);
          // the M side (128 rows, 8 KB planes) is the factor when TALL
          const uint64_t da0 = desc_sw64(smem_u32(TALL ? sB : sA)), db0 = desc_sw64(smem_u32(TALL ? sA : sB));
          for (int ks = 0; ks < ksteps; ++ks) {
            const uint64_t dak = da0 + (uint64_t)(ks * 2), dbk = db0 + (uint64_t)(ks * 2);  // 32 bytes per K step
#pragma unroll
            for (int d = 0; d < OZ_DIGITS; ++d) {
#pragma unroll
              for (int a = 0; a <= d; ++a)
                mma_bf16(tmem + d * OZ_COLS, dak + (uint64_t)(a * (OZ_A_PLANE >> 4)),
                         dbk + (uint64_t)((d - a) * (OZ_B_PLANE >> 4)), idesc, (kb > 0 || ks > 0 || a > 0) ? 1u : 0u);
            }
          }
        }
        mma_commit(b ? &mma_bar[1] : &mma_bar[0]);
      }
      if (b) { fph1 ^= 1u; rph1 ^= 1u; fpend1 = 0; mpend1 = 1; } else { fph0 ^= 1u; rph0 ^= 1u; fpend0 = 0; mpend0 = 1; }
      if (st + 1 < nstage) load_stage(st + 1);  // overlaps the MMAs
      if (kb == nkb - 1) {
        // segment s complete: add its diagonals, aligned to the tile's exponents, to S
        if (mpend0) wait_mma(0);
        if (mpend1) wait_mma(1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int L = q * 32 + lane;  // TMEM lane: tensor row (else) / output (TALL)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          uint32_t v[OZ_DIGITS][8];
          const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ch * 16 + cc * 8);
#pragma unroll
          for (int d = 0; d < OZ_DIGITS; ++d)
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3]), "=r"(v[d][4]), "=r"(v[d][5]),
                  "=r"(v[d][6]), "=r"(v[d][7])
                : "r"(tb + (uint32_t)(d * OZ_COLS)));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          // the shift of segment s's sum: guard + (emax - E_s) + (fmax - F_s) - del,
          // the lane's own part (its output, or its row) taken once
          const int own = guard + (TALL ? s_fmax[L] - s_fs[s][L] : s_emax[L] - s_es[s][L]);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const long long V = oz_diagonals(v, i);
            const int cidx = ch * 16 + cc * 8 + i;  // TMEM column
            const int row = TALL ? cidx : L, col = TALL ? L : cidx;
            const int sh = own + (TALL ? s_emax[row] - s_es[s][row] : s_fmax[col] - s_fs[s][col]) -
                           (nseg > 1 ? (int)s_del[row][col] : 0);
            if (sh < 62) S[cc * 8 + i] += V >> sh;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // the next segment's MMAs overwrite the accumulators
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
    }
    if (!abort_flag) {
      const int L = q * 32 + lane;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int row = TALL ? ch * 16 + i : L, col = TALL ? L : ch * 16 + i;
        const int gr = row0 + row, j = h * TC + col;
        if (gr < R && j < N) {
          const int EA = s_emax[row];
          {
            const int EB = s_fmax[col];
            const int del = nseg > 1 ? (int)s_del[row][col] : 0;
            double val = (EA == 2047 || EB == 2047) ? __longlong_as_double(0x7FF8000000000000LL)
                                                    : oz_to_double(S[i], EA + EB - del - 2056 - OZ_G + guard);
            const i64 o = (i64)j * R + gr;
            if (op.D) val = fma(op.gamma, op.D[o], val);
            if (op.beta != 0.0) val = fma(op.beta, op.out[o], val);
            op.out[o] = val;
          }
        }
      }
    }
    __syncthreads();
  }
  // after a timeout: let the outstanding copies and MMAs land (bounded) before freeing TMEM
  if (tid == 0) {
    if (fpend0) mbar_wait(&full_bar[0], fph0);
    if (fpend1) mbar_wait(&full_bar[1], fph1);
  }
  if (mpend0) mbar_wait(&mma_bar[0], mph0);
  if (mpend1) mbar_wait(&mma_bar[1], mph1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_DIGITS * OZ_COLS)
                 : "memory");
  }
}

void launch_oz_modes(const OzOp* d_ops, int nops, i64 total_tiles, int n, int* status, cudaStream_t st) {
  if (nops <= 0 || total_tiles <= 0) return;
  static int sms = 0;
  static bool attr = false;
  if (!attr) {
    int dev = 0;
    GPFVM_CUDA(cudaGetDevice(&dev));
    GPFVM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GPFVM_CUDA(cudaFuncSetAttribute(oz_mode_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_DYN_SMEM));
    GPFVM_CUDA(cudaFuncSetAttribute(oz_mode_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_DYN_SMEM));
    attr = true;
  }
  const int grid = (int)std::min<i64>(total_tiles, std::max(sms, 1));
  if (oz_tall(n))
    launch_pdl(oz_mode_kernel<true>, grid, OZ_MTHREADS, OZ_DYN_SMEM, st, d_ops, nops, total_tiles, status);
  else
    launch_pdl(oz_mode_kernel<false>, grid, OZ_MTHREADS, OZ_DYN_SMEM, st, d_ops, nops, total_tiles, status);
}

// ---------------------------------------------------------------------------
// FP64 GEMM by digit products for long K (the dense FP64 work of the IC/BC
// Cholesky stage): C = beta C + gamma D + alpha A B.  K is cut into windows of
// OZ_KMAX with their own row / column exponents (oz_gemm_exponents); every
// window's 8 diagonals are exact as above, and are added into per-output
// block-floating 64-bit sums: S with exponent eS, rescaled when a window with
// a larger scale arrives, each window shifted down by `guard` bits so that up
// to 2^guard windows cannot overflow.

// largest exponent field of every (row, window) of a K-major (sk == 1, warp per
// row) or row-major-across-rows (sr == 1, thread per row) operand; `tri`
// zeroes (kk > row) for 1 and (kk < row) for 2
__global__ void __launch_bounds__(256) oz_winexp_kernel(const double* __restrict__ X, i64 sr, i64 sk, int rows, int K,
                                                        int nwin, int tri, int* __restrict__ ex, const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  if (sk == 1) {
    const i64 total = (i64)rows * nwin, nw = (i64)gridDim.x * 8;
    for (i64 w = (i64)blockIdx.x * 8 + (threadIdx.x >> 5); w < total; w += nw) {
      const int r = (int)(w / nwin), win = (int)(w % nwin);
      int e = 0;
      for (int k = win * OZ_KMAX + lane; k < min(K, (win + 1) * OZ_KMAX); k += 32) {
        if ((tri == 1 && k > r) || (tri == 2 && k < r)) continue;
        e = max(e, oz_field((unsigned long long)__double_as_longlong(__ldg(X + r * sr + k))));
      }
      e = __reduce_max_sync(0xffffffffu, e);
      if (lane == 0) ex[(i64)r * nwin + win] = e;
    }
  } else {
    const i64 total = (i64)rows * nwin;
    for (i64 w = (i64)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (i64)gridDim.x * blockDim.x) {
      const int win = (int)(w / rows), r = (int)(w % rows);  // consecutive threads: consecutive rows
      int e = 0;
      for (int k = win * OZ_KMAX; k < min(K, (win + 1) * OZ_KMAX); ++k) {
        if ((tri == 1 && k > r) || (tri == 2 && k < r)) continue;
        e = max(e, oz_field((unsigned long long)__double_as_longlong(__ldg(X + r * sr + k * sk))));
      }
      ex[(i64)r * nwin + win] = e;
    }
  }
}

__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(const __grid_constant__ OzGemm g, int* status) {
  extern __shared__ __align__(1024) unsigned char oz_smem[];
  unsigned char* base = (unsigned char*)(((uintptr_t)oz_smem + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t mma_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int s_ea[OZ_ROWS], s_eb[OZ_COLS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(OZ_DIGITS * OZ_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  pdl_wait();
  if (g.skip && *g.skip) goto done;
  {
    uint32_t mph0 = 0, mph1 = 0;
    int mpend0 = 0, mpend1 = 0;
    auto wait_mma = [&](int b) {
      const bool ok = b ? mbar_wait(&mma_bar[1], mph1) : mbar_wait(&mma_bar[0], mph0);
      if (b) { mph1 ^= 1u; mpend1 = 0; } else { mph0 ^= 1u; mpend0 = 0; }
      if (!ok) {
        atomicOr(status, (int)DEV_TIMEOUT);
        abort_flag = 1;
      }
    };
    const uint32_t idesc = idesc_bf16(OZ_COLS);
    const int q = warp & 3, ch = warp >> 2;
    const int srow = tid >> 1, kh = tid & 1;
    const bool bk = g.b_rs == 1;  // B K-major (rows of B^T contiguous)
    const int bj = bk ? (tid >> 2) : (tid & 63), bq = bk ? (tid & 3) : (tid >> 6);
    const int tiles_n = (g.n + OZ_COLS - 1) / OZ_COLS;
    const i64 total = (i64)((g.m + OZ_ROWS - 1) / OZ_ROWS) * tiles_n;
    for (i64 t = blockIdx.x; t < total; t += gridDim.x) {
      if (abort_flag) break;
      const int row0 = (int)(t / tiles_n) * OZ_ROWS, col0 = (int)(t % tiles_n) * OZ_COLS;
      if ((g.tri & TRI_C_LOWER) && col0 > row0 + OZ_ROWS - 1) continue;
      // windows that can be nonzero for this tile
      int w_lo = 0, w_hi = g.nwin - 1;
      if (g.tri & TRI_A_LOWER) w_hi = min(w_hi, (row0 + OZ_ROWS - 1) / OZ_KMAX);
      if (g.tri & TRI_A_UPPER) w_lo = max(w_lo, row0 / OZ_KMAX);
      if (g.tri & TRI_B_UPPER) w_hi = min(w_hi, (col0 + OZ_COLS - 1) / OZ_KMAX);
      if (g.tri & TRI_B_LOWER) w_lo = max(w_lo, col0 / OZ_KMAX);
      const int nw = w_hi - w_lo + 1;
      const int guard = nw > 1 ? 32 - __clz(nw - 1) : 0;
      long long S[32];
      int eS[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) { S[i] = 0; eS[i] = -1000000; }
      const int nstage = nw > 0 ? nw * (OZ_KMAX / OZ_KB) : 0;
      double ra[16], rb[8];
      auto load_stage = [&](int st2) {
        const int kk0 = (w_lo + st2 / (OZ_KMAX / OZ_KB)) * OZ_KMAX + (st2 % (OZ_KMAX / OZ_KB)) * OZ_KB;
        const int gr = row0 + srow, ka = kk0 + kh * 16;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int k = ka + i;
          const bool z = gr >= g.m || k >= g.k || ((g.tri & TRI_A_LOWER) && k > gr) || ((g.tri & TRI_A_UPPER) && k < gr);
          ra[i] = z ? 0.0 : __ldg(g.A + (i64)gr * g.a_rs + k);
        }
        const int gj = col0 + bj, kb2 = kk0 + bq * 8;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = kb2 + i;
          const bool z = gj >= g.n || k >= g.k || ((g.tri & TRI_B_UPPER) && k > gj) || ((g.tri & TRI_B_LOWER) && k < gj);
          rb[i] = z ? 0.0 : __ldg(g.B + (i64)k * g.b_rs + (i64)gj * g.b_cs);
        }
      };
      if (nstage > 0) load_stage(0);
      for (int st = 0; st < nstage; ++st) {
        const int kb = st % (OZ_KMAX / OZ_KB), win = w_lo + st / (OZ_KMAX / OZ_KB), b = st & 1;
        if (kb == 0) {  // this window's exponents (the previous window is drained)
          if (tid < OZ_ROWS) s_ea[tid] = row0 + tid < g.m ? g.Aexp[(i64)(row0 + tid) * g.nwin + win] : 0;
          else if (tid < OZ_ROWS + OZ_COLS) {
            const int j = col0 + tid - OZ_ROWS;
            s_eb[tid - OZ_ROWS] = j < g.n ? g.Bexp[(i64)j * g.nwin + win] : 0;
          }
          __syncthreads();
        }
        if (b ? mpend1 : mpend0) wait_mma(b);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char* sA = base + b * OZ_SET;
        unsigned char* sB = sA + OZ_DIGITS * OZ_A_PLANE;
        {  // A: 16 values of row srow
          const int emax = s_ea[srow];
#pragma unroll
          for (int q2 = 0; q2 < 2; ++q2) {
            uint32_t w[OZ_DIGITS][4];
#pragma unroll
            for (int p2 = 0; p2 < 4; ++p2) {
              uint32_t h0, l0, h1, l1;
              float s0, o0, s1, o1;
              oz_prep((unsigned long long)__double_as_longlong(ra[q2 * 8 + 2 * p2]), emax, h0, l0, s0, o0);
              oz_prep((unsigned long long)__double_as_longlong(ra[q2 * 8 + 2 * p2 + 1]), emax, h1, l1, s1, o1);
#define OZ_PAIR(J) w[J][p2] = __byte_perm(oz_digit_f32<J>(h0, l0, s0, o0), oz_digit_f32<J>(h1, l1, s1, o1), 0x7632)
              OZ_PAIR(0); OZ_PAIR(1); OZ_PAIR(2); OZ_PAIR(3); OZ_PAIR(4); OZ_PAIR(5); OZ_PAIR(6); OZ_PAIR(7);
#undef OZ_PAIR
            }
            const uint32_t off = sw64(srow, kh * 16 + q2 * 8);
#pragma unroll
            for (int j = 0; j < OZ_DIGITS; ++j)
              *(uint4*)(sA + j * OZ_A_PLANE + off) = make_uint4(w[j][0], w[j][1], w[j][2], w[j][3]);
          }
        }
        {  // B: 8 values of B^T row bj (K-block chunk bq)
          const int emax = s_eb[bj];
          uint32_t w[OZ_DIGITS][4];
#pragma unroll
          for (int p2 = 0; p2 < 4; ++p2) {
            uint32_t h0, l0, h1, l1;
            float s0, o0, s1, o1;
            oz_prep((unsigned long long)__double_as_longlong(rb[2 * p2]), emax, h0, l0, s0, o0);
            oz_prep((unsigned long long)__double_as_longlong(rb[2 * p2 + 1]), emax, h1, l1, s1, o1);
#define OZ_PAIR(J) w[J][p2] = __byte_perm(oz_digit_f32<J>(h0, l0, s0, o0), oz_digit_f32<J>(h1, l1, s1, o1), 0x7632)
            OZ_PAIR(0); OZ_PAIR(1); OZ_PAIR(2); OZ_PAIR(3); OZ_PAIR(4); OZ_PAIR(5); OZ_PAIR(6); OZ_PAIR(7);
#undef OZ_PAIR
          }
          const uint32_t off = sw64(bj, bq * 8);
#pragma unroll
          for (int j = 0; j < OZ_DIGITS; ++j)
            *(uint4*)(sB + j * OZ_B_PLANE + off) = make_uint4(w[j][0], w[j][1], w[j][2], w[j][3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (abort_flag) break;
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t da0 = desc_sw64(smem_u32(sA)), db0 = desc_sw64(smem_u32(sB));
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t dak = da0 + (uint64_t)(ks * 2), dbk = db0 + (uint64_t)(ks * 2);
#pragma unroll
            for (int d = 0; d < OZ_DIGITS; ++d) {
#pragma unroll
              for (int a = 0; a <= d; ++a)
                mma_bf16(tmem + d * OZ_COLS, dak + (uint64_t)(a * (OZ_A_PLANE >> 4)),
                         dbk + (uint64_t)((d - a) * (OZ_B_PLANE >> 4)), idesc, (kb > 0 || ks > 0 || a > 0) ? 1u : 0u);
            }
          }
          mma_commit(b ? &mma_bar[1] : &mma_bar[0]);
        }
        if (b) mpend1 = 1; else mpend0 = 1;
        if (st + 1 < nstage) load_stage(st + 1);
        if (kb == OZ_KMAX / OZ_KB - 1) {
          // window complete: fold its diagonals into the block-floating sums
          if (mpend0) wait_mma(0);
          if (mpend1) wait_mma(1);
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int row = q * 32 + lane;
          const int ea = s_ea[row];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            uint32_t v[OZ_DIGITS][8];
            const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ch * 32 + cc * 8);
#pragma unroll
            for (int d = 0; d < OZ_DIGITS; ++d)
              asm volatile(
                  "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                  : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3]), "=r"(v[d][4]), "=r"(v[d][5]),
                    "=r"(v[d][6]), "=r"(v[d][7])
                  : "r"(tb + (uint32_t)(d * OZ_COLS)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const long long V = oz_diagonals(v, i);
              const int k = cc * 8 + i;
              const int eb = s_eb[ch * 32 + k];
              const int ew = ea + eb;
              if (ea == 2047 || eb == 2047) eS[k] = OZ_NONFINITE;  // a NaN or infinity in this window
              if (V != 0 && eS[k] != OZ_NONFINITE) {
                if (ew > eS[k]) {  // rescale the sum to the new, larger scale
                  const int dsh = ew - eS[k];
                  S[k] = dsh < 62 ? (S[k] >> dsh) : 0;
                  eS[k] = ew;
                }
                const int sh = guard + eS[k] - ew;
                if (sh < 62) S[k] += V >> sh;
              }
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncthreads();
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
      }
      if (!abort_flag) {
        const int row = q * 32 + lane, gr = row0 + row;
        if (gr < g.m) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int j = col0 + ch * 32 + i;
            if (j < g.n) {
              double val = eS[i] == OZ_NONFINITE ? __longlong_as_double(0x7FF8000000000000LL)
                           : S[i] == 0                ? 0.0
                                                      : oz_to_double(S[i], eS[i] - 2056 - OZ_G + guard);
              val *= g.alpha;
              double* c = g.C + (i64)gr * g.c_rs + j;
              if (g.beta != 0.0) val = fma(g.beta, *c, val);
              if (g.D) val = fma(g.gamma, g.D[(i64)gr * g.d_rs + j], val);
              *c = val;
            }
          }
        }
      }
      __syncthreads();
    }
    if (mpend0) mbar_wait(&mma_bar[0], mph0);
    if (mpend1) mbar_wait(&mma_bar[1], mph1);
  }
done:
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_DIGITS * OZ_COLS)
                 : "memory");
  }
}

void oz_gemm(const OzGemm& g0, int* Aexp, int* Bexp, int* status, cudaStream_t st) {
  if (g0.m <= 0 || g0.n <= 0) return;
  OzGemm g = g0;
  g.nwin = (g.k + OZ_KMAX - 1) / OZ_KMAX;
  g.Aexp = Aexp;
  g.Bexp = Bexp;
  const int triA = (g.tri & TRI_A_LOWER) ? 1 : (g.tri & TRI_A_UPPER) ? 2 : 0;
  const int triB = (g.tri & TRI_B_UPPER) ? 1 : (g.tri & TRI_B_LOWER) ? 2 : 0;
  if (g.k > 0) {
    const i64 ra = (i64)g.m * g.nwin, rb = (i64)g.n * g.nwin;
    launch_pdl(oz_winexp_kernel, (int)std::min<i64>((ra + 7) / 8, 8 * 152), 256, 0, st, g.A, g.a_rs, (i64)1, g.m, g.k,
               g.nwin, triA, Aexp, g.skip);
    if (g.b_rs == 1)
      launch_pdl(oz_winexp_kernel, (int)std::min<i64>((rb + 7) / 8, 8 * 152), 256, 0, st, g.B, g.b_cs, (i64)1, g.n,
                 g.k, g.nwin, triB, Bexp, g.skip);
    else
      launch_pdl(oz_winexp_kernel, (int)std::min<i64>((rb + 255) / 256, 8 * 152), 256, 0, st, g.B, g.b_cs, g.b_rs,
                 g.n, g.k, g.nwin, triB, Bexp, g.skip);
  }
  static int sms = 0;
  static bool attr = false;
  if (!attr) {
    int dev = 0;
    GPFVM_CUDA(cudaGetDevice(&dev));
    GPFVM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GPFVM_CUDA(cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_DYN_SMEM));
    attr = true;
  }
  const i64 tiles = (i64)((g.m + OZ_ROWS - 1) / OZ_ROWS) * ((g.n + OZ_COLS - 1) / OZ_COLS);
  launch_pdl(oz_gemm_kernel, (int)std::min<i64>(tiles, std::max(sms, 1)), OZ_THREADS, OZ_DYN_SMEM, st, g, status);
}

}  // namespace gpfvm
