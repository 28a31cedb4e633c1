// Device building blocks of the SIMT GEMM/GEMV kernels (gemm64.cu), shared
// with the persistent plan kernel (persist.cu): one pipelined output tile of
// a grouped/segmented GEMM and one warp-wide row dot product.
#pragma once
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

// CTA item `item` (8 warps) of a merged multi-GEMV with S warps per output
// row (S = 1, 2 or 4): y = alpha A x + beta z (z scaled by zs when given).
// Warp k of a row sums the k-th of S equal column chunks; the row's first
// warp adds the chunks in order, so the result is fixed for a given S.  All
// threads of the CTA call this when S > 1 (it synchronises the CTA).  With PDL
// the op is read before waiting on the previous grid.
template <typename T, bool PDL>
__device__ __forceinline__ void mgemv_item(const MGemv* __restrict__ ops, int nops, i64 total_rows, int S, i64 item,
                                           T* part) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const i64 w = item * 8 + wib;
  const i64 row = w / S;
  const int sp = (int)(w - row * S);
  const bool active = row < total_rows;
  int lo = 0;
  if (active) {
    int hi = nops - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ops[mid].row_begin <= row) lo = mid; else hi = mid - 1;
    }
  }
  const MGemv op = ops[lo];  // in registers before the wait
  if (PDL) pdl_wait();
  if (op.skip && *op.skip) return;  // one flag for the whole launch
  T s = T(0);
  int i = 0;
  if (active) {
    i = (int)(row - op.row_begin);
    int jlo = 0, jhi = op.n;
    if (op.tri == 1) jhi = min(op.n, i + 1);
    if (op.tri == 2) jlo = i;
    const int len = max(jhi - jlo, 0), ch = (len + S - 1) / S;
    const int a = jlo + sp * ch, b = max(a, min(jhi, a + ch));
    s = warp_row_dot(reinterpret_cast<const T*>(op.A) + (i64)i * op.lda, reinterpret_cast<const T*>(op.x), a, b,
                     lane);
  }
  if (S > 1) {
    if (lane == 0) part[wib] = s;
    __syncthreads();
    if (active && sp == 0 && lane == 0)
      for (int k = 1; k < S; ++k) s += part[wib + k];
  }
  if (active && sp == 0 && lane == 0) {
    T v = (T)op.alpha * s;
    if (op.beta != 0.0) {
      const T zi = reinterpret_cast<const T*>(op.z)[i];
      v += (T)op.beta * (op.zs ? (T)op.zs[i] * zi : zi);
    }
    reinterpret_cast<T*>(op.y)[i] = v;
  }
  if (S > 1) __syncthreads();  // part is free again
}

}  // namespace gpfvm
