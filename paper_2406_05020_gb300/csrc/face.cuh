// Products with point sets that lie on faces of the box (Sec. 4.1, Eq.
// kronecker-structure, for the IC/BC blocks): a set with few coordinates n_a
// on one axis a (the initial condition at t = 0, the pair of walls x = 0, 1)
// has an n_a x N_a factor on that axis, so for each of its faces m < n_a
//   (G_BP in)_m = sum_t c_t F_tb^T (f_u(t),m x_a in) F_tc      (contract, then bilinear)
//   G_PB w     = sum_{u,m} f_u,m (x) [sum_{t: u(t) = u} c_t F_tb W_m F_tc^T]   (bilinear, then expand)
// with b < c the other two axes, f_u,m row m of the distinct factors on a and
// W_m the face-m slice of the set's values.
// Three device operations cover both directions; each is split into items of
// one CTA (256 threads) so that a launch (or the persistent plan kernel) can
// serve the ops of all sets of a phase at once:
//   CONTR   Y_u = alpha f_u x_a in                      (one read of `in` for all u)
//   BILIN   out = sum_t alpha_t A_t X_t B_t^T            (R x C, inner K1 x K2 <= 128;
//           the distinct A, X, B are staged once in shared memory)
//   EXPADD  dst += sum_k P_k + sum_j alpha_j f_j (x)_{a_j} Z_j   (in a fixed order)
#pragma once
#include "common.cuh"
#include "gemm_tiles.cuh"

namespace gpfvm {

constexpr int FACE_THREADS = 256;
constexpr int FACE_MAXF = 4;    // factor vectors per contraction
constexpr int FACE_MAXT = 8;    // terms per bilinear form
constexpr int FACE_MAXJ = 16;   // expansion terms per expand-add
constexpr int FACE_MAXN = 128;  // largest dimension of a bilinear form
constexpr int FACE_RB = 4;      // output rows per bilinear item
constexpr int FACE_EXP_EPT = 4;                             // expand-add elements per thread
constexpr int FACE_EXP_ELEMS = FACE_EXP_EPT * FACE_THREADS;  // elements per expand-add item
constexpr int FACE_BATCH = 16;                 // loads issued before their FMAs
constexpr int FACE_SMEM_MAX = 220 * 1024;      // shared memory of one bilinear item
constexpr int FACE_MAXO = 4;                   // distinct operands of each kind per bilinear form

// in viewed as (pre, na, post) row-major; out_u[p * post + q] =
// alpha sum_k f_u[k fs] in[(p na + k) post + q].  post > 1: 64 outputs per
// item, the k range split over 4 thread slices whose sums are added in slice
// order; post == 1: one warp per output (8 per item).
struct ContrOp {
  const void* in;
  const void* f[FACE_MAXF];
  void* out[FACE_MAXF];
  i64 fs, pre, post;
  int na, nf;
  double alpha;
  const int* skip;
  i64 item_begin, items;
};

struct BilMat {  // element (r, c) = p[r rs + c cs]
  const void* p;
  i64 rs, cs;
};
// out[i ldo + j ocs] = sum_t alpha_t (A_ta[t] X_tx[t] B_tb[t]^T)(i, j), with
// A_k R x K1, X_k K1 x K2, B_k C x K2; items of FACE_RB rows.  With batch > 1
// the form is repeated for b < batch with every X advanced by b xbs elements
// and out by b obs.
struct BilOp {
  void* out;
  i64 ldo, ocs;
  int R, C, K1, K2;
  int batch;
  i64 xbs, obs;
  int nA, nX, nB, nt;
  BilMat A[FACE_MAXO], X[FACE_MAXO], B[FACE_MAXO];
  int ta[FACE_MAXT], tx[FACE_MAXT], tb[FACE_MAXT];
  double alpha[FACE_MAXT];
  const int* skip;
  i64 item_begin, items;
};

struct ExpTerm {
  const void* f;  // vector along `axis`, stride fs
  i64 fs;
  const void* Z;  // the other two axes, row-major
  int axis;
  double alpha;
};
// dst (d0 x d1 x d2 row-major, n elements): dst[e] = dst[e] + P_0[e] + ... +
// P_{np-1}[e] + sum_j alpha_j f_j[e_a] Z_j[e without a], added in that order.
// With zbs != 0, dst holds n / nper such grids (nper elements each) and grid
// r reads every Z_j advanced by r zbs; with zero, dst[e] starts from 0.
struct ExpAddOp {
  void* dst;
  i64 n, nper, zbs;
  int zero;
  int d1, d2;
  int vec;  // d2 % 4 == 0, dst, P, the Z of axes 0 / 1 16-byte aligned, pstride % 4 == 0
  const void* P;
  i64 pstride;
  int np, nj;
  ExpTerm j[FACE_MAXJ];
  const int* skip;
  i64 item_begin, items;
};

// op of a merged table that owns item `it` (tables sorted by item_begin)
template <typename Op>
__device__ __forceinline__ const Op& face_find(const Op* __restrict__ ops, int nops, i64 it) {
  int lo = 0, hi = nops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ops[mid].item_begin <= it) lo = mid; else hi = mid - 1;
  }
  return ops[lo];
}

constexpr int FACE_CQ = 64;  // outputs per contraction item (post > 1)
constexpr int FACE_CS = FACE_THREADS / FACE_CQ;  // k slices per output

// Every thread of the CTA calls this (it synchronises the CTA); red holds
// FACE_THREADS * FACE_MAXF elements.
template <typename T>
__device__ __forceinline__ void contr_item(const ContrOp& op, i64 item, T* red) {
  const int tid = threadIdx.x;
  const T* __restrict__ in = static_cast<const T*>(op.in);
  const int nf = op.nf;
  T acc[FACE_MAXF];
#pragma unroll
  for (int u = 0; u < FACE_MAXF; ++u) acc[u] = T(0);
  if (op.post > 1) {
    const int ql = tid % FACE_CQ, sl = tid / FACE_CQ;
    const unsigned o = (unsigned)(item * FACE_CQ) + ql;
    const bool live = o < (unsigned)(op.pre * op.post);
    const int kper = (op.na + FACE_CS - 1) / FACE_CS;
    const int k_lo = sl * kper, k_hi = min(op.na, k_lo + kper);
    if (live) {
      const unsigned post = (unsigned)op.post;
      const unsigned p = o / post, q = o - p * post;
      const T* __restrict__ base = in + ((i64)p * op.na) * op.post + q;
      for (int k0 = k_lo; k0 < k_hi; k0 += FACE_BATCH) {
        T v[FACE_BATCH], fv[FACE_MAXF][FACE_BATCH];
#pragma unroll
        for (int kk = 0; kk < FACE_BATCH; ++kk) {
          const bool ok = k0 + kk < k_hi;
          v[kk] = ok ? base[(i64)(k0 + kk) * op.post] : T(0);
#pragma unroll
          for (int u = 0; u < FACE_MAXF; ++u)
            fv[u][kk] = (ok && u < nf) ? static_cast<const T*>(op.f[u])[(i64)(k0 + kk) * op.fs] : T(0);
        }
#pragma unroll
        for (int kk = 0; kk < FACE_BATCH; ++kk)
#pragma unroll
          for (int u = 0; u < FACE_MAXF; ++u) acc[u] = fma(fv[u][kk], v[kk], acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < FACE_MAXF; ++u) red[u * FACE_THREADS + tid] = acc[u];
    __syncthreads();
    if (sl == 0 && live) {
#pragma unroll
      for (int u = 0; u < FACE_MAXF; ++u) {
        if (u >= nf) continue;
        T s = red[u * FACE_THREADS + ql];
        for (int k = 1; k < FACE_CS; ++k) s += red[u * FACE_THREADS + k * FACE_CQ + ql];
        static_cast<T*>(op.out[u])[o] = (T)op.alpha * s;
      }
    }
    __syncthreads();  // red is free again
  } else {
    const int lane = tid & 31;
    const i64 p = item * (FACE_THREADS / 32) + (tid >> 5);
    if (p >= op.pre) return;  // warp-uniform
    const T* __restrict__ row = in + p * op.na;
    for (int k = lane; k < op.na; k += 32) {
      const T v = row[k];
#pragma unroll
      for (int u = 0; u < FACE_MAXF; ++u)
        if (u < nf) acc[u] = fma(static_cast<const T*>(op.f[u])[(i64)k * op.fs], v, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < FACE_MAXF; ++u) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < FACE_MAXF; ++u)
        if (u < nf) static_cast<T*>(op.out[u])[p] = (T)op.alpha * acc[u];
    }
  }
}

// items of a contraction op
__host__ __device__ inline i64 contr_items(i64 pre, i64 post) {
  return post > 1 ? (pre * post + FACE_CQ - 1) / FACE_CQ : (pre + FACE_THREADS / 32 - 1) / (FACE_THREADS / 32);
}

// Host side: adds the term alpha A X B^T to a bilinear op, reusing equal
// operands; false if a limit is exceeded.
inline bool bil_add(BilOp& o, const BilMat& A, const BilMat& X, const BilMat& B, double alpha) {
  auto find = [](BilMat* v, int& n, const BilMat& m) -> int {
    for (int k = 0; k < n; ++k)
      if (v[k].p == m.p && v[k].rs == m.rs && v[k].cs == m.cs) return k;
    if (n >= FACE_MAXO) return -1;
    v[n] = m;
    return n++;
  };
  if (o.nt >= FACE_MAXT) return false;
  const int ia = find(o.A, o.nA, A), ix = find(o.X, o.nX, X), ib = find(o.B, o.nB, B);
  if (ia < 0 || ix < 0 || ib < 0) return false;
  o.ta[o.nt] = ia;
  o.tx[o.nt] = ix;
  o.tb[o.nt] = ib;
  o.alpha[o.nt] = alpha;
  ++o.nt;
  return true;
}

// Shared memory of a bilinear item, in elements: the distinct X (K1 x K2),
// B (C x K2, row stride K2 + 1 so that the lanes of a warp, which read
// different rows j, hit different banks) and A rows (FACE_RB x K1), and one
// P = A_rows X (FACE_RB x K2) per term.
__host__ __device__ inline i64 bilin_smem_elems(int C, int K1, int K2, int nA, int nX, int nB, int nt) {
  return (i64)nX * K1 * K2 + (i64)nB * C * (K2 + 1) + (i64)nA * FACE_RB * K1 + (i64)nt * FACE_RB * K2;
}

// dst[r ld + c] = src(r0 + r, c) for r < rows, c < cols (offsets fit 32
// bits), as cp.async copies (global -> shared without registers; the caller
// commits and waits), the unit-stride index fastest.  A thread's elements are
// FACE_THREADS apart, so its (r, c) advances by a fixed step (no division per
// element).
template <typename T>
__device__ __forceinline__ void face_stage(T* dst, int ld, const BilMat& m, int r0, int rows, int cols) {
  const T* __restrict__ src = static_cast<const T*>(m.p) + (i64)r0 * m.rs;
  const bool cfast = m.cs == 1 || m.rs != 1;
  const int n = rows * cols;
  const int nf = cfast ? cols : rows;          // extent of the fast index
  const int sf = cfast ? (int)m.cs : (int)m.rs, ss = cfast ? (int)m.rs : (int)m.cs;  // source strides (fast, slow)
  const int df = cfast ? 1 : ld, ds = cfast ? ld : 1;                                // destination strides
  const int tid = threadIdx.x;
  int slow = tid / nf, fast = tid - slow * nf;
  const int step_s = FACE_THREADS / nf, step_f = FACE_THREADS - step_s * nf;
  for (int e = tid; e < n; e += FACE_THREADS) {
    cp_async_el(dst + slow * ds + fast * df, src + slow * ss + fast * sf, true);
    fast += step_f;
    slow += step_s;
    if (fast >= nf) {
      fast -= nf;
      ++slow;
    }
  }
}

// Every thread of the CTA calls this (it synchronises the CTA): stage the
// distinct operands (all copies in flight together), form P_t = A_ta[t],rows
// X_tx[t] for every term, then
// out_rows = sum_t alpha_t P_t B_tb[t]^T.  Dot products run on four
// accumulators (fixed order).
template <typename T>
__device__ __forceinline__ void bilin_item(const BilOp& op, i64 item, T* sm) {
  const int tid = threadIdx.x;
  const int nrb = (op.R + FACE_RB - 1) / FACE_RB;
  const i64 bt = item / nrb;  // batch index
  const int i0 = (int)(item - bt * nrb) * FACE_RB;
  const int rows = min(FACE_RB, op.R - i0);
  const int C = op.C, K1 = op.K1, K2 = op.K2, nt = op.nt;
  const int lb = K2 + 1;
  T* Xs = sm;
  T* Bs = Xs + op.nX * K1 * K2;
  T* As = Bs + op.nB * C * lb;
  T* Ps = As + op.nA * FACE_RB * K1;
  __syncthreads();  // the buffers are free (previous item)
  for (int k = 0; k < op.nX; ++k) {
    BilMat xm = op.X[k];
    xm.p = static_cast<const T*>(xm.p) + bt * op.xbs;
    face_stage<T>(Xs + k * K1 * K2, K2, xm, 0, K1, K2);
  }
  for (int k = 0; k < op.nB; ++k) face_stage<T>(Bs + k * C * lb, lb, op.B[k], 0, C, K2);
  for (int k = 0; k < op.nA; ++k) face_stage<T>(As + k * FACE_RB * K1, K1, op.A[k], i0, rows, K1);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  // P_t(r, k2) = sum_k1 A(r, k1) X(k1, k2)
  for (int o = tid; o < nt * rows * K2; o += FACE_THREADS) {
    const int t = o / (rows * K2), rk = o - t * rows * K2;
    const int r = rk / K2, k2 = rk - r * K2;
    const T* __restrict__ a = As + op.ta[t] * FACE_RB * K1 + r * K1;
    const T* __restrict__ x = Xs + op.tx[t] * K1 * K2 + k2;
    T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
    int k1 = 0;
    for (; k1 + 3 < K1; k1 += 4) {
      s0 = fma(a[k1], x[k1 * K2], s0);
      s1 = fma(a[k1 + 1], x[(k1 + 1) * K2], s1);
      s2 = fma(a[k1 + 2], x[(k1 + 2) * K2], s2);
      s3 = fma(a[k1 + 3], x[(k1 + 3) * K2], s3);
    }
    for (; k1 < K1; ++k1) s0 = fma(a[k1], x[k1 * K2], s0);
    Ps[(t * FACE_RB + r) * K2 + k2] = (s0 + s1) + (s2 + s3);
  }
  __syncthreads();
  // out(i0 + r, j) = sum_t alpha_t sum_k2 P_t(r, k2) B(j, k2)
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int o = tid + h * FACE_THREADS;
    if (o < rows * C) {
      const int r = o / C, j = o - r * C;
      T acc = T(0);
      for (int t = 0; t < nt; ++t) {
        const T* __restrict__ pv = Ps + (t * FACE_RB + r) * K2;
        const T* __restrict__ bv = Bs + op.tb[t] * C * lb + j * lb;
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        int k2 = 0;
        for (; k2 + 3 < K2; k2 += 4) {
          s0 = fma(pv[k2], bv[k2], s0);
          s1 = fma(pv[k2 + 1], bv[k2 + 1], s1);
          s2 = fma(pv[k2 + 2], bv[k2 + 2], s2);
          s3 = fma(pv[k2 + 3], bv[k2 + 3], s3);
        }
        for (; k2 < K2; ++k2) s0 = fma(pv[k2], bv[k2], s0);
        acc = fma((T)op.alpha[t], (s0 + s1) + (s2 + s3), acc);
      }
      static_cast<T*>(op.out)[bt * op.obs + (i64)(i0 + r) * op.ldo + (i64)j * op.ocs] = acc;
    }
  }
}

template <typename T>
__device__ __forceinline__ void expadd_item_scalar(const ExpAddOp& op, i64 item) {
  T* __restrict__ dst = static_cast<T*>(op.dst);
  const T* __restrict__ P = static_cast<const T*>(op.P);
  const unsigned n = (unsigned)op.n, d1 = (unsigned)op.d1, d2 = (unsigned)op.d2;
  const unsigned base = (unsigned)(item * FACE_EXP_ELEMS) + threadIdx.x;
  const unsigned nper = (unsigned)op.nper;
  unsigned e[FACE_EXP_EPT], i0[FACE_EXP_EPT], i1[FACE_EXP_EPT], i2[FACE_EXP_EPT];
  i64 zo[FACE_EXP_EPT];
  T v[FACE_EXP_EPT];
#pragma unroll
  for (int q = 0; q < FACE_EXP_EPT; ++q) {
    e[q] = base + q * FACE_THREADS;
    const unsigned r = op.zbs ? e[q] / nper : 0u, el = e[q] - r * nper;
    zo[q] = (i64)r * op.zbs;
    const unsigned c01 = el / d2;
    i2[q] = el - c01 * d2;
    i0[q] = c01 / d1;
    i1[q] = c01 - i0[q] * d1;
    v[q] = (e[q] < n && !op.zero) ? dst[e[q]] : T(0);
  }
  for (int k = 0; k < op.np; ++k) {
    const T* __restrict__ pk = P + (i64)k * op.pstride;
#pragma unroll
    for (int q = 0; q < FACE_EXP_EPT; ++q)
      if (e[q] < n) v[q] += pk[e[q]];
  }
  for (int j = 0; j < op.nj; ++j) {
    const ExpTerm x = op.j[j];
    const T al = (T)x.alpha;
    const T* __restrict__ f = static_cast<const T*>(x.f);
    const T* __restrict__ Z = static_cast<const T*>(x.Z);
#pragma unroll
    for (int q = 0; q < FACE_EXP_EPT; ++q) {
      if (e[q] >= n) continue;
      unsigned ia, iz;
      if (x.axis == 0) { ia = i0[q]; iz = i1[q] * d2 + i2[q]; }
      else if (x.axis == 1) { ia = i1[q]; iz = i0[q] * d2 + i2[q]; }
      else { ia = i2[q]; iz = i0[q] * d1 + i1[q]; }
      v[q] = fma(al * f[(i64)ia * x.fs], Z[zo[q] + iz], v[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < FACE_EXP_EPT; ++q)
    if (e[q] < n) dst[e[q]] = v[q];
}

template <typename T>
__device__ __forceinline__ void face_ld4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}
template <typename T>
__device__ __forceinline__ void face_st4(T* p, const T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
}

// Four consecutive elements of one innermost row per thread, vector loads;
// every element is summed in the order of expadd_item_scalar.
template <typename T>
__device__ __forceinline__ void expadd_item_vec(const ExpAddOp& op, i64 item) {
  const unsigned n = (unsigned)op.n, d1 = (unsigned)op.d1, d2 = (unsigned)op.d2;
  const unsigned e0 = (unsigned)(item * FACE_EXP_ELEMS) + 4 * threadIdx.x;
  if (e0 >= n) return;
  T* __restrict__ dst = static_cast<T*>(op.dst);
  const T* __restrict__ P = static_cast<const T*>(op.P);
  const unsigned r = op.zbs ? e0 / (unsigned)op.nper : 0u, el = e0 - r * (unsigned)op.nper;
  const i64 zo = (i64)r * op.zbs;
  const unsigned c01 = el / d2, c2 = el - c01 * d2;
  const unsigned c0 = c01 / d1, c1 = c01 - c0 * d1;
  T v[4];
  if (op.zero) {
    v[0] = v[1] = v[2] = v[3] = T(0);
  } else {
    face_ld4(dst + e0, v);
  }
  for (int k = 0; k < op.np; ++k) {
    T w[4];
    face_ld4(P + (i64)k * op.pstride + e0, w);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] += w[q];
  }
  for (int j = 0; j < op.nj; ++j) {
    const ExpTerm x = op.j[j];
    const T al = (T)x.alpha;
    const T* __restrict__ f = static_cast<const T*>(x.f);
    const T* __restrict__ Z = static_cast<const T*>(x.Z) + zo;
    if (x.axis == 2) {
      const T z = Z[c0 * d1 + c1];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = fma(al * f[(i64)(c2 + q) * x.fs], z, v[q]);
    } else {
      const T fa = al * f[(i64)(x.axis == 0 ? c0 : c1) * x.fs];
      T z[4];
      face_ld4(Z + (x.axis == 0 ? c1 : c0) * d2 + c2, z);
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = fma(fa, z[q], v[q]);
    }
  }
  face_st4(dst + e0, v);
}

template <typename T>
__device__ __forceinline__ void expadd_item(const ExpAddOp& op, i64 item) {
  if (op.vec) expadd_item_vec<T>(op, item);
  else expadd_item_scalar<T>(op, item);
}

}  // namespace gpfvm
