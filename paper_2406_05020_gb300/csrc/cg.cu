// CG / IterGP iteration kernels (Sec. 4.1 "Iterative techniques", Sec. 4.2).
//
// Per iteration j (x0 = 0, r0 = p0 = b):
//   q = G^ p                           (structured matvec plan, also w = G_BB^-1 G_BP p)
//   eta_j = p.q                        (k_dot_eta)
//   u = Lhat k(X*)^T p,  down += u^2/eta_j   (IterGP combined-posterior downdate)
//   alpha = r.r/eta, x += alpha p, r -= alpha q, beta = r'.r'/r.r   (k_update)
//   p = r' + beta p                    (k_pupdate)
//   p -= sum_i (q_i.p / eta_i) p_i     (full reorthogonalisation, Sec. 7)
// All scalars live in device memory (CGState), so an iteration is a fixed
// launch sequence that a CUDA graph replays; reductions use a fixed-order
// "last block" sum so results do not depend on block scheduling.
#include <algorithm>

#include "cg.cuh"

namespace gpfvm {

constexpr int RT = 256;  // threads per reduction block

__device__ __forceinline__ bool last_block(unsigned int* ticket) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return am_last;
}

__device__ double sum_partials(const double* part, int n, double* smem) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += ((volatile const double*)part)[i];
  return block_sum<RT>(v, smem);
}

template <typename TB, typename T>
__global__ void __launch_bounds__(RT) k_init(const TB* __restrict__ b, T* __restrict__ x, T* __restrict__ r,
                                              T* __restrict__ p, i64 n, CGState* st, const double* nrm2,
                                              const int* skip) {
  pdl_wait();
  if (skip && *skip) return;
  __shared__ double red[32];
  // optional normalisation to a unit right-hand side (x0 = 0): b / ||b||
  double sc = 1.0;
  if (nrm2) {
    const double s = *nrm2;
    if (s > 0.0 && isfinite(s)) sc = 1.0 / sqrt(s);
  }
  double acc = 0.0;
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) {
    const T v = (T)(sc * (double)b[i]);
    x[i] = T(0);
    r[i] = v;
    p[i] = v;
    acc += (double)v * (double)v;
  }
  acc = block_sum<RT>(acc, red);
  if (threadIdx.x == 0) st->part[blockIdx.x] = acc;
  if (last_block(&st->ticket[0])) {
    const double s = sum_partials(st->part, gridDim.x, red);
    if (threadIdx.x == 0) {
      st->rr = s;
      st->bnorm2 = s;
      st->aux[7] = 1.0 / sc;  // undoes the normalisation of the solution
      st->k = st->kbase;
      st->loops = 0;
      st->status = 0;
      st->converged = (s == 0.0);
      st->done = (s == 0.0) || (st->max_iter <= 0);
      st->ticket[0] = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(RT) k_dot_eta(const T* __restrict__ p, const T* __restrict__ q, i64 n,
                                                 CGState* st, double* __restrict__ eta_hist) {
  pdl_wait();
  if (st->done) return;
  __shared__ double red[32];
  double acc = 0.0;
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT)
    acc = fma((double)p[i], (double)q[i], acc);
  acc = block_sum<RT>(acc, red);
  if (threadIdx.x == 0) st->part[blockIdx.x] = acc;
  if (last_block(&st->ticket[1])) {
    const double s = sum_partials(st->part, gridDim.x, red);
    if (threadIdx.x == 0) {
      st->eta = s;
      if (!(s > 0.0) || !isfinite(s)) {
        st->status |= DEV_BREAKDOWN;
        st->done = 1;
      } else if (st->k < st->cap) {
        eta_hist[st->k] = s;
      }
      st->ticket[1] = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(RT) k_downdate(const T* __restrict__ u, double* __restrict__ down, i64 n,
                                                  const CGState* st) {
  pdl_wait();
  if (st->done || st->nodown) return;
  const double inv = 1.0 / st->eta;
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) {
    const double v = (double)u[i];
    down[i] = fma(v * v, inv, down[i]);
  }
}

template <typename T>
__global__ void __launch_bounds__(RT) k_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                const T* __restrict__ q, i64 n, CGState* st, T* __restrict__ S,
                                                T* __restrict__ Q, i64 ld, int gen) {
  pdl_wait();
  if (st->done) return;
  __shared__ double red[32];
  // CG step r.r/eta; a general direction (not built from r) takes p.r/eta
  const double alpha = (gen ? st->aux[5] : st->rr) / st->eta;
  const int k = st->k;
  const bool keep = (S != nullptr) && (k < st->cap);
  double acc = 0.0;
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) {
    const T pi = p[i], qi = q[i];
    x[i] = (T)fma(alpha, (double)pi, (double)x[i]);
    const double ri = fma(-alpha, (double)qi, (double)r[i]);
    r[i] = (T)ri;
    acc = fma(ri, ri, acc);
    if (keep) {
      S[(i64)k * ld + i] = pi;
      Q[(i64)k * ld + i] = qi;
    }
  }
  acc = block_sum<RT>(acc, red);
  if (threadIdx.x == 0) st->part[blockIdx.x] = acc;
  if (last_block(&st->ticket[2])) {
    const double s = sum_partials(st->part, gridDim.x, red);
    if (threadIdx.x == 0) {
      st->alpha = alpha;
      st->beta = s / st->rr;
      st->rr = s;
      st->k = k + 1;
      if (!isfinite(s)) {
        st->status |= DEV_BREAKDOWN;
        st->done = 1;
      }
      if (s <= st->rtol2 * st->bnorm2) {
        st->converged = 1;
        st->done = 1;
      }
      if (k + 1 >= st->max_iter) st->done = 1;
      st->ticket[2] = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(RT) k_pupdate(const T* __restrict__ r, T* __restrict__ p, i64 n,
                                                 const CGState* st) {
  pdl_wait();
  if (st->done) return;
  const double beta = st->beta;
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT)
    p[i] = (T)fma(beta, (double)p[i], (double)r[i]);
}

// ---- full reorthogonalisation  p -= sum_j (q_j . p / eta_j) s_j  (Sec. 7)
// The direction stores hold one row of ld = store_ld(n) elements per
// direction (rows 16-byte aligned), so both kernels read them with 16-byte
// vector loads.  Chunk c of RCH elements of p stays in registers while each
// warp sweeps its share of the directions; per-lane partial dots are formed in
// the working precision, reduced across the warp and over chunks in FP64 in a
// fixed order (deterministic), and the last block turns the sums into the
// coefficients q_j.p / eta_j.
constexpr int RCH = 1024;  // elements of p per dots chunk

template <typename T>
__device__ __forceinline__ void ldv(const T* __restrict__ a, i64 e, i64 lim, T (&o)[16 / sizeof(T)]) {
  constexpr int W = 16 / sizeof(T);
  if (e + W <= lim) {
    if constexpr (sizeof(T) == 4) {
      const float4 v = *reinterpret_cast<const float4*>(a + e);
      o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
      const double2 v = *reinterpret_cast<const double2*>(a + e);
      o[0] = v.x; o[1] = v.y;
    }
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) o[w] = (e + w < lim) ? a[e + w] : T(0);
  }
}

template <typename T>
__global__ void __launch_bounds__(RT) k_reorth_dots(const T* __restrict__ Q, i64 ld, const T* __restrict__ p, i64 n,
                                                     CGState* st, double* __restrict__ part2,
                                                     const double* __restrict__ eta_hist, double* __restrict__ coef) {
  pdl_wait();
  if (st->done) return;
  constexpr int W = 16 / sizeof(T);
  constexpr int NV = RCH / (32 * W);  // vectors per lane
  const int k = min(st->k, st->cap);
  const int c = blockIdx.x, nchunk = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const i64 base = (i64)c * RCH;
  T pv[NV][W];
#pragma unroll
  for (int v = 0; v < NV; ++v) ldv(p, base + (i64)(v * 32 + lane) * W, n, pv[v]);
  // four directions per warp at a time: eight independent FMA chains per lane
  // (the FP64 FMA pipe, not HBM, bounds this kernel on parts with a low FP64 rate)
  const int wstride = gridDim.y * (RT / 32);
  for (int j0 = (blockIdx.y * (RT / 32) + warp) * 4; j0 < k; j0 += wstride * 4) {
    const T* __restrict__ qj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) qj[u] = Q + (i64)min(j0 + u, k - 1) * ld;
    T a[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u][0] = a[u][1] = T(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T qv[4][W];
#pragma unroll
      for (int u = 0; u < 4; ++u) ldv(qj[u], base + (i64)(v * 32 + lane) * W, n, qv[u]);
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u][w & 1] = fma(qv[u][w], pv[v][w], a[u][w & 1]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      double sum = (double)a[u][0] + (double)a[u][1];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0 && j0 + u < k) part2[(i64)(j0 + u) * nchunk + c] = sum;
    }
  }
}

// coef_j = (sum over chunks of part2[j][.]) / eta_j, one block per direction
// (the chunk sums are added in a fixed order: deterministic)
__global__ void __launch_bounds__(RT) k_reorth_coef(const CGState* st, int nchunk, const double* __restrict__ part2,
                                                     const double* __restrict__ eta_hist, double* __restrict__ coef) {
  pdl_wait();
  if (st->done) return;
  const int j = blockIdx.x;
  if (j >= min(st->k, st->cap)) return;
  __shared__ double red[32];
  const double* __restrict__ row = part2 + (i64)j * nchunk;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int cc = threadIdx.x;
  for (; cc + 3 * RT < nchunk; cc += 4 * RT) {
    a0 += row[cc];
    a1 += row[cc + RT];
    a2 += row[cc + 2 * RT];
    a3 += row[cc + 3 * RT];
  }
  for (; cc < nchunk; cc += RT) a0 += row[cc];
  const double sum = block_sum<RT>((a0 + a1) + (a2 + a3), red);
  if (threadIdx.x == 0) coef[j] = sum / eta_hist[j];
}

template <typename T>
__global__ void __launch_bounds__(RT) k_reorth_apply(const T* __restrict__ S, i64 ld, T* __restrict__ p, i64 n,
                                                      const CGState* st, const double* __restrict__ coef,
                                                      double sgn) {
  pdl_wait();
  if (st->done) return;
  constexpr int W = 16 / sizeof(T);
  __shared__ T cs[1024];
  const int k = min(st->k, st->cap);
  const i64 e = ((i64)blockIdx.x * RT + threadIdx.x) * W;
  T acc0[W], acc1[W];
#pragma unroll
  for (int w = 0; w < W; ++w) acc0[w] = acc1[w] = T(0);
  for (int j0 = 0; j0 < k; j0 += 1024) {
    const int jn = min(1024, k - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < jn; t += RT) cs[t] = (T)(sgn * coef[j0 + t]);
    __syncthreads();
    if (e < n) {
      const T* __restrict__ Sj = S + (i64)j0 * ld;
      int j = 0;
      for (; j + 1 < jn; j += 2) {
        T s0[W], s1[W];
        ldv(Sj + (i64)j * ld, e, n, s0);
        ldv(Sj + (i64)(j + 1) * ld, e, n, s1);
        const T c0 = cs[j], c1 = cs[j + 1];
#pragma unroll
        for (int w = 0; w < W; ++w) {
          acc0[w] = fma(s0[w], c0, acc0[w]);
          acc1[w] = fma(s1[w], c1, acc1[w]);
        }
      }
      if (j < jn) {
        T s0[W];
        ldv(Sj + (i64)j * ld, e, n, s0);
#pragma unroll
        for (int w = 0; w < W; ++w) acc0[w] = fma(s0[w], cs[j], acc0[w]);
      }
    }
  }
  if (e < n) {
    T pv[W];
    ldv(p, e, n, pv);
#pragma unroll
    for (int w = 0; w < W; ++w)
      if (e + w < n) p[e + w] = pv[w] - (acc0[w] + acc1[w]);
  }
}

// ---------------------------------------------------------------------------
int reduce_grid(i64 n) {
  int g = ceil_div(n, RT * 4);
  if (g > 1024) g = 1024;
  if (g < 1) g = 1;
  return g;
}

template <typename TB, typename T>
void cg_init(const TB* b, T* x, T* r, T* p, i64 n, CGState* st, cudaStream_t s, const double* nrm2,
             const int* skip) {
  launch_pdl(k_init<TB, T>, reduce_grid(n), RT, 0, s, b, x, r, p, n, st, nrm2, skip);
}
template <typename T>
void cg_dot_eta(const T* p, const T* q, i64 n, CGState* st, double* eta_hist, cudaStream_t s) {
  launch_pdl(k_dot_eta<T>, reduce_grid(n), RT, 0, s, p, q, n, st, eta_hist);
}
template <typename T>
void cg_downdate(const T* u, double* down, i64 n, const CGState* st, cudaStream_t s) {
  launch_pdl(k_downdate<T>, ceil_div(n, RT), RT, 0, s, u, down, n, st);
}
template <typename T>
void cg_update(T* x, T* r, const T* p, const T* q, i64 n, CGState* st, T* S, T* Q, cudaStream_t s, bool gen) {
  launch_pdl(k_update<T>, reduce_grid(n), RT, 0, s, x, r, p, q, n, st, S, Q, store_ld(n), gen ? 1 : 0);
}

// eta = p.q (into the history, as k_dot_eta) and aux[5] = p.r in one pass
template <typename T>
__global__ void __launch_bounds__(RT) k_dot_eta_pr(const T* __restrict__ p, const T* __restrict__ q,
                                                    const T* __restrict__ r, i64 n, CGState* st,
                                                    double* __restrict__ eta_hist) {
  pdl_wait();
  if (st->done) return;
  __shared__ double red[32];
  double a = 0.0, b = 0.0;
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) {
    const double pi = (double)p[i];
    a = fma(pi, (double)q[i], a);
    b = fma(pi, (double)r[i], b);
  }
  a = block_sum<RT>(a, red);
  b = block_sum<RT>(b, red);
  if (threadIdx.x == 0) {
    st->part[blockIdx.x] = a;
    st->part[CG_MAX_PART / 2 + blockIdx.x] = b;
  }
  if (last_block(&st->ticket[6])) {
    const double sa = sum_partials(st->part, gridDim.x, red);
    const double sb = sum_partials(st->part + CG_MAX_PART / 2, gridDim.x, red);
    if (threadIdx.x == 0) {
      st->eta = sa;
      st->aux[5] = sb;
      if (!(sa > 0.0) || !isfinite(sa) || !isfinite(sb)) {
        st->status |= DEV_BREAKDOWN;
        st->done = 1;
      } else if (st->k < st->cap) {
        eta_hist[st->k] = sa;
      }
      st->ticket[6] = 0;
    }
  }
}
template <typename T>
void cg_dot_eta_pr(const T* p, const T* q, const T* r, i64 n, CGState* st, double* eta_hist, cudaStream_t s) {
  launch_pdl(k_dot_eta_pr<T>, std::min(reduce_grid(n), CG_MAX_PART / 2), RT, 0, s, p, q, r, n, st, eta_hist);
}

// p -= Q c with c_j = s_j . p / eta_j: the residual of the system G^ z = p with
// respect to the inverse approximation C = sum_j s_j s_j^T / eta_j (p - G^ C p)
template <typename T>
void cg_residual_wrt(const T* S, const T* Q, T* p, i64 n, int cap, CGState* st, double* part2, double* coef,
                     const double* eta_hist, cudaStream_t s) {
  const i64 ld = store_ld(n);
  reorth_coefs(S, (const T*)p, n, cap, st, part2, coef, eta_hist, s);
  launch_pdl(k_reorth_apply<T>, ceil_div(n, RT * (16 / (int)sizeof(T))), RT, 0, s, Q, ld, p, n, st, coef, 1.0);
}
template <typename T>
void cg_pupdate(const T* r, T* p, i64 n, const CGState* st, cudaStream_t s) {
  launch_pdl(k_pupdate<T>, ceil_div(n, RT), RT, 0, s, r, p, n, st);
}
i64 store_ld(i64 n) { return (n + 31) / 32 * 32; }
int reorth_chunks(i64 n) {
  const i64 c = (n + RCH - 1) / RCH;
  return c < 1 ? 1 : (int)c;
}
// partial dots Q^T p per chunk, then the coefficients (one block per direction)
template <typename T>
void reorth_coefs(const T* Q, const T* p, i64 n, int cap, CGState* st, double* part2, double* coef,
                  const double* eta_hist, cudaStream_t s) {
  const i64 ld = store_ld(n);
  const int nchunk = reorth_chunks(n);
  // split the directions (in groups of four per warp) over blockIdx.y until
  // about four CTAs per SM are busy
  int gy = (4 * 152 + nchunk - 1) / nchunk;
  gy = std::max(1, std::min(gy, ceil_div(cap, 4 * (RT / 32))));
  launch_pdl(k_reorth_dots<T>, dim3(nchunk, gy), RT, 0, s, Q, ld, p, n, st, part2, eta_hist, coef);
  if (cap > 0) launch_pdl(k_reorth_coef, cap, RT, 0, s, (const CGState*)st, nchunk, (const double*)part2, eta_hist, coef);
}

template <typename T>
void cg_reorth(const T* S, const T* Q, T* p, i64 n, int cap, CGState* st, double* part2, double* coef,
               const double* eta_hist, cudaStream_t s) {
  const i64 ld = store_ld(n);
  reorth_coefs(Q, (const T*)p, n, cap, st, part2, coef, eta_hist, s);
  launch_pdl(k_reorth_apply<T>, ceil_div(n, RT * (16 / (int)sizeof(T))), RT, 0, s, S, ld, p, n, st, coef, 1.0);
}

// p = r, rr = r.r (bnorm2 is kept: the run's tolerance stays relative to its
// right-hand side before the projection)
template <typename T>
__global__ void __launch_bounds__(RT) k_restart(const T* __restrict__ r, T* __restrict__ p, i64 n, CGState* st) {
  pdl_wait();
  if (st->done) return;
  __shared__ double red[32];
  double acc = 0.0;
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) {
    const T v = r[i];
    p[i] = v;
    acc = fma((double)v, (double)v, acc);
  }
  acc = block_sum<RT>(acc, red);
  if (threadIdx.x == 0) st->part[blockIdx.x] = acc;
  if (last_block(&st->ticket[5])) {
    const double s = sum_partials(st->part, gridDim.x, red);
    if (threadIdx.x == 0) {
      st->rr = s;
      if (!isfinite(s)) {
        st->status |= DEV_BREAKDOWN;
        st->done = 1;
      } else if (s <= st->rtol2 * st->bnorm2) {
        st->converged = 1;
        st->done = 1;
      }
      st->ticket[5] = 0;
    }
  }
}

template <typename T>
void cg_project(const T* S, const T* Q, T* r, T* d, T* p, i64 n, int cap, CGState* st, double* part2,
                double* coef, const double* eta_hist, cudaStream_t s) {
  const i64 ld = store_ld(n);
  const int ga = ceil_div(n, RT * (16 / (int)sizeof(T)));
  // c_j = s_j . r / eta_j  (the dots with the directions in place of Q)
  reorth_coefs(S, (const T*)r, n, cap, st, part2, coef, eta_hist, s);
  launch_pdl(k_reorth_apply<T>, ga, RT, 0, s, Q, ld, r, n, st, coef, 1.0);   // r -= Q c
  launch_pdl(k_reorth_apply<T>, ga, RT, 0, s, S, ld, d, n, st, coef, -1.0);  // d += S c
  launch_pdl(k_restart<T>, reduce_grid(n), RT, 0, s, r, p, n, st);
  cg_reorth(S, Q, p, n, cap, st, part2, coef, eta_hist, s);
}

#define GPFVM_CG_INST(T)                                                                                    \
  template void cg_dot_eta<T>(const T*, const T*, i64, CGState*, double*, cudaStream_t);                   \
  template void cg_downdate<T>(const T*, double*, i64, const CGState*, cudaStream_t);                      \
  template void cg_update<T>(T*, T*, const T*, const T*, i64, CGState*, T*, T*, cudaStream_t, bool);       \
  template void cg_dot_eta_pr<T>(const T*, const T*, const T*, i64, CGState*, double*, cudaStream_t);        \
  template void cg_residual_wrt<T>(const T*, const T*, T*, i64, int, CGState*, double*, double*,             \
                                   const double*, cudaStream_t);                                             \
  template void cg_pupdate<T>(const T*, T*, i64, const CGState*, cudaStream_t);                            \
  template void cg_reorth<T>(const T*, const T*, T*, i64, int, CGState*, double*, double*, const double*,       \
                             cudaStream_t);                                                                 \
  template void cg_project<T>(const T*, const T*, T*, T*, T*, i64, int, CGState*, double*, double*,          \
                              const double*, cudaStream_t);
GPFVM_CG_INST(double)
GPFVM_CG_INST(float)
template void cg_init<double, double>(const double*, double*, double*, double*, i64, CGState*, cudaStream_t,
                                      const double*, const int*);
template void cg_init<double, float>(const double*, float*, float*, float*, i64, CGState*, cudaStream_t,
                                     const double*, const int*);

// ---- small vector helpers -------------------------------------------------
__global__ void k_axpby(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                        double sa, double sb, i64 n) {
  pdl_wait();
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) out[i] = sa * a[i] + sb * b[i];
}
void axpby(const double* a, const double* b, double* out, double sa, double sb, i64 n, cudaStream_t s) {
  if (n <= 0) return;
  int g = ceil_div(n, RT);
  if (g > 4096) g = 4096;
  launch_pdl(k_axpby, g, RT, 0, s, a, b, out, sa, sb, n);
}

__global__ void k_norm2(const double* __restrict__ v, i64 n, double* out, double* part, unsigned int* ticket) {
  pdl_wait();
  __shared__ double red[32];
  double acc = 0.0;
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) acc = fma(v[i], v[i], acc);
  acc = block_sum<RT>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
  if (last_block(ticket)) {
    const double s = sum_partials(part, gridDim.x, red);
    if (threadIdx.x == 0) {
      *out = s;
      *ticket = 0;
    }
  }
}
void norm2(const double* v, i64 n, double* out, CGState* st, cudaStream_t s) {
  launch_pdl(k_norm2, reduce_grid(n), RT, 0, s, v, n, out, st->part, &st->ticket[3]);
}

__global__ void k_loop_ctl(CGState* st, cudaGraphConditionalHandle h) {
  pdl_wait();
  const int n = ++st->loops;
  const int lim = min(max(st->max_iter, 0), 1 << 24) + 2;  // bounded whatever the CG state holds
  cudaGraphSetConditional(h, (!st->done && n < lim) ? 1u : 0u);
}
void loop_ctl(CGState* st, cudaGraphConditionalHandle h, cudaStream_t s) {
  launch_pdl(k_loop_ctl, 1, 1, 0, s, st, h);
}

__global__ void k_add_f2d(double* __restrict__ x, const float* __restrict__ d, i64 n, const double* scale,
                          double sign) {
  pdl_wait();
  const double a = sign * (scale ? *scale : 1.0);
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) x[i] = fma(a, (double)d[i], x[i]);
}
void add_f2d(double* x, const float* d, i64 n, cudaStream_t s, const double* scale, double sign) {
  if (n <= 0) return;
  int g = ceil_div(n, RT);
  if (g > 4096) g = 4096;
  launch_pdl(k_add_f2d, g, RT, 0, s, x, d, n, scale, sign);
}

__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, i64 n) {
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) b[i] = (double)a[i];
}
void f2d(const float* a, double* b, i64 n, cudaStream_t s) {
  if (n <= 0) return;
  int g = ceil_div(n, RT);
  if (g > 4096) g = 4096;
  k_f2d<<<g, RT, 0, s>>>(a, b, n);
  GPFVM_LAUNCH_CHECK();
}

// var = outputscale - vB - down
__global__ void k_var_final(const double* __restrict__ vB, const double* __restrict__ down, double* __restrict__ var,
                            double s2, i64 n) {
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT)
    var[i] = s2 - (vB ? vB[i] : 0.0) - (down ? down[i] : 0.0);
}
void var_final(const double* vB, const double* down, double* var, double s2, i64 n, cudaStream_t s) {
  if (n <= 0) return;
  int g = ceil_div(n, RT);
  if (g > 4096) g = 4096;
  k_var_final<<<g, RT, 0, s>>>(vB, down, var, s2, n);
  GPFVM_LAUNCH_CHECK();
}

// acc[j] += sum_{i < rows} Y[i][j]^2   (column sums of squares, fixed order over i)
__global__ void k_colsumsq(const double* __restrict__ Y, int rows, i64 cols, double* __restrict__ acc) {
  const i64 j = (i64)blockIdx.x * RT + threadIdx.x;
  if (j >= cols) return;
  double s0 = 0.0, s1 = 0.0;
  int i = 0;
  for (; i + 1 < rows; i += 2) {
    const double a = Y[(i64)i * cols + j], b = Y[(i64)(i + 1) * cols + j];
    s0 = fma(a, a, s0);
    s1 = fma(b, b, s1);
  }
  if (i < rows) {
    const double a = Y[(i64)i * cols + j];
    s0 = fma(a, a, s0);
  }
  acc[j] += s0 + s1;
}
void colsumsq(const double* Y, int rows, i64 cols, double* acc, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  k_colsumsq<<<ceil_div(cols, RT), RT, 0, s>>>(Y, rows, cols, acc);
  GPFVM_LAUNCH_CHECK();
}

__global__ void k_transpose(const double* __restrict__ A, double* __restrict__ B, int m, int n) {
  __shared__ double t[32][33];
  const int x = blockIdx.x * 32 + threadIdx.x, y0 = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += 8)
    if (x < n && y0 + yy < m) t[yy][threadIdx.x] = A[(i64)(y0 + yy) * n + x];
  __syncthreads();
  const int xo = y0 + threadIdx.x;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int yo = blockIdx.x * 32 + yy;
    if (xo < m && yo < n) B[(i64)yo * m + xo] = t[threadIdx.x][yy];
  }
}
void transpose(const double* A, double* B, int m, int n, cudaStream_t s) {
  if (m <= 0 || n <= 0) return;
  k_transpose<<<dim3(ceil_div(n, 32), ceil_div(m, 32)), dim3(32, 8), 0, s>>>(A, B, m, n);
  GPFVM_LAUNCH_CHECK();
}

// ---- variable coefficients ------------------------------------------------
template <typename T>
__global__ void k_field_combine(T* __restrict__ out, i64 n, const FieldTerms t, const T* __restrict__ D,
                                double gamma, double beta) {
  pdl_wait();
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) {
    double v = beta != 0.0 ? beta * (double)out[i] : 0.0;
    for (int k = 0; k < t.nt; ++k) {
      const double y = (double)((const T*)t.y[k])[i];
      const double f = t.f[k] ? (double)((const T*)t.f[k])[i] : 1.0;
      v = fma(t.scale[k] * f, y, v);
    }
    if (D) v = fma(gamma, (double)D[i], v);
    out[i] = (T)v;
  }
}
void field_combine(void* out, i64 n, const FieldTerms& t, const void* D, double gamma, double beta, bool f32,
                   cudaStream_t s) {
  if (n <= 0) return;
  int g = ceil_div(n, RT);
  if (g > 4096) g = 4096;
  if (f32) launch_pdl(k_field_combine<float>, g, RT, 0, s, (float*)out, n, t, (const float*)D, gamma, beta);
  else launch_pdl(k_field_combine<double>, g, RT, 0, s, (double*)out, n, t, (const double*)D, gamma, beta);
}

// ---- multigrid warm start --------------------------------------------------
__device__ __forceinline__ i64 coarse_index(i64 i, const CoarseGeom& g) {
  i64 c = 0, mul = 1;
  for (int a = g.d - 1; a >= 0; --a) {
    const i64 k = i % g.n[a];
    i /= g.n[a];
    c += (k / g.f) * mul;
    mul *= g.nc[a];
  }
  return c;
}
__global__ void k_coarse_gather(double* __restrict__ p, i64 n, const CoarseGeom g, const double* __restrict__ row,
                                i64 c) {
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) {
    const i64 ci = coarse_index(i, g);
    p[i] = row ? row[ci] : (ci == c ? 1.0 : 0.0);
  }
}
void coarse_gather(double* p, i64 n, const CoarseGeom& g, const double* row, i64 c, cudaStream_t s) {
  int gr = ceil_div(n, RT);
  if (gr > 4096) gr = 4096;
  k_coarse_gather<<<gr, RT, 0, s>>>(p, n, g, row, c);
  GPFVM_LAUNCH_CHECK();
}
// one thread per coarse cell, its f^d fine cells summed in a fixed order
__global__ void k_coarse_restrict(const double* __restrict__ v, const CoarseGeom g, double* __restrict__ out,
                                  i64 stride, i64 nc) {
  const i64 c = (i64)blockIdx.x * RT + threadIdx.x;
  if (c >= nc) return;
  int cc[3] = {0, 0, 0};
  i64 r = c;
  for (int a = g.d - 1; a >= 0; --a) {
    cc[a] = (int)(r % g.nc[a]);
    r /= g.nc[a];
  }
  const int f0 = g.f, f1 = g.d > 1 ? g.f : 1, f2 = g.d > 2 ? g.f : 1;
  double acc = 0.0;
  for (int a = 0; a < f0; ++a)
    for (int b = 0; b < f1; ++b)
      for (int e = 0; e < f2; ++e) {
        int k[3] = {cc[0] * g.f + a, g.d > 1 ? cc[1] * g.f + b : 0, g.d > 2 ? cc[2] * g.f + e : 0};
        i64 i = 0;
        for (int ax = 0; ax < g.d; ++ax) i = i * g.n[ax] + k[ax];
        acc += v[i];
      }
  out[c * stride] = acc;
}
void coarse_restrict(const double* v, const CoarseGeom& g, double* out, i64 stride, cudaStream_t s) {
  i64 nc = 1;
  for (int a = 0; a < g.d; ++a) nc *= g.nc[a];
  k_coarse_restrict<<<ceil_div(nc, RT), RT, 0, s>>>(v, g, out, stride, nc);
  GPFVM_LAUNCH_CHECK();
}
__global__ void k_add_squares(double* __restrict__ down, const double* __restrict__ u, i64 n) {
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) down[i] = fma(u[i], u[i], down[i]);
}
void add_squares(double* down, const double* u, i64 n, cudaStream_t s) {
  int gr = ceil_div(n, RT);
  if (gr > 4096) gr = 4096;
  k_add_squares<<<gr, RT, 0, s>>>(down, u, n);
  GPFVM_LAUNCH_CHECK();
}

// ---- device-driven mixed refinement --------------------------------------
__global__ void k_mixed_ctl(MixedCtl* c, const CGState* s64, CGState* s32, cudaGraphConditionalHandle ho,
                            cudaGraphConditionalHandle hi) {
  pdl_wait();
  if (c->stop) {  // never reached with a live loop; keeps a stray pass inert
    cudaGraphSetConditional(hi, 0u);
    cudaGraphSetConditional(ho, 0u);
    return;
  }
  const double b2 = s64->aux[1];
  double rel = b2 > 0.0 ? sqrt(s64->aux[0] / b2) : 0.0;
  int stop = 0, status = 0;
  if (s32->pad[1] & DEV_TIMEOUT) {
    stop = 1; status = -6;
  } else if (!isfinite(rel)) {
    stop = 1; status = -4;
  } else if (c->outer > 0 && rel > 10.0 * c->rel_prev) {  // divergence: undo the last correction
    stop = 1; status = 1;
    c->undo = 1;
    rel = c->rel_prev;
  } else {
    c->rel_prev = rel;
    if (rel <= c->rtol || (c->cont && c->outer > 0 && c->tscale >= 1.0 && rel <= 2.0 * c->rtol)) {
      stop = 1; status = 0;
    } else if (c->total >= c->max_iter || c->idle >= 3 || c->outer >= c->max_outer) {
      stop = 1; status = 1;
    } else {
      if (c->outer > 0 && rel <= 2.0 * c->rtol) c->tscale *= 0.5;
      const int kbase = c->cont ? c->kstore : 0;
      const int run_cap = min(c->icap_opt, c->max_iter - c->total);
      const int icap = max(1, min(c->cap32 - kbase, run_cap));
      const double itol = fmax(c->itol, rel > 0.0 ? c->tscale * c->rtol / rel : c->itol);
      s32->rtol2 = itol * itol;
      s32->max_iter = kbase + icap;
      s32->cap = c->cap32;
      s32->kbase = kbase;
      s32->nodown = (c->want_var && (c->cont || c->outer == 0)) ? 0 : 1;
      s32->pad[1] = 0;
      c->kbase = kbase;
    }
  }
  c->rel = rel;
  c->stop = stop;
  if (stop) {
    c->status = status == 0 ? 0 : (status == 1 ? 1 : status);
    s32->done = 1;
  }
  cudaGraphSetConditional(hi, stop ? 0u : 1u);
  cudaGraphSetConditional(ho, stop ? 0u : 1u);
}
void mixed_ctl(MixedCtl* c, const CGState* s64, CGState* s32, cudaGraphConditionalHandle h_outer,
               cudaGraphConditionalHandle h_inner, cudaStream_t s) {
  launch_pdl(k_mixed_ctl, 1, 1, 0, s, c, s64, s32, h_outer, h_inner);
}

__global__ void k_mixed_resid(const double* __restrict__ b, const double* __restrict__ gx, double* __restrict__ r,
                              i64 n, const MixedCtl* c) {
  pdl_wait();
  if (c->stop) return;
  const bool first = c->first != 0;
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT)
    r[i] = first ? b[i] : b[i] - gx[i];
}
void mixed_resid(const double* b, const double* gx, double* r, i64 n, const MixedCtl* c, cudaStream_t s) {
  int g = ceil_div(n, RT);
  if (g > 4096) g = 4096;
  launch_pdl(k_mixed_resid, g, RT, 0, s, b, gx, r, n, c);
}

// one thread: bookkeeping of the finished run (before the x update)
__global__ void k_mixed_count(MixedCtl* c, CGState* s32, cudaGraphConditionalHandle ho) {
  c->first = 0;
  if (c->stop) return;
  const int k = s32->k - s32->kbase;
  c->total += k;
  c->inner_passes += s32->loops;
  if (c->cont) c->kstore = min(s32->k, c->cap32);
  if (k == 0 && !s32->converged) {  // not even one inner step
    c->stop = 1;
    c->status = -4;
    cudaGraphSetConditional(ho, 0u);
    return;
  }
  c->idle = k == 0 ? c->idle + 1 : 0;
  c->outer += 1;
}
__global__ void k_mixed_xupd(const MixedCtl* c, const CGState* s32, double* __restrict__ x,
                             const float* __restrict__ d, i64 n) {
  pdl_wait();
  if (c->stop && !c->undo) return;
  const double a = (c->undo ? -1.0 : 1.0) * s32->aux[7];
  for (i64 i = (i64)blockIdx.x * RT + threadIdx.x; i < n; i += (i64)gridDim.x * RT) x[i] = fma(a, (double)d[i], x[i]);
}
void mixed_post(MixedCtl* c, CGState* s32, double* x, const float* d, i64 n, cudaGraphConditionalHandle h_outer,
                cudaStream_t s) {
  // a plain launch: its predecessor in the graph is the inner loop's conditional node
  k_mixed_count<<<1, 1, 0, s>>>(c, s32, h_outer);
  GPFVM_LAUNCH_CHECK();
  int g = ceil_div(n, RT);
  if (g > 4096) g = 4096;
  launch_pdl(k_mixed_xupd, g, RT, 0, s, (const MixedCtl*)c, (const CGState*)s32, x, d, n);
}

}  // namespace gpfvm
