// CG / IterGP device state and launch helpers (see cg.cu).
#pragma once
#include "common.cuh"

namespace gpfvm {

constexpr int CG_MAX_PART = 1024;

struct CGState {
  double rr, bnorm2, rtol2, eta, alpha, beta;
  double aux[8];
  int k, done, converged, status, max_iter, cap;
  int pad[2];
  int loops;  // passes of the device-side iteration loop (reset by cg_init)
  int kbase;  // directions already stored when a run starts: cg_init sets k = kbase
  int nodown, pad3;  // nodown: the variance downdate of this run is skipped
  unsigned int ticket[8];
  double part[CG_MAX_PART];
};

int reduce_grid(i64 n);
// chunks of the reorthogonalisation dots (the partial-sum buffer holds cap x chunks)
int reorth_chunks(i64 n);
// row stride (elements) of the direction stores S and Q: n rounded up to 32
i64 store_ld(i64 n);
// r = p = b (scaled by 1/sqrt(*nrm2) when nrm2 is given; st->aux[7] keeps the
// inverse factor), x = 0, and the scalar header reset for a new run.
template <typename TB, typename T>
void cg_init(const TB* b, T* x, T* r, T* p, i64 n, CGState* st, cudaStream_t s, const double* nrm2 = nullptr,
             const int* skip = nullptr);
template <typename T>
void cg_dot_eta(const T* p, const T* q, i64 n, CGState* st, double* eta_hist, cudaStream_t s);
template <typename T>
void cg_downdate(const T* u, double* down, i64 n, const CGState* st, cudaStream_t s);
// x += alpha p, r -= alpha q (stores p, q as direction k), alpha = r.r/eta, or
// with gen = true alpha = p.r/eta (aux[5], from cg_dot_eta_pr): the step along
// a conjugate direction that was not built from r
template <typename T>
void cg_update(T* x, T* r, const T* p, const T* q, i64 n, CGState* st, T* S, T* Q, cudaStream_t s,
               bool gen = false);
template <typename T>
void cg_dot_eta_pr(const T* p, const T* q, const T* r, i64 n, CGState* st, double* eta_hist, cudaStream_t s);
template <typename T>
void cg_residual_wrt(const T* S, const T* Q, T* p, i64 n, int cap, CGState* st, double* part2, double* coef,
                     const double* eta_hist, cudaStream_t s);
template <typename T>
void cg_pupdate(const T* r, T* p, i64 n, const CGState* st, cudaStream_t s);
template <typename T>
void cg_reorth(const T* S, const T* Q, T* p, i64 n, int cap, CGState* st, double* part2, double* coef,
               const double* eta_hist, cudaStream_t s);
// Restart of a CG run that continues a G^-conjugate direction set (S, Q =
// G^ S, the st->k = kbase directions stored so far): Galerkin projection of the
// new residual r onto span S, i.e. d += S c and r -= Q c with c_j = s_j.r/eta_j;
// then p = r made conjugate to every stored direction and rr = r.r.
template <typename T>
void cg_project(const T* S, const T* Q, T* r, T* d, T* p, i64 n, int cap, CGState* st, double* part2,
                double* coef, const double* eta_hist, cudaStream_t s);
// Control node of a device-side CG loop (a graph WHILE node): one more pass
// while the CG state is not done, and never more than max_iter + 2 passes.
void loop_ctl(CGState* st, cudaGraphConditionalHandle h, cudaStream_t s);
// x += sign * (*scale) d  (scale defaults to 1)
void add_f2d(double* x, const float* d, i64 n, cudaStream_t s, const double* scale = nullptr, double sign = 1.0);
void f2d(const float* a, double* b, i64 n, cudaStream_t s);
void axpby(const double* a, const double* b, double* out, double sa, double sb, i64 n, cudaStream_t s);
void norm2(const double* v, i64 n, double* out, CGState* st, cudaStream_t s);
void var_final(const double* vB, const double* down, double* var, double s2, i64 n, cudaStream_t s);
void colsumsq(const double* Y, int rows, i64 cols, double* acc, cudaStream_t s);
void transpose(const double* A, double* B, int m, int n, cudaStream_t s);

// ---- variable coefficients: out = beta out + sum_t scale_t (f_t .* y_t) + gamma D
// (f_t null: 1); FP64 or FP32 (f32) data
constexpr int FIELD_MAXT = 8;
struct FieldTerms {
  const void* y[FIELD_MAXT];
  const void* f[FIELD_MAXT];
  double scale[FIELD_MAXT];
  int nt;
};
void field_combine(void* out, i64 n, const FieldTerms& t, const void* D, double gamma, double beta, bool f32,
                   cudaStream_t s);

// ---- multigrid warm start: coarse cells of `f`^d fine cells (row-major axes)
struct CoarseGeom {
  int d, f;
  int n[3], nc[3];
};
// p[i] = row[coarse(i)] (row != null) or the indicator of coarse cell c
void coarse_gather(double* p, i64 n, const CoarseGeom& g, const double* row, i64 c, cudaStream_t s);
// out[c' * stride] = sum of v over the fine cells of coarse cell c' (the restriction W^T v)
void coarse_restrict(const double* v, const CoarseGeom& g, double* out, i64 stride, cudaStream_t s);
// down += u .* u
void add_squares(double* down, const double* u, i64 n, cudaStream_t s);

// ---- device-driven mixed refinement (one graph per solve, see api.cu) ----
// The refinement decisions of the host-driven solver (residual test,
// divergence guard, run tolerance, conjugate continuation bookkeeping) taken
// on the device between the runs of an outer graph loop.
struct MixedCtl {
  // options
  double rtol, itol;
  int max_iter, icap_opt, cap32, cont, want_var, max_outer;
  // state
  double rel, rel_prev, tscale;
  int outer, total, kstore, idle, kbase;
  int first, stop, undo, status;  // status: 0 running, else a gpfvm_status
  long long inner_passes;
};
// control step after the FP64 residual (r, with ||r||^2 in s64->aux[0] and
// ||b||^2 in s64->aux[1]): decides stop / next run, writes the inner state
void mixed_ctl(MixedCtl* c, const CGState* s64, CGState* s32, cudaGraphConditionalHandle h_outer,
               cudaGraphConditionalHandle h_inner, cudaStream_t s);
// r = b - (first ? 0 : Gx), skipped once the solve stopped
void mixed_resid(const double* b, const double* gx, double* r, i64 n, const MixedCtl* c, cudaStream_t s);
// after a run: bookkeeping (iterations, stores, breakdown), then x += |r| d
// (or the undo of the last correction after a divergence)
void mixed_post(MixedCtl* c, CGState* s32, double* x, const float* d, i64 n, cudaGraphConditionalHandle h_outer,
                cudaStream_t s);

}  // namespace gpfvm
