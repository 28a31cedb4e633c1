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
void cg_init(const TB* b, T* x, T* r, T* p, i64 n, CGState* st, cudaStream_t s, const double* nrm2 = nullptr);
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

}  // namespace gpfvm
