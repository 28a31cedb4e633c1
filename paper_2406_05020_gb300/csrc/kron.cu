// Kronecker-structured products as plans of grouped FP64 GEMMs.
//
// A product  out = scale * sum_t c_t (F_t0 (x) F_t1 (x) F_t2) in  is the
// matrix-free form of Eq. kronecker-structure (Sec. 4.1): only the 1D factors
// are touched.  Mode products are shared between terms: with the axes taken
// in the order (p0, p1, p2),
//   level 1:  Y[u] = in x_{p0} F_u            for every distinct factor u on p0
//   level 2:  Z[w] = sum_{t: F_t,p2 = w} c_t  Y[u(t)] x_{p1} F_t,p1
//   level 3:  out  = scale * sum_w Z[w] x_{p2} F_w  (+ beta out + gamma D)
// For the three-term heat/wave operators this is 4 + 9 + 4 = 17 mode products
// per Gram matvec instead of 27.  The processing order puts the most
// shrinking axis first (dims_out/dims_in ascending), which matters for the
// rectangular PDE <-> point-set factors (e.g. cells -> the t = 0 grid).
#include <algorithm>
#include <map>

#include "kron.cuh"

namespace gpfvm {

static thread_local int g_tile_policy = -1;
void set_tile_policy(int policy) { g_tile_policy = (policy >= 0 && policy <= 2) ? policy : -1; }
int tile_policy() { return g_tile_policy; }

static int pick_tile(int m, i64 ctas_per_rowtile) {
  if (g_tile_policy >= 0) return g_tile_policy;
  // row tile 64/32/16: avoid padding waste for short factors, and keep at
  // least two waves of CTAs on the 152 SMs when the output is small
  if (m <= 16) return 2;
  if (m <= 32) return 1;
  if ((i64)ceil_div(m, 64) * ctas_per_rowtile >= 304) return 0;
  if ((i64)ceil_div(m, 32) * ctas_per_rowtile >= 304) return 1;
  return 2;
}

// out (dims with `ax` replaced by n_out) = sum over segs of alpha F x_ax in (+ beta out + gamma D)
void add_mode_gemm(Plan& plan, int d, const int* dims, int ax, int n_out, i64 batch,
                   const std::vector<std::pair<GemmGroup, std::vector<std::pair<MatRef, std::pair<const double*, double>>>>>& groups,
                   bool f32) {
  i64 pre = batch;
  for (int i = 0; i < ax; ++i) pre *= dims[i];
  const int n_in = dims[ax];
  i64 post = 1;
  for (int i = ax + 1; i < d; ++i) post *= dims[i];
  const MatRef F0 = groups[0].second[0].first;
  GemmDesc g{};
  std::vector<std::pair<GemmGroup, std::vector<GemmSeg>>> gs;
  if (post > 1) {
    // left multiplication: out[b] (n_out x post) = F (n_out x n_in) * in[b] (n_in x post)
    g.m = n_out; g.n = (int)post; g.k = n_in;
    g.a_rs = F0.rs; g.a_cs = F0.cs; g.a_bs = 0;
    g.b_rs = post; g.b_cs = 1; g.b_bs = (i64)n_in * post;
    g.c_rs = post; g.c_bs = (i64)n_out * post;
    g.d_rs = post; g.d_bs = (i64)n_out * post;
    g.batch = (int)pre;
    g.tile = pick_tile(n_out, ceil_div(post, 64) * pre * (i64)groups.size());
    for (auto& G : groups) {
      std::vector<GemmSeg> segs;
      for (auto& s : G.second) {
        if (s.first.rs != F0.rs || s.first.cs != F0.cs) throw CudaError{cudaErrorInvalidValue, "kron: stride mismatch"};
        segs.push_back(GemmSeg{s.first.p, s.second.first, s.second.second});
      }
      gs.push_back({G.first, segs});
    }
  } else {
    // right multiplication: out (pre x n_out) = in (pre x n_in) * F^T
    g.m = (int)pre; g.n = n_out; g.k = n_in;
    g.a_rs = n_in; g.a_cs = 1; g.a_bs = 0;
    g.b_rs = F0.cs; g.b_cs = F0.rs; g.b_bs = 0;
    g.c_rs = n_out; g.c_bs = 0;
    g.d_rs = n_out; g.d_bs = 0;
    g.batch = 1;
    g.tile = pick_tile((int)pre, ceil_div(n_out, 64) * (i64)groups.size());
    for (auto& G : groups) {
      std::vector<GemmSeg> segs;
      for (auto& s : G.second) {
        if (s.first.rs != F0.rs || s.first.cs != F0.cs) throw CudaError{cudaErrorInvalidValue, "kron: stride mismatch"};
        segs.push_back(GemmSeg{s.second.first, s.first.p, s.second.second});
      }
      gs.push_back({G.first, segs});
    }
  }
  g.tri = 0;
  g.f32 = f32 ? 1 : 0;
  plan.gemm(g, gs);
}

static bool same(const MatRef& a, const MatRef& b) { return a.p == b.p && a.rs == b.rs && a.cs == b.cs; }

void plan_kron(Plan& plan, Scratch& scratch, int d, const int* din, const int* dout, i64 batch,
               const std::vector<KTerm>& terms, double scale, const double* in, double* out, double beta,
               const double* D, double gamma, int* n_modeprods, bool f32) {
  if (terms.empty()) throw CudaError{cudaErrorInvalidValue, "kron: no terms"};
  // axis order: most shrinking first
  int order[3] = {0, 1, 2};
  std::stable_sort(order, order + d, [&](int a, int b) {
    return (double)dout[a] / din[a] < (double)dout[b] / din[b];
  });
  int count = 0;
  if (d == 1) {
    GemmGroup G{out, D, beta, gamma, 0, 0};
    std::vector<std::pair<MatRef, std::pair<const double*, double>>> segs;
    for (auto& t : terms) segs.push_back({t.f[0], {in, scale * t.c}});
    int dims[1] = {din[0]};
    add_mode_gemm(plan, 1, dims, 0, dout[0], batch, {{G, segs}}, f32);
    count = 1;
  } else {
    const int p0 = order[0], plast = order[d - 1];
    // level 1 (only for d == 3): distinct factors on p0
    std::vector<MatRef> U;
    std::vector<int> uidx(terms.size());
    std::vector<double*> Y;
    int dims1[3];
    for (int i = 0; i < d; ++i) dims1[i] = din[i];
    if (d == 3) {
      for (size_t t = 0; t < terms.size(); ++t) {
        int f = -1;
        for (size_t u = 0; u < U.size(); ++u)
          if (same(U[u], terms[t].f[p0])) f = (int)u;
        if (f < 0) { f = (int)U.size(); U.push_back(terms[t].f[p0]); }
        uidx[t] = f;
      }
      dims1[p0] = dout[p0];
      i64 sz = batch;
      for (int i = 0; i < 3; ++i) sz *= dims1[i];
      std::vector<std::pair<GemmGroup, std::vector<std::pair<MatRef, std::pair<const double*, double>>>>> gs;
      for (size_t u = 0; u < U.size(); ++u) {
        double* y = scratch.take(sz);
        Y.push_back(y);
        gs.push_back({GemmGroup{y, nullptr, 0.0, 0.0, 0, 0}, {{U[u], {in, 1.0}}}});
      }
      add_mode_gemm(plan, 3, din, p0, dout[p0], batch, gs, f32);
      count += (int)U.size();
    }
    // level 2: axis pm (middle for d == 3, first for d == 2), grouped by the factor on plast
    const int pm = (d == 3) ? order[1] : order[0];
    std::vector<MatRef> Wf;
    std::vector<std::vector<std::pair<MatRef, std::pair<const double*, double>>>> wsegs;
    for (size_t t = 0; t < terms.size(); ++t) {
      int w = -1;
      for (size_t k = 0; k < Wf.size(); ++k)
        if (same(Wf[k], terms[t].f[plast])) w = (int)k;
      if (w < 0) { w = (int)Wf.size(); Wf.push_back(terms[t].f[plast]); wsegs.emplace_back(); }
      const double* src = (d == 3) ? Y[uidx[t]] : in;
      bool merged = false;
      for (auto& s : wsegs[w])
        if (same(s.first, terms[t].f[pm]) && s.second.first == src) { s.second.second += terms[t].c; merged = true; }
      if (!merged) wsegs[w].push_back({terms[t].f[pm], {src, terms[t].c}});
    }
    int dims2[3];
    for (int i = 0; i < d; ++i) dims2[i] = dims1[i];
    dims2[pm] = dout[pm];
    i64 sz2 = batch;
    for (int i = 0; i < d; ++i) sz2 *= dims2[i];
    std::vector<double*> Z;
    std::vector<std::pair<GemmGroup, std::vector<std::pair<MatRef, std::pair<const double*, double>>>>> gs2;
    for (size_t w = 0; w < Wf.size(); ++w) {
      double* z = scratch.take(sz2);
      Z.push_back(z);
      gs2.push_back({GemmGroup{z, nullptr, 0.0, 0.0, 0, 0}, wsegs[w]});
      count += (int)wsegs[w].size();
    }
    add_mode_gemm(plan, d, dims1, pm, dout[pm], batch, gs2, f32);
    // level 3: last axis, one group summing over the distinct factors
    std::vector<std::pair<MatRef, std::pair<const double*, double>>> segs3;
    for (size_t w = 0; w < Wf.size(); ++w) segs3.push_back({Wf[w], {Z[w], scale}});
    add_mode_gemm(plan, d, dims2, plast, dout[plast], batch, {{GemmGroup{out, D, beta, gamma, 0, 0}, segs3}}, f32);
    count += (int)Wf.size();
  }
  if (n_modeprods) *n_modeprods += count;
}

}  // namespace gpfvm
