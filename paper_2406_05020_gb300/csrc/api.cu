// C ABI of the GP-FVM hot path: problem setup, assembly, solve, query.
//
// Data layout in device memory (all FP64, row-major, axis order t, x, y):
//   coordinates   cell edges per axis, point-set coordinates, prediction grid
//   factors       every 1D covariance factor the problem needs (one buffer)
//   A, L, Linv, LinvT   M x M IC/BC Gram, its Cholesky factor and inverse factor
//   b, x, r, p, q        N-vectors of the deflated CG
//   g, t, w              M-vectors (G_BP p, L^-1 g, G_BB^-1 G_BP p)
//   S, Q                 cap x N stored directions p_j and G^ p_j (reorthogonalisation)
//   u, down, mean, var, vB   P-vectors on the prediction grid
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <deque>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <memory>
#include <tuple>
#include <type_traits>

#include "cg.cuh"
#include "kron.cuh"
#include "oz.cuh"
#include "tc.cuh"

using namespace gpfvm;

namespace gpfvm {
static std::atomic<long long> g_launches{0};
void count_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace gpfvm

namespace {

// An IC/BC point set: a tensor grid of points observing the derivative of
// the given order on each axis.  Two given sets that differ only in the order
// on axis 0, where both sit at one common coordinate (u and u_t at t = 0 of a
// second-order-in-time problem), are held as one "stacked" set with two
// axis-0 points at that coordinate: point 0 with order[0] and noise, point 1
// with order2 and noise2.  Their joint covariance is then one Kronecker
// product (the axis-0 factor becomes 2 x 2), so the structured IC/BC stage
// inverts both through one eigenbasis instead of placing the second in the
// Schur complement.  Layouts agree: axis 0 is the slowest, so the stacked
// set's values are the first set's followed by the second's.
struct SetC {
  int comp = 0;         // the output component observed (systems, Sec. 3.3)
  int order[3] = {0, 0, 0};
  int order2 = -1;      // axis-0 order of point 1 of a stacked set (else -1)
  double noise2 = 0.0;  // its noise variance
  int n[3] = {1, 1, 1};
  std::vector<double> coords[3];
  std::vector<double> values;
  double noise = 0.0;
  i64 off = 0, size = 0;
};

// Factor key: axis, family A (kind, arg), family B (kind, arg).
// kind 0 = cell family with derivative order arg, 1 = point set arg, 2 = prediction grid.
typedef std::tuple<int, int, int, int, int> FKey;

struct DevBuf {
  std::vector<void*> ptrs;
  std::vector<i64> sizes;
  i64 bytes = 0;
  template <typename T>
  T* alloc(i64 n) {
    if (n <= 0) return nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      throw CudaError{cudaErrorMemoryAllocation, "cudaMalloc"};
    }
    ptrs.push_back(p);
    sizes.push_back(n * (i64)sizeof(T));
    bytes += n * (i64)sizeof(T);
    return (T*)p;
  }
  // true if [p, p + len) lies inside one allocation
  bool contains(const void* p, i64 len) const {
    const char* c = (const char*)p;
    for (size_t i = 0; i < ptrs.size(); ++i) {
      const char* b = (const char*)ptrs[i];
      if (c >= b && c + len <= b + sizes[i]) return true;
    }
    return false;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    sizes.clear();
    bytes = 0;
  }
};

// Host-side bounds check of every GEMM/GEMV operand of a plan against the
// problem's allocations, done once when the plan is built (before any launch).
void check_plan_ranges(const Plan& plan, const DevBuf& mem, const char* name) {
  for (auto& b : plan.bgs) check_plan_ranges(*b, mem, name);
  auto need = [&](const void* p, i64 len, const char* what) {
    if (!p || len <= 0) return;
    if (!mem.contains(p, len)) {
      fprintf(stderr, "gpfvm: plan %s: %s operand out of bounds\n", name, what);
      throw CudaError{cudaErrorInvalidValue, "plan operand out of bounds"};
    }
  };
  for (const PlanOp& op : plan.ops) {
    if (op.kind == PlanOp::GEMM) {
      const GemmDesc& g = op.g;
      const i64 e = g.f32 ? 4 : 8;
      const i64 nb = (i64)g.batch - 1;
      for (int gi = 0; gi < g.n_groups; ++gi) {
        const GemmGroup& G = plan.groups[op.group0 + gi];
        need(G.C, e * (nb * g.c_bs + (i64)(g.m - 1) * g.c_rs + g.n), "C");
        need(G.D, e * (nb * g.d_bs + (i64)(g.m - 1) * g.d_rs + g.n), "D");
        for (int si = 0; si < G.nseg; ++si) {
          const GemmSeg& S = plan.segs[G.seg0 + si];
          need(S.A, e * (nb * g.a_bs + (i64)(g.m - 1) * g.a_rs + (i64)(g.k - 1) * g.a_cs + 1), "A");
          need(S.B, e * (nb * g.b_bs + (i64)(g.k - 1) * g.b_rs + (i64)(g.n - 1) * g.b_cs + 1), "B");
        }
      }
    } else if (op.kind == PlanOp::GEMV || op.kind == PlanOp::GEMV32) {
      const i64 e = op.kind == PlanOp::GEMV32 ? 4 : 8;
      need(op.A, e * ((i64)(op.m - 1) * op.lda + op.n), "gemv A");
      need(op.x, e * op.n, "gemv x");
      need(op.y, e * op.m, "gemv y");
      need(op.z, e * op.m, "gemv z");
      need(op.zs, 8 * op.m, "gemv zs");
    } else if (op.kind == PlanOp::COPY) {
      need(op.cp_dst, op.cp_bytes, "copy dst");
      need(op.cp_src, op.cp_bytes, "copy src");
    } else if (op.kind == PlanOp::CONTR) {
      const ContrOp& o = op.fco;
      const i64 e = op.fc_f32 ? 4 : 8;
      need(o.in, e * o.pre * o.na * o.post, "contr in");
      for (int k = 0; k < o.nf; ++k) {
        need(o.f[k], e * ((i64)(o.na - 1) * o.fs + 1), "contr f");
        need(o.out[k], e * o.pre * o.post, "contr out");
      }
    } else if (op.kind == PlanOp::BILIN) {
      const BilOp& o = op.fbo;
      const i64 e = op.fc_f32 ? 4 : 8;
      if (o.R > FACE_MAXN || o.C > FACE_MAXN || o.K1 > FACE_MAXN || o.K2 > FACE_MAXN || o.nt > FACE_MAXT)
        throw CudaError{cudaErrorInvalidValue, "plan: bilinear form too large"};
      const i64 nb = std::max(o.batch, 1) - 1;
      need(o.out, e * (nb * o.obs + (i64)(o.R - 1) * o.ldo + (i64)(o.C - 1) * o.ocs + 1), "bilin out");
      if (o.nA > FACE_MAXO || o.nX > FACE_MAXO || o.nB > FACE_MAXO)
        throw CudaError{cudaErrorInvalidValue, "plan: bilinear form too large"};
      for (int k = 0; k < o.nA; ++k)
        need(o.A[k].p, e * ((i64)(o.R - 1) * o.A[k].rs + (i64)(o.K1 - 1) * o.A[k].cs + 1), "bilin A");
      for (int k = 0; k < o.nX; ++k)
        need(o.X[k].p, e * (nb * o.xbs + (i64)(o.K1 - 1) * o.X[k].rs + (i64)(o.K2 - 1) * o.X[k].cs + 1), "bilin X");
      for (int k = 0; k < o.nB; ++k)
        need(o.B[k].p, e * ((i64)(o.C - 1) * o.B[k].rs + (i64)(o.K2 - 1) * o.B[k].cs + 1), "bilin B");
      for (int k = 0; k < o.nt; ++k)
        if (o.ta[k] < 0 || o.ta[k] >= o.nA || o.tx[k] < 0 || o.tx[k] >= o.nX || o.tb[k] < 0 || o.tb[k] >= o.nB)
          throw CudaError{cudaErrorInvalidValue, "plan: bilinear term operand out of range"};
    } else if (op.kind == PlanOp::EXPADD) {
      const ExpAddOp& o = op.feo;
      const i64 e = op.fc_f32 ? 4 : 8;
      if (o.nj > FACE_MAXJ) throw CudaError{cudaErrorInvalidValue, "plan: too many expansion terms"};
      need(o.dst, e * o.n, "expadd dst");
      need(o.P, e * ((i64)(o.np - 1) * o.pstride + o.n), "expadd parts");
      if (o.nper <= 0 || o.n % o.nper != 0) throw CudaError{cudaErrorInvalidValue, "plan: expand-add batch"};
      const i64 d0 = o.nper / ((i64)o.d1 * o.d2), nbz = o.n / o.nper - 1;
      for (int k = 0; k < o.nj; ++k) {
        const ExpTerm& t = o.j[k];
        const i64 na = t.axis == 0 ? d0 : (t.axis == 1 ? o.d1 : o.d2);
        need(t.f, e * ((na - 1) * t.fs + 1), "expadd f");
        need(t.Z, e * (nbz * o.zbs + o.nper / na), "expadd Z");
      }
    }
  }
}

int map_error(const CudaError& e) {
  static const bool trace = [] {
    const char* v = getenv("GPFVM_DEBUG");
    return v && std::atoi(v) != 0;
  }();
  if (trace) fprintf(stderr, "gpfvm: %s failed: %s\n", e.where ? e.where : "?", cudaGetErrorString(e.err));
  if (e.err == cudaErrorMemoryAllocation) return GPFVM_ERR_OUT_OF_MEMORY;
  if (e.err == cudaErrorInvalidValue) return GPFVM_ERR_INVALID_ARG;
  return GPFVM_ERR_DEVICE;
}

}  // namespace

struct gpfvm_problem {
  // ---- descriptor copy
  int d = 0;
  int nc[3] = {1, 1, 1};
  std::vector<double> edges[3];
  double ell[3] = {1, 1, 1};
  double s2 = 1.0, jitter = 0.0;
  int nterms = 0;
  int alpha[GPFVM_MAX_TERMS][3] = {};
  double coef[GPFVM_MAX_TERMS] = {};
  std::vector<double> rhs;
  int nsets = 0;
  SetC sets[GPFVM_MAX_SETS];
  // systems (Sec. 3.3): neq equations over nout independent outputs; term a
  // belongs to equation teq[a] and differentiates output tout[a].  PDE vectors
  // hold neq blocks of Nc cells, predictions nout blocks of Pp points.
  bool multi = false;
  int neq = 1, nout = 1;
  int teq[GPFVM_MAX_TERMS] = {}, tout[GPFVM_MAX_TERMS] = {};
  i64 Nc = 0, Pp = 0;
  // the caller's sets: set u is internal set uset[u], and with uslice[u] >= 0
  // the axis-0 point uslice[u] of that stacked set
  int nusets = 0;
  int uset[GPFVM_MAX_SETS] = {}, uslice[GPFVM_MAX_SETS] = {};
  int npred[3] = {1, 1, 1};
  std::vector<double> pred[3];
  bool colloc = false;  // PDE observed at the cell centres (collocation) instead of cell integrals
  // variable coefficients: term a's coefficient is coef[a] * field[fclass[a]] per cell (fclass -1:
  // constant); the distinct fields live in d_field / f_field (nfield x N)
  int nfield = 0;
  int fclass[GPFVM_MAX_TERMS];  // set to -1 for every term at creation
  std::vector<double> fields;
  double* d_field = nullptr;
  float* f_field = nullptr;
  i64 N = 0, M = 0, P = 0;
  int cap = 0;

  // ---- device memory
  DevBuf mem;
  double* d_coords = nullptr;
  i64 off_edges[3] = {0, 0, 0}, off_pred[3] = {0, 0, 0}, off_set[GPFVM_MAX_SETS][3] = {}, off_mid[3] = {0, 0, 0};
  double* d_fac = nullptr;
  std::map<FKey, i64> fac_off;
  std::vector<FactorJob> jobs;
  FactorJob* d_jobs = nullptr;
  i64 max_entries = 0;
  double *d_A = nullptr, *d_L = nullptr, *d_Linv = nullptr, *d_LinvT = nullptr, *d_cscr = nullptr;
  double *d_yB = nullptr, *d_rhs = nullptr, *d_b = nullptr;
  double *d_x = nullptr, *d_r = nullptr, *d_p = nullptr, *d_q = nullptr;
  double *d_g = nullptr, *d_t = nullptr, *d_w = nullptr, *d_g2 = nullptr;
  double *d_u = nullptr, *d_down = nullptr, *d_mean = nullptr, *d_var = nullptr, *d_vB = nullptr;
  double *d_S = nullptr, *d_Q = nullptr, *d_eta = nullptr, *d_part2 = nullptr, *d_coef = nullptr;
  double *d_vin = nullptr, *d_vout = nullptr, *d_win = nullptr, *d_wout = nullptr;
  double *d_vbchunk = nullptr, *d_vbY = nullptr;
  double* d_tbeta = nullptr;  // weights of one targeted action on the prediction grid (P)
  // mixed precision (FP32 inner operator)
  float *f_fac = nullptr, *f_Linv = nullptr, *f_LinvT = nullptr;
  float *f_p = nullptr, *f_q = nullptr, *f_r = nullptr, *f_d = nullptr, *f_g = nullptr, *f_t = nullptr,
        *f_w = nullptr, *f_u = nullptr, *f_S = nullptr, *f_Q = nullptr, *f_vin = nullptr, *f_vout = nullptr;
  double* d_eta32 = nullptr;
  // structured IC/BC stage: set 0 inverted through its Kronecker eigen-structure,
  // the other sets through the Schur complement S (see icbc.cu)
  bool sicbc = false;
  int MK = 0, MR = 0, nK[3] = {1, 1, 1};
  double *d_QK[3] = {}, *d_lam[3] = {}, *d_lt = nullptr, *d_ltinv = nullptr;
  // E~ = G_RK (x)Q Lambda~^-1 (MR x MK) and its transpose; set 0's parts of the
  // solve vectors are coordinates in the eigenbasis (x)Q_i
  double *d_Tsc = nullptr, *d_Et = nullptr, *d_EtT = nullptr, *d_Sc = nullptr, *d_LS = nullptr,
         *d_LSinv = nullptr, *d_LSinvT = nullptr, *d_sscr = nullptr, *d_R = nullptr;
  double *d_tR = nullptr, *d_uR = nullptr, *d_Hsq[3] = {}, *d_yBt = nullptr;
  float *f_QK[3] = {}, *f_Et = nullptr, *f_EtT = nullptr, *f_LSinv = nullptr, *f_LSinvT = nullptr, *f_tR = nullptr,
        *f_uR = nullptr;
  // set-0 factors with the eigenbasis multiplied in: F_i Q_i (cells x set 0)
  // under the key of F_i, Q_i^T C_i (set 0 x prediction grid) under that of C_i
  std::map<FKey, i64> facq_off;
  double* d_facq = nullptr;
  float* f_facq = nullptr;
  i64 nfacq = 0;
  JacobiJob* d_jac = nullptr;
  unsigned int* d_psync = nullptr;  // grid-barrier words of the persistent plan kernel
  int* d_jac_sweeps = nullptr;  // 2 per axis: FP32 and FP64 sweeps of the last assembly
  // tensor-core G_PP (split TF32): factor splits, rotated intermediates, op tables
  bool tc_ok = false;
  int tc_mode = -1;  // operator of the inner CG: -1 FP32 SIMT, else the TcMode of the tensor-core G_PP
  float* f_tcsplit = nullptr;
  float *f_tcY = nullptr, *f_tcZ = nullptr;
  float* f_tcpart = nullptr;  // partial sums of split tensor-core tiles
  i64 tc_part_total = 0;      // floats f_tcpart needs (largest level)
  std::vector<std::tuple<i64, float, i64, i64, int>> tc_jobs;  // (factor offset in f_fac, alpha, size, split offset, mode)
  TcOp* d_tcops = nullptr;
  struct TcLevel {
    int off, nops, maxn;
    i64 tiles;
    int any_split;
  };
  std::vector<TcLevel> tc_levels[6];  // instance 2 m + 0: f_p -> f_q, 2 m + 1: f_vin -> f_vout (TcMode m)
  i64 tc_split_total = 0, tc_ops_total = 0;
  int tc_nu = 0, tc_nw = 0;
  // FP64 G_PP on the tensor cores by exact digit products (oz.cu): factor digit
  // images, rotated FP64 intermediates, row exponents, op tables per instance
  // (0: d_p -> d_q of the CG plans, 1: d_vin -> d_vout, 2: the same for the
  // refinement residual, skipped with it)
  bool oz_ok = false;   // every axis <= 128 cells, constant coefficients
  bool oz_on = true;    // the FP64 CG and residual plans use it (desc fp64_products == 0)
  struct OzJob { i64 fac_off; int n; double alpha; i64 img_off, fexp_off; };
  std::vector<OzJob> oz_jobs;
  struct OzLevel { int off, nops; i64 tiles; OzExpJobs jobs; int n; };  // n: the level's outputs per row (uniform)
  std::vector<OzLevel> oz_levels[3];
  OzOp* d_ozops = nullptr;
  unsigned char* d_ozimg = nullptr;
  int* d_ozfexp = nullptr;
  int* d_ozexp = nullptr;
  double *d_ozY = nullptr, *d_ozZ = nullptr;
  i64 oz_ops_total = 0, oz_img_total = 0, oz_fexp_total = 0, oz_exp_total = 0;
  int oz_nu = 0, oz_nw = 0;
  int* d_ozgexp = nullptr;  // window exponents of the digit-product dense GEMMs (2 x ozg_cap ints)
  i64 ozg_cap = 0;
  // digit-product forms of other FP64 Kronecker chains (Builder::kron_digits):
  // op tables, factor images (strided views) and their slicing jobs
  struct OzxJob { const double* F; i64 rs, cs; int N, K; double alpha; i64 img_off, fexp_off; };
  std::vector<OzxJob> ozx_jobs;
  std::map<std::tuple<const double*, i64, i64, int, int, double>, std::pair<i64, i64>> ozx_img;
  std::vector<OzOp> ozx_ops;
  OzOp* d_ozxops = nullptr;
  unsigned char* d_ozximg = nullptr;
  int* d_ozxfexp = nullptr;
  i64 ozx_ops_cap = 0, ozx_img_n = 0, ozx_fexp_n = 0;
  int cap64 = 0, cap32 = 0;  // directions the allocated stores hold
  CGState* d_st32 = nullptr;
  CGState* h_st32 = nullptr;
  i64 nfac = 0;
  bool building_f32 = false;
  double* d_scratch = nullptr;
  i64 scratch_cap = 0;
  int vb_rows = 0;
  CGState* d_st = nullptr;
  CGState* h_st = nullptr;  // pinned mirror of the scalar header
  MixedCtl* d_mctl = nullptr;  // device-driven refinement state (batch graph)
  MixedCtl* h_mctl = nullptr;  // its pinned mirror

  // ---- plans
  Plan p_setup, p_chol, p_rhs, p_mv_cg, p_var_cg, p_mean, p_vB, p_tgt;
  Plan p_res;  // G^ x for the FP64 residual of the device-driven refinement (skipped on its first pass)
  Plan p_op[6];  // ops 0-3, then 12 / 13 (G_PP / G^ with the digit-product G_PP)
  Plan p_mv32, p_var32, p_pp32, p_mvv_cg, p_mvv32;
  Plan p_mv32tc[3], p_mvv32tc[3], p_pp32tc[3];  // per TcMode
  int modeprods_pp = 0;
  Fan fan;  // side streams for the independent launches of a plan phase
  // GPFVM_HOST_LOOP=1: the host replays the captured iteration pass by pass
  // instead of a device-side WHILE loop (same kernels; for per-kernel profilers,
  // which see kernels inside conditional graph bodies only as one workload)
  bool host_loop = false;

  // ---- state
  bool assembled = false, solved = false, vB_ready = false, want_var_last = false;
  cudaGraphExec_t graph = nullptr;
  int graph_key = -1;
  long long graph_kernels = 0;
  cudaGraphExec_t graph32 = nullptr;
  int graph32_key = -1;
  long long graph32_kernels = 0;
  gpfvm_solve_info last{};
  int last_outer = 0;
  int tuned_tile = -1, tuned_tc = 0;  // plan policies chosen by gpfvm_autotune
  int last_store = 0;   // directions of the last solve: 0 none, 1 FP64 store, 2 FP32 store
  int last_kstore = 0;  // how many

  ~gpfvm_problem() {
    fan.destroy();
    if (graph) cudaGraphExecDestroy(graph);
    if (graph32) cudaGraphExecDestroy(graph32);
    if (h_st) cudaFreeHost(h_st);
    if (h_st32) cudaFreeHost(h_st32);
    if (h_mctl) cudaFreeHost(h_mctl);
    if (d_S) cudaFree(d_S);
    if (d_Q) cudaFree(d_Q);
    if (f_S) cudaFree(f_S);
    if (f_Q) cudaFree(f_Q);
    mem.release();
  }
};

namespace {


i64 fam_n(const gpfvm_problem* p, int ax, int kind, int arg) {
  if (kind == 0) return p->nc[ax];
  if (kind == 1) return p->sets[arg].n[ax];
  return p->npred[ax];
}

// Stack consecutive given sets s, s + 1 that differ only in the derivative
// order on axis 0 and sit at one common axis-0 coordinate (see SetC), unless
// GPFVM_STACK_SETS=0.  Offsets and the order of the M values are unchanged.
void stack_sets(gpfvm_problem* p) {
  const char* env = std::getenv("GPFVM_STACK_SETS");
  if ((env && std::atoi(env) == 0) || p->d < 2) return;
  auto stackable = [&](const SetC& a, const SetC& b) {
    if (a.n[0] != 1 || b.n[0] != 1 || a.coords[0][0] != b.coords[0][0] || a.order[0] == b.order[0]) return false;
    if (a.comp != b.comp) return false;
    for (int i = 1; i < p->d; ++i)
      if (a.n[i] != b.n[i] || a.order[i] != b.order[i] || a.coords[i] != b.coords[i]) return false;
    return true;
  };
  int ns = 0;
  for (int u = 0; u < p->nusets;) {
    SetC& out = p->sets[ns];
    if (u + 1 < p->nusets && stackable(p->sets[u], p->sets[u + 1])) {
      SetC a = p->sets[u];
      const SetC& b = p->sets[u + 1];
      a.n[0] = 2;
      a.coords[0] = {a.coords[0][0], a.coords[0][0]};
      a.order2 = b.order[0];
      a.noise2 = b.noise;
      a.values.insert(a.values.end(), b.values.begin(), b.values.end());
      a.size *= 2;
      p->uset[u] = p->uset[u + 1] = ns;
      p->uslice[u] = 0;
      p->uslice[u + 1] = 1;
      out = std::move(a);
      u += 2;
    } else {
      if (&out != &p->sets[u]) out = std::move(p->sets[u]);
      p->uset[u] = ns;
      p->uslice[u] = -1;
      u += 1;
    }
    ++ns;
  }
  for (int s = ns; s < p->nsets; ++s) p->sets[s] = SetC();
  p->nsets = ns;
}

void need_factor(gpfvm_problem* p, int ax, int ka, int aa, int kb, int ab) {
  FKey key(ax, ka, aa, kb, ab);
  if (p->fac_off.count(key)) return;
  FactorJob J{};
  // family kinds of the kernel: 0 = cell integrals, 1 = points (collocation
  // observes the PDE families at the cell centres, with their derivative order)
  J.kind_a = (ka == 0 && !p->colloc) ? 0 : 1;
  J.kind_b = (kb == 0 && !p->colloc) ? 0 : 1;
  J.ord_a = ka == 0 ? aa : (ka == 1 ? p->sets[aa].order[ax] : 0);
  J.ord_b = kb == 0 ? ab : (kb == 1 ? p->sets[ab].order[ax] : 0);
  if (ka == 1 && ax == 0 && p->sets[aa].order2 >= 0) {
    J.has2_a = 1;
    J.ord2_a = p->sets[aa].order2;
  }
  if (kb == 1 && ax == 0 && p->sets[ab].order2 >= 0) {
    J.has2_b = 1;
    J.ord2_b = p->sets[ab].order2;
  }
  J.n_a = (int)fam_n(p, ax, ka, aa);
  J.n_b = (int)fam_n(p, ax, kb, ab);
  J.ell = p->ell[ax];
  i64 off = 0;
  for (auto& j : p->jobs) off += (i64)j.n_a * j.n_b;
  p->fac_off[key] = off;
  // coordinate pointers are patched once the coordinate buffer exists
  J.ca = (const double*)(intptr_t)(ka * 1000 + aa);
  J.cb = (const double*)(intptr_t)(kb * 1000 + ab);
  J.out = (double*)(intptr_t)off;
  p->jobs.push_back(J);
  p->max_entries = std::max(p->max_entries, (i64)J.n_a * J.n_b);
}

MatRef fac_ref(const gpfvm_problem* p, int ax, int ka, int aa, int kb, int ab, bool transpose) {
  const i64 off = p->fac_off.at(FKey(ax, ka, aa, kb, ab));
  const i64 nb = fam_n(p, ax, kb, ab);
  MatRef m{p->building_f32 ? (const double*)(p->f_fac + off) : p->d_fac + off, nb, 1};
  if (transpose) std::swap(m.rs, m.cs);
  return m;
}

// Terms of G_PP: pairs of operator terms, factor per axis A_i^{a_i b_i}.
std::vector<KTerm> pp_terms(const gpfvm_problem* p) {
  std::vector<KTerm> ts;
  for (int a = 0; a < p->nterms; ++a)
    for (int b = 0; b < p->nterms; ++b) {
      KTerm t{};
      t.c = p->coef[a] * p->coef[b];
      for (int i = 0; i < p->d; ++i) t.f[i] = fac_ref(p, i, 0, p->alpha[a][i], 0, p->alpha[b][i], false);
      ts.push_back(t);
    }
  return ts;
}

// Factors of set 0 with its eigenbasis multiplied in (structured IC/BC stage):
// F_i Q_i for cells x set 0, Q_i^T C_i for set 0 x prediction grid.
MatRef facq_ref(const gpfvm_problem* p, int ax, int ka, int aa, int kb, int ab, bool transpose) {
  const i64 off = p->facq_off.at(FKey(ax, ka, aa, kb, ab));
  const i64 nb = fam_n(p, ax, kb, ab);
  MatRef m{p->building_f32 ? (const double*)(p->f_facq + off) : p->d_facq + off, nb, 1};
  if (transpose) std::swap(m.rs, m.cs);
  return m;
}

// cells -> set s (transpose=true) or set s -> cells (transpose=false); with
// fold, set 0 of the structured stage in its eigenbasis
std::vector<KTerm> pb_terms(const gpfvm_problem* p, int s, bool to_set, bool fold = false) {
  const bool q = fold && s == 0 && p->sicbc;
  std::vector<KTerm> ts;
  for (int a = 0; a < p->nterms; ++a) {
    KTerm t{};
    t.c = p->coef[a];
    for (int i = 0; i < p->d; ++i)
      t.f[i] = q ? facq_ref(p, i, 0, p->alpha[a][i], 1, s, to_set) : fac_ref(p, i, 0, p->alpha[a][i], 1, s, to_set);
    ts.push_back(t);
  }
  return ts;
}

std::vector<KTerm> ppred_terms(const gpfvm_problem* p) {
  std::vector<KTerm> ts;
  for (int a = 0; a < p->nterms; ++a) {
    KTerm t{};
    t.c = p->coef[a];
    for (int i = 0; i < p->d; ++i) t.f[i] = fac_ref(p, i, 0, p->alpha[a][i], 2, 0, true);
    ts.push_back(t);
  }
  return ts;
}

// prediction grid -> cells (the adjoint of ppred_terms)
std::vector<KTerm> predp_terms(const gpfvm_problem* p) {
  std::vector<KTerm> ts;
  for (int a = 0; a < p->nterms; ++a) {
    KTerm t{};
    t.c = p->coef[a];
    for (int i = 0; i < p->d; ++i) t.f[i] = fac_ref(p, i, 0, p->alpha[a][i], 2, 0, false);
    ts.push_back(t);
  }
  return ts;
}

// prediction grid -> set s (the adjoint of bpred_terms; fold: set 0 in its eigenbasis)
std::vector<KTerm> predb_terms(const gpfvm_problem* p, int s, bool fold = false) {
  const bool q = fold && s == 0 && p->sicbc;
  KTerm t{};
  t.c = 1.0;
  for (int i = 0; i < p->d; ++i) t.f[i] = q ? facq_ref(p, i, 1, s, 2, 0, false) : fac_ref(p, i, 1, s, 2, 0, false);
  return {t};
}

// ---- variable coefficients: terms grouped by field class (-1 = constant)
std::vector<int> field_classes(const gpfvm_problem* p) {
  std::vector<int> c;
  for (int a = 0; a < p->nterms; ++a)
    if (std::find(c.begin(), c.end(), p->fclass[a]) == c.end()) c.push_back(p->fclass[a]);
  std::sort(c.begin(), c.end());
  return c;
}
template <typename F>
std::vector<KTerm> class_terms(const std::vector<KTerm>& all, const gpfvm_problem* p, int cls, F term_of) {
  std::vector<KTerm> out;
  for (size_t t = 0; t < all.size(); ++t)
    if (p->fclass[term_of(t)] == cls) out.push_back(all[t]);
  return out;
}
// G_PP pairs (a, b) with field classes (P, Q)
std::vector<KTerm> pp_terms_pq(const gpfvm_problem* p, int P, int Q) {
  std::vector<KTerm> ts;
  for (int a = 0; a < p->nterms; ++a)
    for (int b = 0; b < p->nterms; ++b) {
      if (p->fclass[a] != P || p->fclass[b] != Q) continue;
      KTerm t{};
      t.c = p->coef[a] * p->coef[b];
      for (int i = 0; i < p->d; ++i) t.f[i] = fac_ref(p, i, 0, p->alpha[a][i], 0, p->alpha[b][i], false);
      ts.push_back(t);
    }
  return ts;
}

std::vector<KTerm> bpred_terms(const gpfvm_problem* p, int s, bool fold = false) {
  const bool q = fold && s == 0 && p->sicbc;
  KTerm t{};
  t.c = 1.0;
  for (int i = 0; i < p->d; ++i) t.f[i] = q ? facq_ref(p, i, 1, s, 2, 0, true) : fac_ref(p, i, 1, s, 2, 0, true);
  return {t};
}

// ---- systems (Sec. 3.3): the terms of one block.  Outputs are a priori
// uncorrelated (Eq. multioutput-cov-def), so a pair of terms contributes only
// where both act on the same output.
// G_PP block (equation e, equation e2): pairs a in e, b in e2 on one output
std::vector<KTerm> pp_terms_mo(const gpfvm_problem* p, int e, int e2) {
  std::vector<KTerm> ts;
  for (int a = 0; a < p->nterms; ++a)
    for (int b = 0; b < p->nterms; ++b) {
      if (p->teq[a] != e || p->teq[b] != e2 || p->tout[a] != p->tout[b]) continue;
      KTerm t{};
      t.c = p->coef[a] * p->coef[b];
      for (int i = 0; i < p->d; ++i) t.f[i] = fac_ref(p, i, 0, p->alpha[a][i], 0, p->alpha[b][i], false);
      ts.push_back(t);
    }
  return ts;
}
// cells of equation e -> set s (to_set) or back: the terms of e on the set's output
std::vector<KTerm> pb_terms_mo(const gpfvm_problem* p, int s, int e, bool to_set) {
  std::vector<KTerm> ts;
  for (int a = 0; a < p->nterms; ++a) {
    if (p->teq[a] != e || p->tout[a] != p->sets[s].comp) continue;
    KTerm t{};
    t.c = p->coef[a];
    for (int i = 0; i < p->d; ++i) t.f[i] = fac_ref(p, i, 0, p->alpha[a][i], 1, s, to_set);
    ts.push_back(t);
  }
  return ts;
}
// cells of equation e -> prediction grid of output j
std::vector<KTerm> ppred_terms_mo(const gpfvm_problem* p, int e, int j) {
  std::vector<KTerm> ts;
  for (int a = 0; a < p->nterms; ++a) {
    if (p->teq[a] != e || p->tout[a] != j) continue;
    KTerm t{};
    t.c = p->coef[a];
    for (int i = 0; i < p->d; ++i) t.f[i] = fac_ref(p, i, 0, p->alpha[a][i], 2, 0, true);
    ts.push_back(t);
  }
  return ts;
}

void dims_cells(const gpfvm_problem* p, int* o) { for (int i = 0; i < p->d; ++i) o[i] = p->nc[i]; }
void dims_set(const gpfvm_problem* p, int s, int* o) { for (int i = 0; i < p->d; ++i) o[i] = p->sets[s].n[i]; }
void dims_pred(const gpfvm_problem* p, int* o) { for (int i = 0; i < p->d; ++i) o[i] = p->npred[i]; }

}  // namespace

namespace {

struct Builder {
  gpfvm_problem* p;
  Scratch scr;
  i64 peak = 0;
  bool f32 = false;  // build FP32 plans (pointers below then address float data)
  // `base` advanced by n elements of the plan's element type
  template <typename P>
  P at(P base, i64 n) const {
    if (!f32) return base + n;
    typedef typename std::conditional<std::is_const<typename std::remove_pointer<P>::type>::value, const float*,
                                      float*>::type FP;
    return (P)((FP)base + n);
  }
  bool keep = false;  // inside a stage of zipped chains: intermediates must not overlap
  bool fma_only = false;  // kron_digits declines (the FP64 FMA operators)
  void stage_begin() {
    scr.used = 0;
    keep = true;
  }
  void stage_end() { keep = false; }
  void kron(Plan& plan, const int* din, const int* dout, i64 batch, const std::vector<KTerm>& terms, double scale,
            const double* in, double* out, double beta, const double* D, double gamma, int* count = nullptr,
            int dd = 0) {
    if (!keep) scr.used = 0;
    plan_kron(plan, scr, dd > 0 ? dd : p->d, din, dout, batch, terms, scale, in, out, beta, D, gamma, count, f32);
    peak = std::max(peak, scr.used);
  }

  // out = scale * sum_t c_t (F_t0 (x) F_t1 (x) F_t2) in + beta out + gamma D in
  // FP64 by exact digit products on the tensor cores (oz.cu), in the shared
  // rotating-axes three-level form (contract the last axis, write the new axis
  // first); false, with nothing added, where that form does not apply (FP32
  // plans, one axis, an axis above 128, the FMA form chosen).  Intermediates
  // and row exponents come from the stage's scratch.
  bool kron_digits(Plan& plan, const int* din, const int* dout, const std::vector<KTerm>& terms, double scale,
                   const double* in, double* out, double beta, const double* D, double gamma, const int* skip) {
    const int d = p->d;
    if (f32 || fma_only || !p->oz_ok || !p->oz_on || d < 2 || terms.empty()) return false;
    for (int i = 0; i < d; ++i)
      if (din[i] < 1 || dout[i] < 1 || din[i] > OZ_KMAX || dout[i] > 128) return false;
    if (!keep) scr.used = 0;
    auto same = [](const MatRef& a, const MatRef& b) { return a.p == b.p && a.rs == b.rs && a.cs == b.cs; };
    auto image = [&](const MatRef& f, int N, int K, double alpha) {
      const auto key = std::make_tuple(f.p, f.rs, f.cs, N, K, alpha);
      auto it = p->ozx_img.find(key);
      if (it == p->ozx_img.end()) {
        it = p->ozx_img.emplace(key, std::make_pair(p->ozx_img_n, p->ozx_fexp_n)).first;
        p->ozx_jobs.push_back({f.p, f.rs, f.cs, N, K, alpha, p->ozx_img_n, p->ozx_fexp_n});
        p->ozx_img_n += oz_image_bytes(N, K);
        p->ozx_fexp_n += (N + 31) / 32 * 32;
      }
      return std::make_pair(p->d_ozximg ? (const unsigned char*)(p->d_ozximg + it->second.first) : nullptr,
                            p->d_ozxfexp ? (const int*)(p->d_ozxfexp + it->second.second) : nullptr);
    };
    struct Lv { int off, nops; i64 tiles; OzExpJobs jobs; int n; };
    std::vector<Lv> lv;
    bool ok = true;
    const size_t first_op = p->ozx_ops.size();
    auto begin_level = [&](i64 R, int K) {
      Lv L{};
      L.off = (int)p->ozx_ops.size();
      L.jobs.R = (int)R;
      L.jobs.K = K;
      L.jobs.skip = skip;
      lv.push_back(L);
    };
    auto job = [&](const double* A, i64 R) -> const int* {
      auto& J = lv.back().jobs;
      if (J.n >= OZ_MAXSEG) { ok = false; return nullptr; }
      J.A[J.n] = A;
      J.ex[J.n] = (int*)take((R + 1) / 2);
      return J.ex[J.n++];
    };
    auto blank = [&](i64 R, int K, int N, double* o) {
      OzOp op{};
      op.R = (int)R; op.K = K; op.N = N; op.out = o;
      op.skip = skip;
      return op;
    };
    auto seg = [&](OzOp& op, const double* A, const int* ex, const MatRef& f, int N, int K, double alpha) {
      if (op.nseg >= OZ_MAXSEG) { ok = false; return; }
      const auto im = image(f, N, K, alpha);
      op.A[op.nseg] = A;
      op.Aexp[op.nseg] = ex;
      op.Bimg[op.nseg] = im.first;
      op.Bexp[op.nseg] = im.second;
      op.nseg++;
    };
    auto add_op = [&](OzOp op) {
      auto& L = lv.back();
      op.tile_begin = L.tiles;
      if (L.nops > 0 && L.n != op.N) ok = false;  // one tiling per launch
      L.n = op.N;
      L.tiles += oz_tiles(op.R, op.N);
      L.nops++;
      p->ozx_ops.push_back(op);
    };
    const i64 n0 = din[0], n1 = din[1], n2 = d == 3 ? din[2] : 1;
    const i64 m0 = dout[0], m1 = dout[1], m2 = d == 3 ? dout[2] : 1;
    std::vector<MatRef> U, Wf;
    std::vector<int> uo(terms.size()), wo(terms.size());
    for (size_t k = 0; k < terms.size(); ++k) {
      if (d == 3) {
        int f = -1;
        for (size_t u = 0; u < U.size(); ++u) if (same(U[u], terms[k].f[2])) f = (int)u;
        if (f < 0) { f = (int)U.size(); U.push_back(terms[k].f[2]); }
        uo[k] = f;
      }
      int w = -1;
      for (size_t j = 0; j < Wf.size(); ++j) if (same(Wf[j], terms[k].f[0])) w = (int)j;
      if (w < 0) { w = (int)Wf.size(); Wf.push_back(terms[k].f[0]); }
      wo[k] = w;
    }
    std::vector<const double*> Y;
    std::vector<const int*> exY;
    if (d == 3) {  // contract axis 2: (n0 n1) x n2 -> Y_u (m2, n0, n1)
      begin_level(n0 * n1, (int)n2);
      const int* ex = job(in, n0 * n1);
      for (size_t u = 0; u < U.size(); ++u) {
        double* y = take(m2 * n0 * n1);
        Y.push_back(y);
        OzOp op = blank(n0 * n1, (int)n2, (int)m2, y);
        seg(op, in, ex, U[u], (int)m2, (int)n2, 1.0);
        add_op(op);
      }
    }
    // contract axis 1: rows (m2, n0) (or n0) x n1 -> Z_w (m1, m2, n0)
    const i64 R2 = m2 * n0;
    begin_level(R2, (int)n1);
    if (d == 3) for (size_t u = 0; u < U.size(); ++u) exY.push_back(job(Y[u], R2));
    else exY.push_back(job(in, R2));
    std::vector<const double*> Z;
    for (size_t w = 0; w < Wf.size(); ++w) {
      double* z = take(m1 * R2);
      Z.push_back(z);
      OzOp op = blank(R2, (int)n1, (int)m1, z);
      std::vector<std::pair<std::pair<int, MatRef>, double>> acc;  // merged (source, factor) pairs
      for (size_t k = 0; k < terms.size(); ++k) {
        if (wo[k] != (int)w) continue;
        const int src = d == 3 ? uo[k] : 0;
        bool merged = false;
        for (auto& a : acc)
          if (a.first.first == src && same(a.first.second, terms[k].f[1])) { a.second += terms[k].c; merged = true; }
        if (!merged) acc.push_back({{src, terms[k].f[1]}, terms[k].c});
      }
      for (auto& a : acc)
        seg(op, d == 3 ? Y[a.first.first] : in, exY[a.first.first], a.first.second, (int)m1, (int)n1, a.second);
      add_op(op);
    }
    // contract axis 0: rows (m1, m2) x n0 -> out (m0, m1, m2)
    const i64 R3 = m1 * m2;
    begin_level(R3, (int)n0);
    OzOp op = blank(R3, (int)n0, (int)m0, out);
    for (size_t w = 0; w < Wf.size(); ++w) seg(op, Z[w], job(Z[w], R3), Wf[w], (int)m0, (int)n0, scale);
    op.D = D;
    op.gamma = gamma;
    op.beta = beta;
    add_op(op);
    peak = std::max(peak, scr.used);
    if (!ok) {
      p->ozx_ops.resize(first_op);
      return false;
    }
    for (const Lv& L : lv) {
      const OzExpJobs J = L.jobs;
      const OzOp* ops = p->d_ozxops ? p->d_ozxops + L.off : nullptr;
      const int nops = L.nops;
      const i64 tiles = L.tiles;
      const int nl = L.n;
      int* status = &p->d_st->status;
      plan.func([=](cudaStream_t st) {
        oz_row_exponents(J, st);
        launch_oz_modes(ops, nops, tiles, nl, status, st);
      });
    }
    return true;
  }

  // ---- variable coefficients (App. C.4): a term's cell-side factor carries
  // diag(f_a); products are grouped by field class and combined elementwise
  bool varcoef() const { return p->nfield > 0; }
  const void* field_ptr(int cls) const {
    if (cls < 0) return nullptr;
    return f32 ? (const void*)(p->f_field + (i64)cls * p->N) : (const void*)(p->d_field + (i64)cls * p->N);
  }
  void combine(Plan& plan, double* out, const std::vector<std::pair<const double*, int>>& ys, double scale,
               const double* D, double gamma, double beta) {
    FieldTerms t{};
    t.nt = (int)ys.size();
    if (t.nt > FIELD_MAXT) throw CudaError{cudaErrorInvalidValue, "too many field classes"};
    for (int k = 0; k < t.nt; ++k) {
      t.y[k] = ys[k].first;
      t.f[k] = field_ptr(ys[k].second);
      t.scale[k] = scale;
    }
    const bool F = f32;
    const i64 n = p->N;
    plan.func([=](cudaStream_t st) { field_combine(out, n, t, D, gamma, beta, F, st); });
  }
  // w_Q = f_Q .* in for every class (the constant class reads in itself)
  std::vector<const double*> vc_inputs(Plan& plan, const double* in, const std::vector<int>& cls) {
    std::vector<const double*> w;
    for (int c : cls) {
      if (c < 0) { w.push_back(in); continue; }
      double* x = take(p->N);
      combine(plan, x, {{in, c}}, 1.0, nullptr, 0.0, 0.0);
      w.push_back(x);
    }
    return w;
  }
  // sum over classes Q of kron(terms of class Q) applied to w_Q into out (din -> dout)
  void vc_sum_in(Plan& plan, const int* din, const int* dout, const std::vector<KTerm>& all,
                 const std::vector<int>& cls, const std::vector<const double*>& w, double scale, double* out,
                 bool accumulate) {
    bool first = !accumulate;
    for (size_t q = 0; q < cls.size(); ++q) {
      const std::vector<KTerm> ts = class_terms(all, p, cls[q], [](size_t t) { return (int)t; });
      if (ts.empty()) continue;
      kron(plan, din, dout, 1, ts, scale, w[q], out, first ? 0.0 : 1.0, nullptr, 0.0);
      first = false;
    }
  }
  // out (+)= scale * sum_P f_P .* kron(terms of class P) in  (din -> cells)
  void vc_sum_out(Plan& plan, const int* din, const std::vector<KTerm>& all, const std::vector<int>& cls,
                  const double* in, double scale, double* out, bool accumulate) {
    int dc[3];
    dims_cells(p, dc);
    std::vector<std::pair<const double*, int>> ys;
    for (int c : cls) {
      const std::vector<KTerm> ts = class_terms(all, p, c, [](size_t t) { return (int)t; });
      if (ts.empty()) continue;
      double* y = take(p->N);
      kron(plan, din, dc, 1, ts, scale, in, y, 0.0, nullptr, 0.0);
      ys.push_back({y, c});
    }
    combine(plan, out, ys, 1.0, nullptr, 0.0, accumulate ? 1.0 : 0.0);
  }
  // G_PP in (+ G_PB / L k(X*) parts): the variable-coefficient operator,
  // sequential (no face sets, no tensor cores, no background chain)
  void vc_ghat(Plan& plan, const double* in, double* out, double* g, double* w, double* u, bool with_icbc) {
    stage_begin();
    int dc[3], ds[3], dp[3];
    dims_cells(p, dc);
    dims_pred(p, dp);
    const std::vector<int> cls = field_classes(p);
    const std::vector<const double*> win = vc_inputs(plan, in, cls);
    std::vector<std::pair<const double*, int>> ys;
    std::vector<double*> y(cls.size());
    for (size_t P = 0; P < cls.size(); ++P) {
      y[P] = take(p->N);
      bool first = true;
      for (size_t Q = 0; Q < cls.size(); ++Q) {
        const std::vector<KTerm> ts = pp_terms_pq(p, cls[P], cls[Q]);
        if (ts.empty()) continue;
        kron(plan, dc, dc, 1, ts, p->s2, win[Q], y[P], first ? 0.0 : 1.0, nullptr, 0.0);
        first = false;
      }
      if (!first) ys.push_back({y[P], cls[P]});
    }
    if (with_icbc && p->M > 0) {
      for (int s = 0; s < p->nsets; ++s) {
        dims_set(p, s, ds);
        vc_sum_in(plan, dc, ds, pb_terms(p, s, true, true), cls, win, p->s2, at(g, p->sets[s].off), false);
      }
      Plan H;
      int ready[2];
      hsolve_chain(H, g, w, ready);
      plan.zip({&H});
      for (size_t P = 0; P < cls.size(); ++P) {
        bool has = false;
        for (auto& e : ys) has = has || e.second == cls[P];
        for (int s = 0; s < p->nsets; ++s) {
          dims_set(p, s, ds);
          const std::vector<KTerm> ts =
              class_terms(pb_terms(p, s, false, true), p, cls[P], [](size_t t) { return (int)t; });
          if (ts.empty()) continue;
          kron(plan, ds, dc, 1, ts, -p->s2, at(w, p->sets[s].off), y[P], has ? 1.0 : 0.0, nullptr, 0.0);
          if (!has) ys.push_back({y[P], cls[P]});
          has = true;
        }
      }
    }
    combine(plan, out, ys, 1.0, in, p->jitter, 0.0);  // + jitter in (G_PP)
    if (u) {
      vc_sum_in(plan, dc, dp, ppred_terms(p), cls, win, p->s2, u, false);
      if (with_icbc && p->M > 0) to_pred_sets(plan, w, u, -1.0, true, true);
    }
    stage_end();
  }

  // out = G_BP in (cells -> all sets), into g (M); fold: set 0 in its eigenbasis
  void bp(Plan& plan, const double* in, double* g, bool fold = false) {
    if (p->multi) {
      mo_bp(plan, in, g);
      return;
    }
    int dc[3], ds[3];
    dims_cells(p, dc);
    if (varcoef()) {
      const bool k0 = keep;
      if (!k0) stage_begin();
      const std::vector<int> cls = field_classes(p);
      const std::vector<const double*> win = vc_inputs(plan, in, cls);
      for (int s = 0; s < p->nsets; ++s) {
        dims_set(p, s, ds);
        vc_sum_in(plan, dc, ds, pb_terms(p, s, true, fold), cls, win, p->s2, at(g, p->sets[s].off), false);
      }
      if (!k0) stage_end();
      return;
    }
    for (int s = 0; s < p->nsets; ++s) {
      dims_set(p, s, ds);
      kron(plan, dc, ds, 1, pb_terms(p, s, true, fold), p->s2, in, at(g, p->sets[s].off), 0.0, nullptr, 0.0);
    }
  }
  // out (+)= scale * G_PB w; fold: the set-0 part of w in its eigenbasis
  void pb(Plan& plan, const double* w, double* out, double scale, bool accumulate, bool fold = false) {
    if (p->multi) {
      mo_pb(plan, w, out, scale, accumulate);
      return;
    }
    int dc[3], ds[3];
    dims_cells(p, dc);
    if (varcoef()) {
      const bool k0 = keep;
      if (!k0) stage_begin();
      const std::vector<int> cls = field_classes(p);
      std::vector<std::pair<const double*, int>> ys;
      for (int c : cls) {
        double* y = take(p->N);
        bool first = true;
        for (int s = 0; s < p->nsets; ++s) {
          dims_set(p, s, ds);
          const std::vector<KTerm> ts =
              class_terms(pb_terms(p, s, false, fold), p, c, [](size_t t) { return (int)t; });
          if (ts.empty()) continue;
          kron(plan, ds, dc, 1, ts, scale * p->s2, at(w, p->sets[s].off), y, first ? 0.0 : 1.0, nullptr, 0.0);
          first = false;
        }
        if (!first) ys.push_back({y, c});
      }
      combine(plan, out, ys, 1.0, nullptr, 0.0, accumulate ? 1.0 : 0.0);
      if (!k0) stage_end();
      return;
    }
    for (int s = 0; s < p->nsets; ++s) {
      dims_set(p, s, ds);
      kron(plan, ds, dc, 1, pb_terms(p, s, false, fold), scale * p->s2, at(w, p->sets[s].off), out,
           (accumulate || s > 0) ? 1.0 : 0.0, nullptr, 0.0);
    }
  }
  // G_BB^-1 with the structured IC/BC stage, in the eigenbasis of set 0: the
  // set-0 parts g~_K, w~_K of g and w are coordinates in (x)Q_i (the folded
  // G_BP / G_PB / prediction factors produce and consume them), so
  //   t_R  = g_R - E~ g~_K            (E~ = G_RK (x)Q Lambda~^-1)
  //   w_R  = L_S^-T L_S^-1 t_R       (S = G_RR - G_RK A^-1 G_KR = L_S L_S^T)
  //   w~_K = Lambda~^-1 g~_K - E~^T w_R
  // is a chain of four dependent GEMVs; without the structured stage it is
  // w = L^-T L^-1 g.  Appends the chain to c (one op per level) and returns in
  // ready[0] / ready[1] the number of levels after which the part of w of set 0
  // / of the other sets is final.
  void hsolve_chain(Plan& c, const double* g, double* w, int* ready) {
    const int M = (int)p->M, MK = p->MK, MR = p->MR;
    const bool F = f32;
    if (!p->sicbc) {
      double* t = F ? (double*)p->f_t : p->d_t;
      const void* Li = F ? (const void*)p->f_Linv : (const void*)p->d_Linv;
      const void* LiT = F ? (const void*)p->f_LinvT : (const void*)p->d_LinvT;
      c.gemvz(F, M, M, Li, M, g, t, 1.0, 0.0, nullptr, nullptr, 1);
      c.gemvz(F, M, M, LiT, M, t, w, 1.0, 0.0, nullptr, nullptr, 2);
      ready[0] = ready[1] = 2;
    } else if (MR > 0) {
      double* tR = F ? (double*)p->f_tR : p->d_tR;
      double* uR = F ? (double*)p->f_uR : p->d_uR;
      const void* Et = F ? (const void*)p->f_Et : (const void*)p->d_Et;
      const void* EtT = F ? (const void*)p->f_EtT : (const void*)p->d_EtT;
      const void* LSi = F ? (const void*)p->f_LSinv : (const void*)p->d_LSinv;
      const void* LSiT = F ? (const void*)p->f_LSinvT : (const void*)p->d_LSinvT;
      c.gemvz(F, MR, MK, Et, MK, g, tR, -1.0, 1.0, at(g, MK), nullptr);
      c.gemvz(F, MR, MR, LSi, MR, tR, uR, 1.0, 0.0, nullptr, nullptr, 1);
      c.gemvz(F, MR, MR, LSiT, MR, uR, at(w, MK), 1.0, 0.0, nullptr, nullptr, 2);
      c.gemvz(F, MK, MR, EtT, MR, at(w, MK), w, -1.0, 1.0, g, p->d_ltinv);
      ready[0] = 4;
      ready[1] = 3;
    } else {
      c.gemvz(F, MK, 0, g, 0, g, w, 0.0, 1.0, g, p->d_ltinv);
      ready[0] = ready[1] = 1;
    }
  }
  // rows x <- rows x (x)Q_i^T over set 0's axes (FP64); singleton axes
  // (Q = [1]) are dropped
  void eig_rows(Plan& plan, i64 rows, const double* x, double* xt) {
    int dK[3], nd = 0;
    KTerm QT{};
    QT.c = 1.0;
    for (int i = 0; i < p->d; ++i) {
      if (p->nK[i] == 1 && !(i == p->d - 1 && nd == 0)) continue;
      QT.f[nd] = MatRef{p->d_QK[i], 1, p->nK[i]};
      dK[nd++] = p->nK[i];
    }
    kron(plan, dK, dK, rows, {QT}, 1.0, x, xt, 0.0, nullptr, 0.0, nullptr, nd);
  }
  // y~ (set 0 in its eigenbasis, the other sets as they are) from y (FP64)
  void to_eigenbasis(Plan& plan, const double* y, double* yt) {
    const int MK = p->MK, MR = p->MR;
    eig_rows(plan, 1, y, yt);
    if (MR > 0) plan.copy(yt + MK, y + MK, (i64)sizeof(double) * MR);
  }
  // w = G_BB^-1 g (w~ / g~ in the eigenbasis of set 0 with the structured stage)
  void hsolve(Plan& plan, const double* g, double* w) {
    Plan c;
    int ready[2];
    hsolve_chain(c, g, w, ready);
    plan.zip({&c});
  }
  // n elements of the plan's element type from the scratch pool
  double* take(i64 n) {
    double* r = scr.take(f32 ? (n + 1) / 2 : n);
    peak = std::max(peak, scr.used);
    return r;
  }

  // ---- sets on faces of the box (face.cuh)
  // The axis on which set s has its fewest coordinates (at most FACE_MAXF:
  // faces), when its other dimensions and those of the grid dt fit the
  // bilinear kernel; else -1.
  int face_axis(int s, const int* dt) const {
    if (p->d != 3 || p->nterms > FACE_MAXT || p->multi) return -1;
    int a = 0;
    for (int i = 1; i < 3; ++i)
      if (p->sets[s].n[i] < p->sets[s].n[a]) a = i;
    if (p->sets[s].n[a] > FACE_MAXF) return -1;
    for (int i = 0; i < 3; ++i)
      if (i != a && (p->sets[s].n[i] > FACE_MAXN || dt[i] > FACE_MAXN)) return -1;
    if ((i64)dt[0] * dt[1] * dt[2] >= ((i64)1 << 31)) return -1;  // 32-bit element indices
    return a;
  }
  // strides of set s's flattened layout (row-major over the three axes)
  void set_strides(int s, i64* st) const {
    st[2] = 1;
    st[1] = p->sets[s].n[2];
    st[0] = (i64)p->sets[s].n[1] * p->sets[s].n[2];
  }
  // distinct factors on axis a of a term list
  static void distinct_on(const std::vector<KTerm>& ts, int a, std::vector<MatRef>& U, std::vector<int>& ui) {
    U.clear();
    ui.assign(ts.size(), -1);
    for (size_t t = 0; t < ts.size(); ++t) {
      for (size_t k = 0; k < U.size(); ++k)
        if (U[k].p == ts[t].f[a].p && U[k].rs == ts[t].f[a].rs && U[k].cs == ts[t].f[a].cs) ui[t] = (int)k;
      if (ui[t] < 0) {
        ui[t] = (int)U.size();
        U.push_back(ts[t].f[a]);
      }
    }
  }
  // G_BP of a face set s into gs: a CONTR chain (level 0) and one BILIN
  // chain per face (level 1), appended to `chains` with their levels in
  // `lv`; false if s does not qualify
  bool bp_face(std::deque<Plan>& chains, std::vector<int>& lv, int s, const double* in, double* gs) {
    int dc[3];
    dims_cells(p, dc);
    const int a = face_axis(s, dc);
    if (a < 0) return false;
    const std::vector<KTerm> ts = pb_terms(p, s, true, true);
    std::vector<MatRef> U;
    std::vector<int> ui;
    distinct_on(ts, a, U, ui);
    const int na = p->sets[s].n[a];
    if ((int)U.size() * na > FACE_MAXF) return false;
    for (auto& f : U)
      if (f.cs != U[0].cs) return false;
    const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
    const i64 Nb = dc[b], Nc = dc[cc];
    i64 sst[3];
    set_strides(s, sst);
    // the bilinear forms of the faces (Y_u,m are placed below; take() only
    // after every check has passed)
    std::vector<BilOp> bos(na);
    for (int m = 0; m < na; ++m) {
      BilOp& bo = bos[m];
      bo = BilOp{};
      bo.batch = 1;
      bo.out = at(gs, m * sst[a]);
      bo.ldo = sst[b];
      bo.ocs = sst[cc];
      bo.R = p->sets[s].n[b];
      bo.C = p->sets[s].n[cc];
      bo.K1 = (int)Nb;
      bo.K2 = (int)Nc;
      for (size_t k = 0; k < ts.size(); ++k) {
        const KTerm& t = ts[k];
        // X is patched to Y_u,m once it exists; the slot index keeps operands apart
        const BilMat X{(const void*)(intptr_t)(1 + ui[k] * na + m), Nc, 1};
        if (!bil_add(bo, BilMat{t.f[b].p, t.f[b].rs, t.f[b].cs}, X, BilMat{t.f[cc].p, t.f[cc].rs, t.f[cc].cs},
                     t.c * p->s2))
          return false;
      }
      if (bilin_smem_elems(bo.C, bo.K1, bo.K2, bo.nA, bo.nX, bo.nB, bo.nt) * (f32 ? 4 : 8) > FACE_SMEM_MAX)
        return false;
    }
    // the factor on a is na x N_a: row m is f(m, k) = p[m rs + k cs]
    ContrOp co{};
    co.in = in;
    co.nf = (int)U.size() * na;
    co.na = dc[a];
    co.fs = U[0].cs;
    co.pre = 1;
    co.post = 1;
    for (int i = 0; i < a; ++i) co.pre *= dc[i];
    for (int i = a + 1; i < 3; ++i) co.post *= dc[i];
    co.alpha = 1.0;
    double* Y[FACE_MAXF];
    for (size_t k = 0; k < U.size(); ++k)
      for (int m = 0; m < na; ++m) {
        const int j = (int)k * na + m;
        Y[j] = take(Nb * Nc);
        co.f[j] = at(U[k].p, m * U[k].rs);
        co.out[j] = Y[j];
      }
    chains.emplace_back();
    chains.back().contr(co, f32);
    lv.push_back(0);
    for (int m = 0; m < na; ++m) {
      BilOp bo = bos[m];
      for (int k = 0; k < bo.nX; ++k) bo.X[k].p = Y[(intptr_t)bo.X[k].p - 1];
      chains.emplace_back();
      chains.back().bilin(bo, f32);
      lv.push_back(1);
    }
    return true;
  }
  // -s2 (G_PB w_s) (pred = false, grid = cells) or -s2 k_s(X*)^T w_s (pred =
  // true) of a face set s: one BILIN chain per distinct factor on the face
  // axis and face (appended to `chains`), expansion terms appended to `xt`
  bool pb_face(std::deque<Plan>& chains, int s, const double* ws, bool pred, std::vector<ExpTerm>& xt) {
    int dt[3];
    if (pred) dims_pred(p, dt);
    else dims_cells(p, dt);
    const int a = face_axis(s, dt);
    if (a < 0) return false;
    const std::vector<KTerm> ts = pred ? bpred_terms(p, s, true) : pb_terms(p, s, false, true);
    std::vector<MatRef> U;
    std::vector<int> ui;
    distinct_on(ts, a, U, ui);
    const int na = p->sets[s].n[a];
    if ((int)(xt.size() + U.size() * na) > FACE_MAXJ) return false;
    const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
    const i64 Nb = dt[b], Nc = dt[cc];
    const int nb = p->sets[s].n[b], nc = p->sets[s].n[cc];
    i64 sst[3];
    set_strides(s, sst);
    std::vector<BilOp> bos;
    for (size_t k = 0; k < U.size(); ++k)
      for (int m = 0; m < na; ++m) {
        BilOp bo{};
        bo.batch = 1;
        bo.ldo = Nc;
        bo.ocs = 1;
        bo.R = (int)Nb;
        bo.C = (int)Nc;
        bo.K1 = nb;
        bo.K2 = nc;
        for (size_t t = 0; t < ts.size(); ++t) {
          if (ui[t] != (int)k) continue;
          const KTerm& x = ts[t];
          if (!bil_add(bo, BilMat{x.f[b].p, x.f[b].rs, x.f[b].cs}, BilMat{at(ws, m * sst[a]), sst[b], sst[cc]},
                       BilMat{x.f[cc].p, x.f[cc].rs, x.f[cc].cs}, -x.c * p->s2))
            return false;
        }
        if (bilin_smem_elems(bo.C, bo.K1, bo.K2, bo.nA, bo.nX, bo.nB, bo.nt) * (f32 ? 4 : 8) > FACE_SMEM_MAX)
          return false;
        bos.push_back(bo);
      }
    for (size_t k = 0; k < U.size(); ++k)
      for (int m = 0; m < na; ++m) {
        double* Z = take(Nb * Nc);
        BilOp bo = bos[k * na + m];
        bo.out = Z;
        chains.emplace_back();
        chains.back().bilin(bo, f32);
        // the factor on a is N_a x na: column m is f(k, m) = p[k rs + m cs]
        xt.push_back(ExpTerm{at(U[k].p, m * U[k].cs), U[k].rs, Z, a, 1.0});
      }
    return true;
  }

  // Rows m0 .. m0 + rows of the Cholesky-stage variance term with the
  // structured stage, Y = s2 (sum over sets s >= 1 of k_s(X*)^T L_S^-1[rows, s])
  // - s2 k~_K(X*)^T R[rows] (rows x P into Y), when every set lies on faces of
  // the box: one batched bilinear form per set and face (over the rows), then
  // one expansion that writes Y.  False (nothing added) otherwise.
  bool var_face_chunk(Plan& pl, int m0, int rows, double* Y) {
    int dp[3];
    dims_pred(p, dp);
    const int MK = p->MK, MR = p->MR;
    struct Part {
      int s, a;
      KTerm t;
    };
    std::vector<Part> parts;
    i64 zbs = 0;
    int nj = 0;
    for (int s = 0; s < p->nsets; ++s) {
      const int a = face_axis(s, dp);
      if (a < 0) return false;
      const std::vector<KTerm> ts = bpred_terms(p, s, true);
      if (ts.size() != 1) return false;
      const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
      if (bilin_smem_elems(dp[cc], p->sets[s].n[b], p->sets[s].n[cc], 1, 1, 1, 1) * 8 > FACE_SMEM_MAX) return false;
      nj += p->sets[s].n[a];
      zbs = std::max<i64>(zbs, (i64)dp[b] * dp[cc]);
      parts.push_back(Part{s, a, ts[0]});
    }
    if (nj > FACE_MAXJ) return false;
    zbs = (zbs + 3) / 4 * 4;  // every row of Z starts 32-byte aligned
    std::deque<Plan> ch;
    std::vector<ExpTerm> xt;
    for (const Part& pt : parts) {
      const int s = pt.s, a = pt.a, b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
      i64 sst[3];
      set_strides(s, sst);
      const double* base = s == 0 ? p->d_R + (i64)m0 * MK : p->d_LSinv + (i64)m0 * MR + (p->sets[s].off - MK);
      const KTerm& t = pt.t;
      const double alpha = (s == 0 ? -1.0 : 1.0) * t.c * p->s2;
      for (int m = 0; m < p->sets[s].n[a]; ++m) {
        double* Z = take((i64)rows * zbs);
        BilOp bo{};
        bo.batch = rows;
        bo.xbs = s == 0 ? MK : MR;
        bo.obs = zbs;
        bo.out = Z;
        bo.ldo = dp[cc];
        bo.ocs = 1;
        bo.R = dp[b];
        bo.C = dp[cc];
        bo.K1 = p->sets[s].n[b];
        bo.K2 = p->sets[s].n[cc];
        bil_add(bo, BilMat{t.f[b].p, t.f[b].rs, t.f[b].cs}, BilMat{base + m * sst[a], sst[b], sst[cc]},
                BilMat{t.f[cc].p, t.f[cc].rs, t.f[cc].cs}, alpha);
        ch.emplace_back();
        ch.back().bilin(bo, false);
        // the factor on a is P_a x n_a: column m is f(k, m) = p[k rs + m cs]
        xt.push_back(ExpTerm{t.f[a].p + m * t.f[a].cs, t.f[a].rs, Z, a, 1.0});
      }
    }
    std::vector<const Plan*> cp;
    for (auto& c : ch) cp.push_back(&c);
    pl.zip(cp);
    ExpAddOp eo{};
    eo.dst = Y;
    eo.n = (i64)rows * p->P;
    eo.nper = p->P;
    eo.zbs = zbs;
    eo.zero = 1;
    eo.d1 = dp[1];
    eo.d2 = dp[2];
    eo.nj = (int)xt.size();
    for (size_t j = 0; j < xt.size(); ++j) eo.j[j] = xt[j];
    bool vec = dp[2] % 4 == 0 && ((uintptr_t)Y & 15) == 0;
    for (auto& x : xt) vec = vec && (x.axis == 2 || ((uintptr_t)x.Z & 15) == 0);
    eo.vec = vec ? 1 : 0;
    Plan E;
    E.expadd(eo, false);
    pl.zip({&E});
    return true;
  }

  // out = G^ in = G_PP in - G_PB G_BB^-1 G_BP in; with u != null also
  // u = Lhat k(X*)^T in.  Every product is a chain of dependent launches; the
  // chains are placed by phase so that each starts as soon as its input is final:
  //   phase 0..        G_PP in (into out), G_BP in (each set, into g), L k(X*)^T in (into u)
  //   after G_BP:      w = G_BB^-1 g (hsolve_chain)
  //   after w_s final: -G_PB w_s and -k_s(X*)^T w_s per set s
  //   last:            out += the G_PB parts, u += the k(X*) parts (EXPADD;
  //                    sets in order, so the result does not depend on the concurrency)
  // Sets on a face of the box take the CONTR / BILIN / EXPADD form (two
  // launches per direction instead of three); the others take Kronecker chains
  // into separate buffers.  With IC/BC sets, G_PP runs beside all of it as a
  // background chain.
  // `skip` is the plan's skip flag (the digit-product chains honour it too).
  void ghat_phased(Plan& plan, const double* in, double* out, double* g, double* w, double* u, int* count,
                   Plan* pp_chain = nullptr, const int* skip = nullptr) {
    if (p->multi) {
      mo_ghat(plan, in, out, g, w, u);
      return;
    }
    if (varcoef()) {
      vc_ghat(plan, in, out, g, w, u, true);
      return;
    }
    int dc[3], ds[3], dp[3];
    dims_cells(p, dc);
    dims_pred(p, dp);
    const int ns = p->nsets;
    stage_begin();  // one stage: every intermediate below is distinct
    Plan PP, PR;
    if (pp_chain) PP = std::move(*pp_chain);
    else kron(PP, dc, dc, 1, pp_terms(p), p->s2, in, out, 0.0, in, p->jitter, count);
    // the Kronecker chains of G_PR (variance) and of the IC/BC sets off the
    // box faces run as digit products when the FP64 form is chosen
    if (u && !kron_digits(PR, dc, dp, ppred_terms(p), p->s2, in, u, 0.0, nullptr, 0.0, skip))
      kron(PR, dc, dp, 1, ppred_terms(p), p->s2, in, u, 0.0, nullptr, 0.0);
    std::vector<const Plan*> cs;
    std::vector<int> st;
    auto put = [&](const Plan& c, int s0) {
      if (c.ops.empty()) return;
      cs.push_back(&c);
      st.push_back(s0);
    };
    // G_PP (the longest chain) runs as the plan's background chain; only the
    // final sum waits for it
    const bool bgpp = p->M > 0 && !PP.ops.empty();
    if (!bgpp) put(PP, 0);
    if (u) put(PR, 0);
    std::vector<Plan> BP(ns), PB(ns), VS(ns);
    std::deque<Plan> FC;  // bilinear chains of face sets
    Plan H, SO, SU;
    if (p->M > 0) {
      int lbp = 0;
      for (int s = 0; s < ns; ++s) {
        dims_set(p, s, ds);
        const size_t f0 = FC.size();
        std::vector<int> lv;
        if (bp_face(FC, lv, s, in, at(g, p->sets[s].off))) {
          for (size_t k = f0; k < FC.size(); ++k) {
            put(FC[k], lv[k - f0]);
            lbp = std::max(lbp, lv[k - f0] + 1);
          }
        } else {
          if (!kron_digits(BP[s], dc, ds, pb_terms(p, s, true, true), p->s2, in, at(g, p->sets[s].off), 0.0, nullptr,
                           0.0, skip))
            kron(BP[s], dc, ds, 1, pb_terms(p, s, true, true), p->s2, in, at(g, p->sets[s].off), 0.0, nullptr, 0.0);
          lbp = std::max(lbp, (int)BP[s].ops.size());
          put(BP[s], 0);
        }
      }
      int ready[2];
      hsolve_chain(H, g, w, ready);
      put(H, lbp);
      const i64 sN = (p->N + 31) / 32 * 32, sP = (p->P + 31) / 32 * 32;
      std::vector<ExpTerm> xo, xu;
      std::vector<int> gen_o, gen_u;  // sets with Kronecker chains (dense parts)
      std::vector<int> r_of(ns);
      for (int s = 0; s < ns; ++s) {
        r_of[s] = lbp + ready[s == 0 ? 0 : 1];
        const size_t f0 = FC.size();
        if (pb_face(FC, s, at(w, p->sets[s].off), false, xo)) {
          for (size_t k = f0; k < FC.size(); ++k) put(FC[k], r_of[s]);
        } else {
          gen_o.push_back(s);
        }
        if (u) {
          const size_t f1 = FC.size();
          if (pb_face(FC, s, at(w, p->sets[s].off), true, xu)) {
            for (size_t k = f1; k < FC.size(); ++k) put(FC[k], r_of[s]);
          } else {
            gen_u.push_back(s);
          }
        }
      }
      double* T = gen_o.empty() ? nullptr : take((i64)gen_o.size() * sN);
      double* V = gen_u.empty() ? nullptr : take((i64)gen_u.size() * sP);
      for (size_t k = 0; k < gen_o.size(); ++k) {
        const int s = gen_o[k];
        dims_set(p, s, ds);
        if (!kron_digits(PB[s], ds, dc, pb_terms(p, s, false, true), -p->s2, at(w, p->sets[s].off),
                         at(T, (i64)k * sN), 0.0, nullptr, 0.0, skip))
          kron(PB[s], ds, dc, 1, pb_terms(p, s, false, true), -p->s2, at(w, p->sets[s].off), at(T, (i64)k * sN), 0.0,
               nullptr, 0.0);
        put(PB[s], r_of[s]);
      }
      for (size_t k = 0; k < gen_u.size(); ++k) {
        const int s = gen_u[k];
        dims_set(p, s, ds);
        if (!kron_digits(VS[s], ds, dp, bpred_terms(p, s, true), -p->s2, at(w, p->sets[s].off), at(V, (i64)k * sP),
                         0.0, nullptr, 0.0, skip))
          kron(VS[s], ds, dp, 1, bpred_terms(p, s, true), -p->s2, at(w, p->sets[s].off), at(V, (i64)k * sP), 0.0,
               nullptr, 0.0);
        put(VS[s], r_of[s]);
      }
      auto expadd = [&](Plan& pl, double* dst, i64 n, const int* dt, const double* parts, int np, i64 stride,
                        const std::vector<ExpTerm>& xt) {
        ExpAddOp eo{};
        eo.dst = dst;
        eo.n = n;
        eo.nper = n;
        eo.d1 = p->d == 3 ? dt[1] : 1;
        eo.d2 = p->d == 3 ? dt[2] : 1;
        eo.P = parts;
        eo.np = np;
        eo.pstride = stride;
        eo.nj = (int)xt.size();
        for (size_t j = 0; j < xt.size(); ++j) eo.j[j] = xt[j];
        auto al16 = [](const void* q) { return ((uintptr_t)q & 15) == 0; };
        bool vec = p->d == 3 && eo.d2 % 4 == 0 && al16(dst) && (np == 0 || (al16(parts) && stride % 4 == 0));
        for (auto& x : xt) vec = vec && (x.axis == 2 || al16(x.Z));
        eo.vec = vec ? 1 : 0;
        pl.expadd(eo, f32);
      };
      expadd(SO, out, p->N, dc, T, (int)gen_o.size(), sN, xo);
      if (u) expadd(SU, u, p->P, dp, V, (int)gen_u.size(), sP, xu);
    }
    if (bgpp) plan.fork(std::move(PP));
    plan.zip_at(cs, st);
    if (bgpp) plan.join();
    if (!SO.ops.empty()) {
      std::vector<const Plan*> last{&SO};
      if (!SU.ops.empty()) last.push_back(&SU);
      plan.zip(last);
    }
    stage_end();
  }

  void pp(Plan& plan, const double* in, double* out, int* count) {
    if (p->multi) {
      mo_pp(plan, in, out);
      return;
    }
    if (varcoef()) {
      vc_ghat(plan, in, out, nullptr, nullptr, nullptr, false);
      return;
    }
    int dc[3];
    dims_cells(p, dc);
    kron(plan, dc, dc, 1, pp_terms(p), p->s2, in, out, 0.0, in, p->jitter, count);
  }
  // u (+)= scale * (L_PDE k(X*))^T v
  void to_pred_cells(Plan& plan, const double* v, double* u, double scale, bool acc) {
    if (p->multi) {
      mo_to_pred_cells(plan, v, u, scale, acc);
      return;
    }
    int dc[3], dp[3];
    dims_cells(p, dc);
    dims_pred(p, dp);
    if (varcoef()) {
      const bool k0 = keep;
      if (!k0) stage_begin();
      const std::vector<int> cls = field_classes(p);
      const std::vector<const double*> win = vc_inputs(plan, v, cls);
      vc_sum_in(plan, dc, dp, ppred_terms(p), cls, win, scale * p->s2, u, acc);
      if (!k0) stage_end();
      return;
    }
    kron(plan, dc, dp, 1, ppred_terms(p), scale * p->s2, v, u, acc ? 1.0 : 0.0, nullptr, 0.0);
  }
  // out = scale * L_PDE k(X*) beta (prediction grid -> cells)
  void from_pred_cells(Plan& plan, const double* beta, double* out, double scale) {
    int dc[3], dp[3];
    dims_cells(p, dc);
    dims_pred(p, dp);
    if (varcoef()) {
      const bool k0 = keep;
      if (!k0) stage_begin();
      vc_sum_out(plan, dp, predp_terms(p), field_classes(p), beta, scale * p->s2, out, false);
      if (!k0) stage_end();
      return;
    }
    kron(plan, dp, dc, 1, predp_terms(p), scale * p->s2, beta, out, 0.0, nullptr, 0.0);
  }
  // g = L_IC,BC k(X*) beta (prediction grid -> all sets; fold: set 0 in its eigenbasis)
  void from_pred_sets(Plan& plan, const double* beta, double* g, bool fold) {
    int ds[3], dp[3];
    dims_pred(p, dp);
    for (int s = 0; s < p->nsets; ++s) {
      dims_set(p, s, ds);
      kron(plan, dp, ds, 1, predb_terms(p, s, fold), p->s2, beta, at(g, p->sets[s].off), 0.0, nullptr, 0.0);
    }
  }
  void to_pred_sets(Plan& plan, const double* w, double* u, double scale, bool acc, bool fold = false) {
    if (p->multi) {
      mo_to_pred_sets(plan, w, u, scale, acc);
      return;
    }
    int ds[3], dp[3];
    dims_pred(p, dp);
    for (int s = 0; s < p->nsets; ++s) {
      dims_set(p, s, ds);
      kron(plan, ds, dp, 1, bpred_terms(p, s, fold), scale * p->s2, at(w, p->sets[s].off), u,
           (acc || s > 0) ? 1.0 : 0.0, nullptr, 0.0);
    }
  }

  // ---- systems (Sec. 3.3): block by block, sequential FP64 Kronecker chains
  // (no face forms, digit products, tensor cores or structured IC/BC stage).
  // PDE vectors: neq blocks of Nc cells; predictions: nout blocks of Pp points.
  void zero(Plan& plan, double* x, i64 n) {
    plan.func([=](cudaStream_t st) { GPFVM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st)); });
  }
  // out_e = sum_e2 G_PP[e, e2] in_e2 + jitter in_e (the diagonal block first: it carries the jitter)
  void mo_pp(Plan& plan, const double* in, double* out) {
    int dc[3];
    dims_cells(p, dc);
    const i64 Nc = p->Nc;
    for (int e = 0; e < p->neq; ++e) {
      bool first = true;
      for (int k = 0; k < p->neq; ++k) {
        const int e2 = (e + k) % p->neq;
        const std::vector<KTerm> ts = pp_terms_mo(p, e, e2);
        if (ts.empty()) continue;
        kron(plan, dc, dc, 1, ts, p->s2, in + e2 * Nc, out + e * Nc, first ? 0.0 : 1.0, first ? in + e * Nc : nullptr,
             first ? p->jitter : 0.0);
        first = false;
      }
    }
  }
  // g_s = sum_e G_BP[s, e] in_e for every set s
  void mo_bp(Plan& plan, const double* in, double* g) {
    int dc[3], ds[3];
    dims_cells(p, dc);
    for (int s = 0; s < p->nsets; ++s) {
      dims_set(p, s, ds);
      bool first = true;
      for (int e = 0; e < p->neq; ++e) {
        const std::vector<KTerm> ts = pb_terms_mo(p, s, e, true);
        if (ts.empty()) continue;
        kron(plan, dc, ds, 1, ts, p->s2, in + e * p->Nc, g + p->sets[s].off, first ? 0.0 : 1.0, nullptr, 0.0);
        first = false;
      }
      if (first) zero(plan, g + p->sets[s].off, p->sets[s].size);  // no equation involves its output
    }
  }
  // out_e (+)= scale sum_s G_PB[e, s] w_s
  void mo_pb(Plan& plan, const double* w, double* out, double scale, bool accumulate) {
    int dc[3], ds[3];
    dims_cells(p, dc);
    for (int e = 0; e < p->neq; ++e) {
      bool first = !accumulate;
      for (int s = 0; s < p->nsets; ++s) {
        const std::vector<KTerm> ts = pb_terms_mo(p, s, e, false);
        if (ts.empty()) continue;
        dims_set(p, s, ds);
        kron(plan, ds, dc, 1, ts, scale * p->s2, w + p->sets[s].off, out + e * p->Nc, first ? 0.0 : 1.0, nullptr, 0.0);
        first = false;
      }
      if (first) zero(plan, out + e * p->Nc, p->Nc);
    }
  }
  // u_j (+)= scale sum_e (L_e k(X*_j))^T v_e for every output j
  void mo_to_pred_cells(Plan& plan, const double* v, double* u, double scale, bool acc) {
    int dc[3], dp[3];
    dims_cells(p, dc);
    dims_pred(p, dp);
    for (int j = 0; j < p->nout; ++j) {
      bool first = !acc;
      for (int e = 0; e < p->neq; ++e) {
        const std::vector<KTerm> ts = ppred_terms_mo(p, e, j);
        if (ts.empty()) continue;
        kron(plan, dc, dp, 1, ts, scale * p->s2, v + e * p->Nc, u + j * p->Pp, first ? 0.0 : 1.0, nullptr, 0.0);
        first = false;
      }
      if (first) zero(plan, u + j * p->Pp, p->Pp);
    }
  }
  // u_j (+)= scale sum over the sets s observing output j of k_s(X*_j)^T w_s
  void mo_to_pred_sets(Plan& plan, const double* w, double* u, double scale, bool acc) {
    int ds[3], dp[3];
    dims_pred(p, dp);
    for (int j = 0; j < p->nout; ++j) {
      bool first = !acc;
      for (int s = 0; s < p->nsets; ++s) {
        if (p->sets[s].comp != j) continue;
        dims_set(p, s, ds);
        kron(plan, ds, dp, 1, bpred_terms(p, s), scale * p->s2, w + p->sets[s].off, u + j * p->Pp,
             first ? 0.0 : 1.0, nullptr, 0.0);
        first = false;
      }
      if (first) zero(plan, u + j * p->Pp, p->Pp);
    }
  }
  // out = G^ in = G_PP in - G_PB G_BB^-1 G_BP in; with u also u = Lhat k(X*)^T in
  void mo_ghat(Plan& plan, const double* in, double* out, double* g, double* w, double* u) {
    mo_pp(plan, in, out);
    if (p->M > 0) {
      mo_bp(plan, in, g);
      hsolve(plan, g, w);
      mo_pb(plan, w, out, -1.0, true);
    }
    if (u) {
      mo_to_pred_cells(plan, in, u, 1.0, false);
      if (p->M > 0) mo_to_pred_sets(plan, w, u, -1.0, true);
    }
  }
};

// Exponent scratch of the digit-product dense GEMMs (null Aexp: FMA GEMMs).
OzChol ozchol(gpfvm_problem* p, int* status) {
  OzChol o{};
  if (!p->oz_on || !p->d_ozgexp) return o;
  o.Aexp = p->d_ozgexp;
  o.Bexp = p->d_ozgexp + p->ozg_cap;
  o.cap = p->ozg_cap;
  o.status = status;
  return o;
}

// Structured IC/BC assembly (see icbc.cu): eigen-decompose set 0's 1D
// factors, form the Schur complement of the other sets and factorise it.
void build_sicbc(gpfvm_problem* p, Builder& B) {
  Plan& pl = p->p_chol;
  const int M = (int)p->M, MK = p->MK, MR = p->MR, d = p->d;
  int maxn = 1;
  for (int i = 0; i < d; ++i) maxn = std::max(maxn, p->nK[i]);
  gpfvm_problem* pp = p;
  pl.func([=](cudaStream_t st) {
    launch_jacobi(pp->d_jac, pp->d, maxn, st);
    lambda_tensor(pp->d_lam[0], d >= 2 ? pp->d_lam[1] : nullptr, d >= 3 ? pp->d_lam[2] : nullptr, pp->nK[0],
                  d >= 2 ? pp->nK[1] : 1, d >= 3 ? pp->nK[2] : 1, pp->s2, pp->sets[0].noise,
                  pp->sets[0].order2 >= 0 ? pp->d_QK[0] : nullptr, pp->sets[0].noise2, pp->d_lt, st);
    recip(pp->d_lt, pp->d_ltinv, MK, st);
  });
  // fold the eigenbasis into set 0's factors: cells (F_i Q_i), prediction
  // grid (Q_i^T C_i) and the other sets (F_i(s, 0) Q_i)
  for (auto& ko : p->facq_off) {
    int ax, ka, aa, kb, ab;
    std::tie(ax, ka, aa, kb, ab) = ko.first;
    const int n = p->nK[ax];
    const double* src = p->d_fac + p->fac_off.at(ko.first);
    GemmDesc g{};
    g.batch = 1;
    if (kb == 1) {  // F Q: (rows x n) (n x n)
      g.m = (int)fam_n(p, ax, ka, aa); g.n = n; g.k = n;
      g.a_rs = n; g.a_cs = 1; g.b_rs = n; g.b_cs = 1; g.c_rs = n;
      g.tile = dense_tile(g.m, g.n);
      pl.gemm(g, {{GemmGroup{p->d_facq + ko.second, nullptr, 0.0, 0.0, 0, 0}, {GemmSeg{src, p->d_QK[ax], 1.0}}}});
    } else {  // Q_i^T C_i: (n x n) (n x pred)
      g.m = n; g.n = p->npred[ax]; g.k = n;
      g.a_rs = 1; g.a_cs = n; g.b_rs = g.n; g.b_cs = 1; g.c_rs = g.n;
      g.tile = dense_tile(g.m, g.n);
      pl.gemm(g, {{GemmGroup{p->d_facq + ko.second, nullptr, 0.0, 0.0, 0, 0}, {GemmSeg{p->d_QK[ax], src, 1.0}}}});
    }
  }
  if (MR > 0) {
    // E~ elementwise from the folded cross factors; S = G_RR - G_RK A^-1 G_KR
    // with G_RK A^-1 G_KR = sigma^2 E~ ((x)C[s'])^T, a Kronecker product
    // applied to the rows of E~ for each set s'
    EtildeSets ES{};
    ES.ns = p->nsets - 1;
    for (int s = 1; s < p->nsets; ++s) {
      ES.off[s - 1] = (int)(p->sets[s].off - MK);
      for (int i = 0; i < 3; ++i) {
        ES.n[s - 1][i] = i < d ? p->sets[s].n[i] : 1;
        ES.c[s - 1][i] = i < d ? p->d_facq + p->facq_off.at(FKey(i, 1, s, 1, 0)) : nullptr;
      }
    }
    const int nk0 = p->nK[0], nk1 = d >= 2 ? p->nK[1] : 1, nk2 = d >= 3 ? p->nK[2] : 1;
    pl.func([=](cudaStream_t st) {
      etilde(ES, nk0, nk1, nk2, pp->s2, pp->d_ltinv, pp->d_Et, MR, st);
      transpose(pp->d_Et, pp->d_EtT, MR, MK, st);
      GPFVM_CUDA(cudaMemcpy2DAsync(pp->d_Sc, sizeof(double) * MR, pp->d_A + (i64)MK * M + MK, sizeof(double) * M,
                                   sizeof(double) * MR, MR, cudaMemcpyDeviceToDevice, st));
      GPFVM_CUDA(cudaMemsetAsync(pp->d_LS, 0, sizeof(double) * MR * MR, st));
      GPFVM_CUDA(cudaMemsetAsync(pp->d_LSinv, 0, sizeof(double) * MR * MR, st));
    });
    int dK[3];
    dims_set(p, 0, dK);
    for (int s = 1; s < p->nsets; ++s) {
      int ds[3];
      dims_set(p, s, ds);
      KTerm T{};
      T.c = 1.0;
      for (int i = 0; i < d; ++i) T.f[i] = MatRef{p->d_facq + p->facq_off.at(FKey(i, 1, s, 1, 0)), p->nK[i], 1};
      B.kron(pl, dK, ds, MR, {T}, p->s2, p->d_Et, p->d_Tsc, 0.0, nullptr, 0.0);
      const i64 offR = p->sets[s].off - MK;
      const int ms = (int)p->sets[s].size;
      pl.func([=](cudaStream_t st) { axpy_block(pp->d_Sc + offR, MR, pp->d_Tsc, ms, MR, ms, -1.0, st); });
    }
    // (FP64 FMA: the factorisation of these decaying, ill-conditioned Gram
    // matrices needs errors relative to sum |a_k b_k|, which the fixed-point
    // digit products, relative to max |a| max |b| per window, do not give)
    plan_chol_inverse(pl, p->d_Sc, p->d_LS, p->d_LSinv, MR, MR, p->d_sscr, p->d_st ? &p->d_st->pad[0] : nullptr);
    pl.func([=](cudaStream_t st) { transpose(pp->d_LSinv, pp->d_LSinvT, MR, MR, st); });
  }
  pl.func([=](cudaStream_t st) {
    for (int i = 0; i < d; ++i) convert_d2f(pp->d_QK[i], pp->f_QK[i], (i64)pp->nK[i] * pp->nK[i], st);
    convert_d2f(pp->d_facq, pp->f_facq, pp->nfacq, st);
    if (MR > 0) {
      convert_d2f(pp->d_Et, pp->f_Et, (i64)MR * MK, st);
      convert_d2f(pp->d_EtT, pp->f_EtT, (i64)MR * MK, st);
      convert_d2f(pp->d_LSinv, pp->f_LSinv, (i64)MR * MR, st);
      convert_d2f(pp->d_LSinvT, pp->f_LSinvT, (i64)MR * MR, st);
    }
  });
}

// Cholesky-stage variance with the structured IC/BC stage:
//   k_B^T G_BB^-1 k_B = k_K^T A^-1 k_K + || L_S^-1 (k_R - F^T k_K) ||^2
// with F = A^-1 G_KR.  Term 1 = sigma^4 sum_m prod_i H_i[m_i,p_i]^2 / lambda~[m]
// with H_i = Q_i^T C_i (the folded prediction factor of set 0) is itself a
// Kronecker product applied to the tensor 1/lambda~; in term 2,
// F^T k_K = E~ (x)H_i k, so R = L_S^-1 E~ meets the folded factors; it runs
// over row chunks.
void build_sicbc_var(gpfvm_problem* p, Builder& B) {
  Plan& pl = p->p_vB;
  const int MK = p->MK, MR = p->MR, d = p->d;
  const i64 P = p->P;
  int dK[3], dP[3], ds[3];
  dims_set(p, 0, dK);
  dims_pred(p, dP);
  KTerm T1{};
  T1.c = 1.0;
  for (int i = 0; i < d; ++i) {
    const int n = p->nK[i], pi = p->npred[i];
    const double* H = p->d_facq + p->facq_off.at(FKey(i, 1, 0, 2, 0));
    double* Hs = p->d_Hsq[i];
    pl.func([=](cudaStream_t st) { square(H, Hs, (i64)n * pi, st); });
    T1.f[i] = MatRef{p->d_Hsq[i], 1, pi};
  }
  B.kron(pl, dK, dP, 1, {T1}, p->s2 * p->s2, p->d_ltinv, p->d_vB, 0.0, nullptr, 0.0);
  if (MR == 0) return;
  {
    GemmDesc g{};
    g.m = MR; g.n = MK; g.k = MR;
    g.a_rs = MR; g.a_cs = 1; g.b_rs = MK; g.b_cs = 1; g.c_rs = MK;
    g.batch = 1; g.tri = TRI_A_LOWER; g.tile = dense_tile(MR, MK);
    OzChol ozc = ozchol(p, &p->d_st->status);
    plan_dense_gemm(pl, g, GemmGroup{p->d_R, nullptr, 0.0, 0.0, 0, 0}, GemmSeg{p->d_LSinv, p->d_Et, 1.0},
                    ozc.Aexp ? &ozc : nullptr);
  }
  const int Rrows = p->vb_rows;
  double* vB = p->d_vB;
  for (int m0 = 0; m0 < MR; m0 += Rrows) {
    const int rows = std::min(Rrows, MR - m0);
    B.stage_begin();  // this chunk's intermediates (the previous chunk has finished with them)
    const bool face = B.var_face_chunk(pl, m0, rows, p->d_vbY);
    B.stage_end();
    if (face) {
      const double* Y = p->d_vbY;
      pl.func([=](cudaStream_t st) { colsumsq(Y, rows, P, vB, st); });
      continue;
    }
    bool first = true;
    for (int s = 1; s < p->nsets; ++s) {
      const i64 offR = p->sets[s].off - MK, ms = p->sets[s].size;
      if (offR > m0 + rows - 1) continue;  // L_S^-1 is lower triangular
      const double* src = p->d_LSinv + (i64)m0 * MR + offR;
      double* dst = p->d_vbchunk;
      pl.func([=](cudaStream_t st) {
        GPFVM_CUDA(cudaMemcpy2DAsync(dst, sizeof(double) * ms, src, sizeof(double) * MR, sizeof(double) * ms, rows,
                                     cudaMemcpyDeviceToDevice, st));
      });
      dims_set(p, s, ds);
      B.kron(pl, ds, dP, rows, bpred_terms(p, s), p->s2, p->d_vbchunk, p->d_vbY, first ? 0.0 : 1.0, nullptr, 0.0);
      first = false;
    }
    B.kron(pl, dK, dP, rows, bpred_terms(p, 0, true), -p->s2, p->d_R + (i64)m0 * MK, p->d_vbY, first ? 0.0 : 1.0,
           nullptr, 0.0);
    const double* Y = p->d_vbY;
    pl.func([=](cudaStream_t st) { colsumsq(Y, rows, P, vB, st); });
  }
}

// FP64 G_PP on the tensor cores by exact digit products (oz.cu): the shared
// three-level form with rotating axes of the tensor-core FP32 form, with FP64
// tensors, a row-exponent pass before every level and factor digit images
// sliced once per assembly.
struct OzBuild {
  gpfvm_problem* p;
  std::vector<OzOp> ops;
  std::map<std::pair<i64, double>, std::pair<i64, i64>> img;  // (factor offset, alpha) -> (image bytes, exponents)
  i64 img_n = 0, fexp_n = 0, exp_n = 0;
  bool ok = true;
  std::pair<const unsigned char*, const int*> image(i64 fo, int n, double alpha) {
    auto key = std::make_pair(fo, alpha);
    auto it = img.find(key);
    if (it == img.end()) {
      it = img.emplace(key, std::make_pair(img_n, fexp_n)).first;
      p->oz_jobs.push_back({fo, n, alpha, img_n, fexp_n});
      img_n += oz_image_bytes(n, n);
      fexp_n += (n + 31) / 32 * 32;
    }
    return {p->d_ozimg ? p->d_ozimg + it->second.first : nullptr,
            p->d_ozfexp ? p->d_ozfexp + it->second.second : nullptr};
  }
};

void build_oz_instance(gpfvm_problem* p, OzBuild& O, const double* in, double* out, int inst, const int* skip) {
  const int d = p->d;
  int n[3] = {1, 1, 1};
  i64 Ntot = 1;
  for (int i = 0; i < d; ++i) {
    n[i] = p->nc[i];
    Ntot *= n[i];
    if (n[i] > OZ_KMAX) O.ok = false;
  }
  struct Term { double c; i64 f[3]; };
  std::vector<Term> terms;
  for (int a = 0; a < p->nterms; ++a)
    for (int b = 0; b < p->nterms; ++b) {
      Term t{p->coef[a] * p->coef[b], {0, 0, 0}};
      for (int i = 0; i < d; ++i) t.f[i] = p->fac_off.at(FKey(i, 0, p->alpha[a][i], 0, p->alpha[b][i]));
      terms.push_back(t);
    }
  auto& levels = p->oz_levels[inst];
  levels.clear();
  i64 exo = 0;  // exponent ints of this instance
  auto begin_level = [&](i64 R, int K) {
    gpfvm_problem::OzLevel L{};
    L.off = (int)O.ops.size();
    L.jobs.R = (int)R;
    L.jobs.K = K;
    L.jobs.skip = skip;
    levels.push_back(L);
  };
  // row exponents of source tensor `A` (index `src` of the level's jobs)
  auto job = [&](int src, const double* A) -> const int* {
    auto& J = levels.back().jobs;
    if (src >= OZ_MAXSEG) { O.ok = false; return nullptr; }
    while (J.n <= src) {
      J.A[J.n] = nullptr;
      J.ex[J.n] = p->d_ozexp ? p->d_ozexp + exo : nullptr;
      exo += ((i64)J.R + 31) / 32 * 32;
      J.n++;
    }
    J.A[src] = A;
    return J.ex[src];
  };
  auto blank = [&](i64 R, int K, int N, double* o) {
    OzOp op{};
    op.R = (int)R; op.K = K; op.N = N; op.out = o;
    op.skip = skip;
    return op;
  };
  auto seg = [&](OzOp& op, const double* A, const int* ex, i64 fo, int nf, double alpha) {
    if (op.nseg >= OZ_MAXSEG) { O.ok = false; return; }
    auto im = O.image(fo, nf, alpha);
    op.A[op.nseg] = A;
    op.Aexp[op.nseg] = ex;
    op.Bimg[op.nseg] = im.first;
    op.Bexp[op.nseg] = im.second;
    op.nseg++;
  };
  auto add_op = [&](OzOp op) {
    auto& L = levels.back();
    op.tile_begin = L.tiles;
    if (L.nops > 0 && L.n != op.N) O.ok = false;  // one tiling per launch
    L.n = op.N;
    L.tiles += oz_tiles(op.R, op.N);
    L.nops++;
    if (op.N > 128 || op.K > OZ_KMAX) O.ok = false;
    O.ops.push_back(op);
  };
  if (d == 1) {
    begin_level(1, n[0]);
    const int* ex = job(0, in);
    OzOp op = blank(1, n[0], n[0], out);
    for (auto& t : terms) seg(op, in, ex, t.f[0], n[0], p->s2 * t.c);
    op.D = in;
    op.gamma = p->jitter;
    add_op(op);
    O.exp_n = std::max(O.exp_n, exo);
    return;
  }
  std::vector<i64> U, Wf;
  std::vector<int> uo(terms.size()), wo(terms.size());
  for (size_t k = 0; k < terms.size(); ++k) {
    if (d == 3) {
      auto it = std::find(U.begin(), U.end(), terms[k].f[2]);
      uo[k] = (int)(it - U.begin());
      if (it == U.end()) U.push_back(terms[k].f[2]);
    }
    auto jt = std::find(Wf.begin(), Wf.end(), terms[k].f[0]);
    wo[k] = (int)(jt - Wf.begin());
    if (jt == Wf.end()) Wf.push_back(terms[k].f[0]);
  }
  p->oz_nu = std::max(p->oz_nu, (int)U.size());
  p->oz_nw = std::max(p->oz_nw, (int)Wf.size());
  auto Y = [&](int u) { return p->d_ozY ? p->d_ozY + (i64)u * Ntot : nullptr; };
  auto Z = [&](int w) { return p->d_ozZ ? p->d_ozZ + (i64)w * Ntot : nullptr; };
  if (d == 3) {
    begin_level((i64)n[0] * n[1], n[2]);
    const int* ex = job(0, in);
    for (size_t u = 0; u < U.size(); ++u) {
      OzOp op = blank((i64)n[0] * n[1], n[2], n[2], Y((int)u));
      seg(op, in, ex, U[u], n[2], 1.0);
      add_op(op);
    }
  }
  begin_level(d == 3 ? (i64)n[2] * n[0] : (i64)n[0], n[1]);
  std::vector<const int*> exY;
  if (d == 3)
    for (size_t u = 0; u < U.size(); ++u) exY.push_back(job((int)u, Y((int)u)));
  else
    exY.push_back(job(0, in));
  for (size_t w = 0; w < Wf.size(); ++w) {
    OzOp op = blank(d == 3 ? (i64)n[2] * n[0] : (i64)n[0], n[1], n[1], Z((int)w));
    std::vector<std::pair<std::pair<int, i64>, double>> acc;  // merged (source, factor) pairs
    for (size_t k = 0; k < terms.size(); ++k) {
      if (wo[k] != (int)w) continue;
      const int src = (d == 3) ? uo[k] : 0;
      bool merged = false;
      for (auto& a : acc)
        if (a.first.first == src && a.first.second == terms[k].f[1]) { a.second += terms[k].c; merged = true; }
      if (!merged) acc.push_back({{src, terms[k].f[1]}, terms[k].c});
    }
    for (auto& a : acc) seg(op, d == 3 ? Y(a.first.first) : in, exY[a.first.first], a.first.second, n[1], a.second);
    add_op(op);
  }
  begin_level(Ntot / n[0], n[0]);
  OzOp op = blank(Ntot / n[0], n[0], n[0], out);
  for (size_t w = 0; w < Wf.size(); ++w) seg(op, Z((int)w), job((int)w, Z((int)w)), Wf[w], n[0], p->s2);
  op.D = in;
  op.gamma = p->jitter;
  add_op(op);
  O.exp_n = std::max(O.exp_n, exo);
}

// The three instances and their op tables (counting pass: null buffers).
void build_oz(gpfvm_problem* p) {
  p->oz_jobs.clear();
  for (auto& L : p->oz_levels) L.clear();
  if (p->nfield > 0 || p->d < 2 || p->multi) {  // (one axis: a single row of up to 128 cells, FMA form)
    p->oz_ok = false;
    return;
  }
  OzBuild O{p};
  build_oz_instance(p, O, p->d_p, p->d_q, 0, p->d_st ? &p->d_st->done : nullptr);
  build_oz_instance(p, O, p->d_vin, p->d_vout, 1, nullptr);
  build_oz_instance(p, O, p->d_vin, p->d_vout, 2, p->d_mctl ? &p->d_mctl->first : nullptr);
  p->oz_ok = O.ok;
  p->oz_ops_total = (i64)O.ops.size();
  p->oz_img_total = O.img_n;
  p->oz_fexp_total = O.fexp_n;
  p->oz_exp_total = O.exp_n;
  if (!p->d_ozops || !O.ok) return;
  // host-side bounds check of every operand before any launch
  for (const OzOp& op : O.ops) {
    bool ok = p->mem.contains(op.out, 8LL * op.N * op.R) && (!op.D || p->mem.contains(op.D, 8LL * op.N * op.R));
    ok = ok && op.nseg >= 1 && op.K >= 1 && op.K <= OZ_KMAX && op.N >= 1 && op.N <= 128;
    for (int s = 0; s < op.nseg; ++s)
      ok = ok && p->mem.contains(op.A[s], 8LL * op.R * op.K) && p->mem.contains(op.Aexp[s], 4LL * op.R) &&
           p->mem.contains(op.Bimg[s], oz_image_bytes(op.N, op.K)) && p->mem.contains(op.Bexp[s], 4LL * op.N) &&
           ((uintptr_t)op.Bimg[s] & 15) == 0;
    if (!ok) throw CudaError{cudaErrorInvalidValue, "digit-product operand out of bounds"};
  }
  for (auto& lv : p->oz_levels)
    for (auto& L : lv)
      for (int j = 0; j < L.jobs.n; ++j)
        if (!p->mem.contains(L.jobs.A[j], 8LL * L.jobs.R * L.jobs.K) || !p->mem.contains(L.jobs.ex[j], 4LL * L.jobs.R))
          throw CudaError{cudaErrorInvalidValue, "digit-product exponent job out of bounds"};
  GPFVM_CUDA(cudaMemcpy(p->d_ozops, O.ops.data(), sizeof(OzOp) * O.ops.size(), cudaMemcpyHostToDevice));
}

// G_PP of instance `inst` as FUNC ops (one per level: exponent pass + mode products).
Plan oz_chain(gpfvm_problem* p, int inst) {
  Plan c;
  for (const auto& L : p->oz_levels[inst]) {
    const OzExpJobs J = L.jobs;
    const OzOp* ops = p->d_ozops ? p->d_ozops + L.off : nullptr;
    const int nops = L.nops;
    const i64 tiles = L.tiles;
    const int nl = L.n;
    int* status = &p->d_st->status;
    c.func([=](cudaStream_t st) {
      oz_row_exponents(J, st);
      launch_oz_modes(ops, nops, tiles, nl, status, st);
    });
  }
  return c;
}

// The op table of the digit-product chains built by Builder::kron_digits:
// bounds-checked on the host and copied once the buffers exist (real pass).
void finish_ozx(gpfvm_problem* p) {
  if (!p->d_ozxops || p->ozx_ops.empty()) return;
  if ((i64)p->ozx_ops.size() > p->ozx_ops_cap) throw CudaError{cudaErrorInvalidValue, "digit-product op table"};
  for (const OzOp& op : p->ozx_ops) {
    bool ok = p->mem.contains(op.out, 8LL * op.N * op.R) && (!op.D || p->mem.contains(op.D, 8LL * op.N * op.R));
    ok = ok && op.nseg >= 1 && op.K >= 1 && op.K <= OZ_KMAX && op.N >= 1 && op.N <= 128;
    for (int s = 0; s < op.nseg; ++s)
      ok = ok && p->mem.contains(op.A[s], 8LL * op.R * op.K) && p->mem.contains(op.Aexp[s], 4LL * op.R) &&
           p->mem.contains(op.Bimg[s], oz_image_bytes(op.N, op.K)) && p->mem.contains(op.Bexp[s], 4LL * op.N) &&
           ((uintptr_t)op.Bimg[s] & 15) == 0;
    if (!ok) throw CudaError{cudaErrorInvalidValue, "digit-product operand out of bounds"};
  }
  for (const auto& j : p->ozx_jobs)
    if (!p->mem.contains(j.F, 8LL * (1 + (j.N - 1) * j.rs + (j.K - 1) * j.cs)))
      throw CudaError{cudaErrorInvalidValue, "digit-product factor out of bounds"};
  GPFVM_CUDA(cudaMemcpy(p->d_ozxops, p->ozx_ops.data(), sizeof(OzOp) * p->ozx_ops.size(), cudaMemcpyHostToDevice));
}

void build_plans(gpfvm_problem* p, Builder& B) {
  const i64 N = p->N, M = p->M, P = p->P;
  p->ozx_ops.clear();
  p->ozx_jobs.clear();
  p->ozx_img.clear();
  p->ozx_img_n = p->ozx_fexp_n = 0;
  gpfvm_problem* pp_ = p;
  // ---- setup: factors + G_BB
  p->p_setup = Plan();
  {
    FactorJob* dj = p->d_jobs;
    const int nj = (int)p->jobs.size();
    const i64 me = p->max_entries;
    p->p_setup.func([=](cudaStream_t st) { launch_factors(dj, nj, me, st); });
    if (M > 0) {
      GbbParams G{};
      G.M = (int)M;
      G.ndim = p->d;
      G.n_sets = p->nsets;
      G.outputscale = p->s2;
      for (int s = 0; s < p->nsets; ++s) {
        G.off[s] = (int)p->sets[s].off;
        G.noise[s] = p->sets[s].noise;
        G.noise2[s] = p->sets[s].order2 >= 0 ? p->sets[s].noise2 : p->sets[s].noise;
        G.comp[s] = p->sets[s].comp;
        for (int i = 0; i < p->d; ++i) G.dims[s][i] = p->sets[s].n[i];
        for (int s2 = 0; s2 < p->nsets; ++s2)
          for (int i = 0; i < p->d; ++i)
            G.fac[s][s2][i] = p->d_fac ? p->d_fac + p->fac_off.at(FKey(i, 1, s, 1, s2)) : nullptr;
      }
      G.off[p->nsets] = (int)M;
      double* A = p->d_A;
      p->p_setup.func([=](cudaStream_t st) { launch_gbb(G, A, st); });
    }
  }
  // ---- IC/BC Cholesky + inverse
  p->p_chol = Plan();
  if (M > 0 && p->sicbc) {
    build_sicbc(p, B);
  } else if (M > 0) {
    int* status = p->d_st ? &p->d_st->pad[0] : nullptr;
    p->p_chol.func([=](cudaStream_t st) {
      GPFVM_CUDA(cudaMemsetAsync(pp_->d_L, 0, sizeof(double) * M * M, st));
      GPFVM_CUDA(cudaMemsetAsync(pp_->d_Linv, 0, sizeof(double) * M * M, st));
    });
    plan_chol_inverse(p->p_chol, p->d_A, p->d_L, p->d_Linv, (int)M, M, p->d_cscr, status);
    double* Li = p->d_Linv;
    double* LiT = p->d_LinvT;
    p->p_chol.func([=](cudaStream_t st) { transpose(Li, LiT, (int)M, (int)M, st); });
  }
  // ---- conditioned right-hand side b = y_P - G_PB G_BB^-1 y_B
  p->p_rhs = Plan();
  {
    double* b = p->d_b;
    const double* rhs = p->d_rhs;
    p->p_rhs.func([=](cudaStream_t st) {
      if (rhs) GPFVM_CUDA(cudaMemcpyAsync(b, rhs, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      else GPFVM_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * N, st));
    });
    if (M > 0 && p->sicbc) {
      B.to_eigenbasis(p->p_rhs, p->d_yB, p->d_yBt);
      B.hsolve(p->p_rhs, p->d_yBt, p->d_w);
      B.pb(p->p_rhs, p->d_w, b, -1.0, true, true);
    } else if (M > 0) {
      B.hsolve(p->p_rhs, p->d_yB, p->d_w);
      B.pb(p->p_rhs, p->d_w, b, -1.0, true);
    }
  }
  // ---- CG iteration plans (phased: independent mode products share launches);
  // G_PP by digit products on the tensor cores where available and chosen
  build_oz(p);
  const bool oz = p->oz_ok && p->oz_on && p->d_ozops;
  p->p_mv_cg = Plan();
  p->modeprods_pp = 0;
  {
    Plan c = oz ? oz_chain(p, 0) : Plan();
    B.ghat_phased(p->p_mv_cg, p->d_p, p->d_q, p->d_g, p->d_w, nullptr, &p->modeprods_pp, oz ? &c : nullptr,
                  &p->d_st->done);
  }
  p->p_mvv_cg = Plan();
  {
    Plan c = oz ? oz_chain(p, 0) : Plan();
    B.ghat_phased(p->p_mvv_cg, p->d_p, p->d_q, p->d_g, p->d_w, p->d_u, nullptr, oz ? &c : nullptr, &p->d_st->done);
  }
  p->p_var_cg = Plan();
  B.to_pred_cells(p->p_var_cg, p->d_p, p->d_u, 1.0, false);
  if (M > 0) B.to_pred_sets(p->p_var_cg, p->d_w, p->d_u, -1.0, true, true);
  // ---- operator plans for gpfvm_gram_matvec / true residual
  for (int k = 0; k < 6; ++k) p->p_op[k] = Plan();
  B.pp(p->p_op[0], p->d_vin, p->d_vout, nullptr);
  B.fma_only = true;  // op 1: every product in FP64 FMA
  B.ghat_phased(p->p_op[1], p->d_vin, p->d_vout, p->d_g2, p->d_wout, nullptr, nullptr);
  B.fma_only = false;
  if (p->oz_ok) {  // (in the counting pass too: the digit chains of G^ need op-table room)
    p->p_op[4] = oz_chain(p, 1);
    Plan c = oz_chain(p, 1);
    B.ghat_phased(p->p_op[5], p->d_vin, p->d_vout, p->d_g2, p->d_wout, nullptr, nullptr, &c);
  }
  p->p_res = Plan();
  {
    Plan c = oz ? oz_chain(p, 2) : Plan();
    B.ghat_phased(p->p_res, p->d_vin, p->d_vout, p->d_g2, p->d_wout, nullptr, nullptr, oz ? &c : nullptr,
                  &p->d_mctl->first);
  }
  if (M > 0) {
    B.bp(p->p_op[2], p->d_vin, p->d_wout);
    B.pb(p->p_op[3], p->d_win, p->d_vout, 1.0, false);
  }
  // ---- posterior mean
  p->p_mean = Plan();
  if (M > 0) {
    // with the structured stage, g and y~_B hold set 0 in its eigenbasis
    B.bp(p->p_mean, p->d_x, p->d_g, true);
    double *g = p->d_g, *g2 = p->d_g2;
    const double* yB = p->sicbc ? p->d_yBt : p->d_yB;
    p->p_mean.func([=](cudaStream_t st) { axpby(yB, g, g2, 1.0, -1.0, M, st); });
    B.hsolve(p->p_mean, p->d_g2, p->d_w);
    B.to_pred_sets(p->p_mean, p->d_w, p->d_mean, 1.0, false, true);
  }
  B.to_pred_cells(p->p_mean, p->d_x, p->d_mean, 1.0, M > 0);
  // ---- targeted actions (appendix "Targeted uncertainty reduction"):
  // p = Lhat k(X*) beta = L_PDE k(X*) beta - G_PB G_BB^-1 L_IC,BC k(X*) beta
  p->p_tgt = Plan();
  if (!p->multi) {  // (targeted actions: one-output problems)
    B.from_pred_cells(p->p_tgt, p->d_tbeta, p->d_p, 1.0);
    if (M > 0) {
      B.from_pred_sets(p->p_tgt, p->d_tbeta, p->d_g2, p->sicbc);
      B.hsolve(p->p_tgt, p->d_g2, p->d_wout);
      B.pb(p->p_tgt, p->d_wout, p->d_p, -1.0, true, p->sicbc);
    }
  }
  // ---- Cholesky-stage variance term vB[p] = || L^-1 k_B(x_p) ||^2 in row chunks
  p->p_vB = Plan();
  if (M > 0 && p->sicbc) {
    build_sicbc_var(p, B);
  } else {
    double* vB = p->d_vB;
    p->p_vB.func([=](cudaStream_t st) { GPFVM_CUDA(cudaMemsetAsync(vB, 0, sizeof(double) * P, st)); });
    const int R = p->vb_rows;
    int dp[3], ds[3];
    dims_pred(p, dp);
    const i64 Pp = p->Pp;
    for (i64 m0 = 0; m0 < M && R > 0; m0 += R) {
      const int rows = (int)std::min<i64>(R, M - m0);
      for (int j = 0; j < p->nout; ++j) {  // (systems: the sets of output j give its grid's term)
        bool first = true;
        for (int s = 0; s < p->nsets; ++s) {
          const i64 off = p->sets[s].off, ms = p->sets[s].size;
          if (p->sets[s].comp != j) continue;
          if (off > m0 + rows - 1) continue;  // L^-1 is lower triangular: these columns are zero
          const double* src = p->d_Linv + m0 * M + off;
          double* dst = p->d_vbchunk;
          p->p_vB.func([=](cudaStream_t st) {
            GPFVM_CUDA(cudaMemcpy2DAsync(dst, sizeof(double) * ms, src, sizeof(double) * M, sizeof(double) * ms, rows,
                                         cudaMemcpyDeviceToDevice, st));
          });
          dims_set(p, s, ds);
          B.kron(p->p_vB, ds, dp, rows, bpred_terms(p, s), p->s2, p->d_vbchunk, p->d_vbY, first ? 0.0 : 1.0, nullptr,
                 0.0);
          first = false;
        }
        if (first) continue;
        const double* Y = p->d_vbY;
        double* vBj = vB + j * Pp;
        p->p_vB.func([=](cudaStream_t st) { colsumsq(Y, rows, Pp, vBj, st); });
      }
    }
  }
  finish_ozx(p);
}

// Tensor-core G_PP: the shared three-level form with rotating axes
// (contract the last axis, write the new axis first), see tc.cu.
// Builds the op tables of one instance (in -> out) and returns them by level.
struct TcBuild {
  gpfvm_problem* p;
  std::vector<TcOp> ops;
  std::map<std::tuple<i64, float, int>, i64> split_off;
  i64 split_n = 0;
  bool ok = true;
  const float* split(i64 fac_off, i64 n, float alpha, bool hi, int mode) {
    auto key = std::make_tuple(fac_off, alpha, mode);
    auto it = split_off.find(key);
    i64 off;
    if (it == split_off.end()) {
      off = split_n;
      split_off[key] = off;
      split_n += 2 * ((n + 63) / 64 * 64);
      p->tc_jobs.push_back(std::make_tuple(fac_off, alpha, n, off, mode));
    } else {
      off = it->second;
    }
    return p->f_tcsplit ? p->f_tcsplit + off + (hi ? 0 : (n + 63) / 64 * 64) : nullptr;
  }
};

// Tiles of the tensor-core levels.  A tile runs its (segment, K block) stages
// one after the other, so a level with few row tiles and several segments per
// op (the t level: 32 row tiles x 4 segments on 64^3 cells) is a long chain on
// a few SMs.  Such ops split their segments into groups, one tile per
// (row tile, group), as long as the level stays within about two resident
// CTAs per SM; the groups' partial sums are added in order by tc_sum.
static thread_local int g_tc_group_policy = 0;  // 0: split idle levels into groups, 1: never

void tc_group_levels(gpfvm_problem* p, TcBuild& T, int inst) {
  const i64 slots = g_tc_group_policy == 1 ? 1 : 2 * 152;
  for (auto& L : p->tc_levels[inst]) {
    i64 rows = 0;
    for (int o = L.off; o < L.off + L.nops; ++o) rows += (T.ops[o].R + 127) / 128;
    const i64 per = std::max<i64>(1, slots / std::max<i64>(rows, 1));
    L.tiles = 0;
    L.any_split = 0;
    i64 part = 0;
    for (int o = L.off; o < L.off + L.nops; ++o) {
      TcOp& op = T.ops[o];
      op.sgroups = (int)std::max<i64>(1, std::min<i64>(per, op.nseg));
      op.tile_begin = L.tiles;
      L.tiles += (i64)((op.R + 127) / 128) * op.sgroups;
      op.part = nullptr;
      if (op.sgroups > 1) {
        op.part = p->f_tcpart ? p->f_tcpart + part : nullptr;
        part += (i64)op.sgroups * op.N * op.R;
        L.any_split = 1;
      }
    }
    p->tc_part_total = std::max(p->tc_part_total, part);
  }
}

void build_tc_instance(gpfvm_problem* p, TcBuild& T, const float* in, float* out, int inst, int mode) {
  const int d = p->d;
  int n[3] = {1, 1, 1};
  i64 Ntot = 1;
  for (int i = 0; i < d; ++i) {
    n[i] = p->nc[i];
    Ntot *= n[i];
  }
  struct Term { double c; i64 f[3]; };
  std::vector<Term> terms;
  for (int a = 0; a < p->nterms; ++a)
    for (int b = 0; b < p->nterms; ++b) {
      Term t{p->coef[a] * p->coef[b], {0, 0, 0}};
      for (int i = 0; i < d; ++i) t.f[i] = p->fac_off.at(FKey(i, 0, p->alpha[a][i], 0, p->alpha[b][i]));
      terms.push_back(t);
    }
  auto fsize = [&](int ax) { return (i64)n[ax] * n[ax]; };
  p->tc_levels[inst].clear();
  auto begin_level = [&]() { p->tc_levels[inst].push_back({(int)T.ops.size(), 0, 0, 0, 0}); };
  auto add_op = [&](TcOp op) {
    auto& L = p->tc_levels[inst].back();
    L.nops++;
    L.maxn = std::max(L.maxn, op.N);
    if (op.nseg > TC_MAXSEG || op.N > 128) T.ok = false;
    T.ops.push_back(op);
  };
  auto seg = [&](TcOp& op, const float* A, i64 fo, int ax, double alpha) {
    if (op.nseg >= TC_MAXSEG) { T.ok = false; return; }
    op.A[op.nseg] = A;
    op.Bhi[op.nseg] = T.split(fo, fsize(ax), (float)alpha, true, mode);
    op.Blo[op.nseg] = T.split(fo, fsize(ax), (float)alpha, false, mode);
    op.nseg++;
  };
  auto blank = [&](int R, int K, int N, float* o) {
    TcOp op{};
    op.R = R; op.K = K; op.N = N; op.out = o;
    op.sgroups = 1;
    op.mode = mode;
    op.skip = (inst % 2 == 0 && p->d_st32) ? &p->d_st32->done : nullptr;
    return op;
  };
  if (d == 1) {
    begin_level();
    TcOp op = blank(1, n[0], n[0], out);
    for (auto& t : terms) seg(op, in, t.f[0], 0, p->s2 * t.c);
    op.D = in;
    op.gamma = (float)p->jitter;
    add_op(op);
    tc_group_levels(p, T, inst);
    return;
  }
  // distinct factors on the last axis (3 axes) and on axis 0
  std::vector<i64> U, Wf;
  std::vector<int> uo(terms.size()), wo(terms.size());
  for (size_t k = 0; k < terms.size(); ++k) {
    if (d == 3) {
      auto it = std::find(U.begin(), U.end(), terms[k].f[2]);
      uo[k] = (int)(it - U.begin());
      if (it == U.end()) U.push_back(terms[k].f[2]);
    }
    auto jt = std::find(Wf.begin(), Wf.end(), terms[k].f[0]);
    wo[k] = (int)(jt - Wf.begin());
    if (jt == Wf.end()) Wf.push_back(terms[k].f[0]);
  }
  p->tc_nu = std::max(p->tc_nu, (int)U.size());
  p->tc_nw = std::max(p->tc_nw, (int)Wf.size());
  if (d == 3) {
    begin_level();
    for (size_t u = 0; u < U.size(); ++u) {
      TcOp op = blank(n[0] * n[1], n[2], n[2], p->f_tcY ? p->f_tcY + u * Ntot : nullptr);
      seg(op, in, U[u], 2, 1.0);
      add_op(op);
    }
  }
  begin_level();
  for (size_t w = 0; w < Wf.size(); ++w) {
    TcOp op = (d == 3) ? blank(n[2] * n[0], n[1], n[1], p->f_tcZ ? p->f_tcZ + w * Ntot : nullptr)
                       : blank(n[0], n[1], n[1], p->f_tcZ ? p->f_tcZ + w * Ntot : nullptr);
    // merge equal (source, factor) pairs of the group
    std::vector<std::pair<std::pair<int, i64>, double>> acc;
    for (size_t k = 0; k < terms.size(); ++k) {
      if (wo[k] != (int)w) continue;
      const int src = (d == 3) ? uo[k] : -1;
      bool merged = false;
      for (auto& a : acc)
        if (a.first.first == src && a.first.second == terms[k].f[1]) { a.second += terms[k].c; merged = true; }
      if (!merged) acc.push_back({{src, terms[k].f[1]}, terms[k].c});
    }
    for (auto& a : acc) {
      const float* A = (d == 3) ? (p->f_tcY ? p->f_tcY + (i64)a.first.first * Ntot : nullptr) : in;
      seg(op, A, a.first.second, 1, a.second);
    }
    add_op(op);
  }
  begin_level();
  TcOp op = blank((int)(Ntot / n[0]), n[0], n[0], out);
  for (size_t w = 0; w < Wf.size(); ++w) seg(op, p->f_tcZ ? p->f_tcZ + (i64)w * Ntot : nullptr, Wf[w], 0, p->s2);
  op.D = in;
  op.gamma = (float)p->jitter;
  add_op(op);
  tc_group_levels(p, T, inst);
}

// G_PP on tensor cores as a chain of FUNC ops (one per level) for a phased plan.
Plan tc_chain(gpfvm_problem* p, int inst) {
  Plan c;
  for (auto L : p->tc_levels[inst])
    c.tc(p->d_tcops + L.off, L.nops, L.tiles, L.maxn, &p->d_st32->pad[1], L.any_split);
  return c;
}

// FP32 plans of the mixed solver's inner operator.
void build_plans32(gpfvm_problem* p, Builder& B) {
  if (p->multi) {  // systems are solved in FP64 only
    p->tc_ok = false;
    return;
  }
  B.f32 = true;
  p->building_f32 = true;
  auto D = [](float* f) { return (double*)f; };
  p->p_mv32 = Plan();
  B.ghat_phased(p->p_mv32, D(p->f_p), D(p->f_q), D(p->f_g), D(p->f_w), nullptr, nullptr);
  p->p_mvv32 = Plan();
  B.ghat_phased(p->p_mvv32, D(p->f_p), D(p->f_q), D(p->f_g), D(p->f_w), D(p->f_u), nullptr);
  p->p_var32 = Plan();
  B.to_pred_cells(p->p_var32, D(p->f_p), D(p->f_u), 1.0, false);
  if (p->M > 0) B.to_pred_sets(p->p_var32, D(p->f_w), D(p->f_u), -1.0, true, true);
  p->p_pp32 = Plan();
  B.pp(p->p_pp32, D(p->f_vin), D(p->f_vout), nullptr);
  // tensor-core variants of G_PP, one pair of instances per operand format
  // (not for variable coefficients: their products run on the SIMT plans)
  if (p->nfield > 0) {
    p->tc_ok = false;
    p->tc_split_total = 0;
    p->tc_ops_total = 0;
  } else {
    TcBuild T{p};
    for (int m = 0; m < 3; ++m) {
      build_tc_instance(p, T, p->f_p, p->f_q, 2 * m, m);
      build_tc_instance(p, T, p->f_vin, p->f_vout, 2 * m + 1, m);
    }
    p->tc_ok = T.ok;
    p->tc_split_total = T.split_n;
    p->tc_ops_total = (i64)T.ops.size();
    if (p->d_tcops && T.ok) {
      // host-side bounds check of every tensor-core operand before any launch
      for (const TcOp& op : T.ops) {
        bool ok = p->mem.contains(op.out, 4LL * op.N * op.R) && (!op.D || p->mem.contains(op.D, 4LL * op.N * op.R));
        ok = ok && op.sgroups >= 1 && op.sgroups <= op.nseg && op.mode >= 0 && op.mode <= 2 &&
             (op.sgroups == 1 || p->mem.contains(op.part, 4LL * op.sgroups * op.N * op.R));
        for (int s = 0; s < op.nseg; ++s)
          ok = ok && p->mem.contains(op.A[s], 4LL * op.R * op.K) && p->mem.contains(op.Bhi[s], 4LL * op.N * op.K) &&
               p->mem.contains(op.Blo[s], 4LL * op.N * op.K);
        if (!ok) throw CudaError{cudaErrorInvalidValue, "tc operand out of bounds"};
      }
      GPFVM_CUDA(cudaMemcpy(p->d_tcops, T.ops.data(), sizeof(TcOp) * T.ops.size(), cudaMemcpyHostToDevice));
    }
    if (p->tc_ok && p->d_tcops) {
      for (int m = 0; m < 3; ++m) {
        p->p_mv32tc[m] = Plan();
        Plan c0 = tc_chain(p, 2 * m);
        B.ghat_phased(p->p_mv32tc[m], D(p->f_p), D(p->f_q), D(p->f_g), D(p->f_w), nullptr, nullptr, &c0);
        p->p_mvv32tc[m] = Plan();
        Plan c1 = tc_chain(p, 2 * m);
        B.ghat_phased(p->p_mvv32tc[m], D(p->f_p), D(p->f_q), D(p->f_g), D(p->f_w), D(p->f_u), nullptr, &c1);
        p->p_pp32tc[m] = tc_chain(p, 2 * m + 1);
      }
    }
  }
  p->building_f32 = false;
  B.f32 = false;
}

void finalize_plans(gpfvm_problem* p) {
  p->p_mv_cg.skip = &p->d_st->done;
  p->p_mvv_cg.skip = &p->d_st->done;
  p->p_var_cg.skip = &p->d_st->done;
  p->p_mv32.skip = &p->d_st32->done;
  p->p_mvv32.skip = &p->d_st32->done;
  p->p_var32.skip = &p->d_st32->done;
  std::vector<Plan*> all = {&p->p_setup, &p->p_chol, &p->p_rhs, &p->p_mv_cg, &p->p_var_cg, &p->p_mean, &p->p_vB,
                            &p->p_op[0], &p->p_op[1], &p->p_op[2], &p->p_op[3], &p->p_mv32, &p->p_var32, &p->p_pp32,
                            &p->p_mvv_cg, &p->p_mvv32, &p->p_tgt, &p->p_res, &p->p_op[4], &p->p_op[5]};
  std::vector<std::string> names = {"setup", "chol", "rhs", "mv_cg", "var_cg", "mean", "vB", "op0", "op1", "op2",
                                    "op3", "mv32", "var32", "pp32", "mvv_cg", "mvv32", "tgt", "res", "op12", "op13"};
  p->p_res.skip = &p->d_mctl->first;
  for (int m = 0; m < 3; ++m) {
    all.push_back(&p->p_mv32tc[m]);
    all.push_back(&p->p_mvv32tc[m]);
    all.push_back(&p->p_pp32tc[m]);
    names.push_back("mv32tc" + std::to_string(m));
    names.push_back("mvv32tc" + std::to_string(m));
    names.push_back("pp32tc" + std::to_string(m));
  }
  for (size_t i = 0; i < all.size(); ++i) check_plan_ranges(*all[i], p->mem, names[i].c_str());
  for (int m = 0; m < 3; ++m) {
    p->p_mv32tc[m].skip = &p->d_st32->done;
    p->p_mvv32tc[m].skip = &p->d_st32->done;
  }
  if (!p->fan.fork) p->fan.create();
  for (Plan* pl : all) {
    pl->finalize();
    pl->fan = &p->fan;
  }
  // persistent forms of the iteration operators (used when GPFVM_PERSIST=1)
  Plan* fp64_plans[] = {&p->p_mv_cg, &p->p_mvv_cg, &p->p_op[0], &p->p_op[1]};
  std::vector<Plan*> fp32_plans = {&p->p_mv32, &p->p_mvv32, &p->p_pp32};
  for (int m = 0; m < 3; ++m) {
    fp32_plans.push_back(&p->p_mv32tc[m]);
    fp32_plans.push_back(&p->p_mvv32tc[m]);
    fp32_plans.push_back(&p->p_pp32tc[m]);
  }
  for (Plan* pl : fp64_plans) pl->prog = persist_build(*pl, p->d_psync, &p->d_st->status);
  for (Plan* pl : fp32_plans) pl->prog = persist_build(*pl, p->d_psync, &p->d_st32->pad[1]);
}

int validate(const gpfvm_desc* D) {
  if (!D) return GPFVM_ERR_INVALID_ARG;
  if (D->ndim < 1 || D->ndim > 3) return GPFVM_ERR_INVALID_ARG;
  if (D->n_terms < 1 || D->n_terms > GPFVM_MAX_TERMS) return GPFVM_ERR_INVALID_ARG;
  if (D->n_sets < 0 || D->n_sets > GPFVM_MAX_SETS) return GPFVM_ERR_INVALID_ARG;
  if (!(D->outputscale > 0) || !(D->jitter >= 0) || !std::isfinite(D->outputscale) || !std::isfinite(D->jitter))
    return GPFVM_ERR_INVALID_ARG;
  if (D->observe != 0 && D->observe != 1) return GPFVM_ERR_INVALID_ARG;
  if (D->fp64_products != 0 && D->fp64_products != 1) return GPFVM_ERR_INVALID_ARG;
  if (D->n_outputs < 0 || D->n_outputs > GPFVM_MAX_OUTPUTS) return GPFVM_ERR_INVALID_ARG;
  int neq = 1;
  const int nout = D->n_outputs > 0 ? D->n_outputs : 1;
  if (D->n_outputs > 0) {  // term_eq / term_out / set_out are read (0: one equation, one output)
    bool used[GPFVM_MAX_TERMS] = {};
    neq = 0;
    for (int k = 0; k < D->n_terms; ++k) {
      if (D->term_eq[k] < 0 || D->term_eq[k] >= GPFVM_MAX_TERMS) return GPFVM_ERR_INVALID_ARG;
      if (D->term_out[k] < 0 || D->term_out[k] >= nout) return GPFVM_ERR_INVALID_ARG;
      used[D->term_eq[k]] = true;
      neq = std::max(neq, D->term_eq[k] + 1);
    }
    for (int e = 0; e < neq; ++e)
      if (!used[e]) return GPFVM_ERR_INVALID_ARG;  // equations numbered without gaps
    for (int s = 0; s < D->n_sets; ++s)
      if (D->set_out[s] < 0 || D->set_out[s] >= nout) return GPFVM_ERR_INVALID_ARG;
    if (nout > 1 || neq > 1)
      for (int k = 0; k < D->n_terms; ++k)
        if (D->coef_field[k]) return GPFVM_ERR_INVALID_ARG;  // systems take constant coefficients
  }
  i64 N = neq, P = nout;
  for (int i = 0; i < D->ndim; ++i) {
    if (D->n_cells[i] < 1 || D->n_cells[i] > 65536 || !D->edges[i]) return GPFVM_ERR_INVALID_ARG;
    if (!(D->lengthscale[i] > 0) || !std::isfinite(D->lengthscale[i])) return GPFVM_ERR_INVALID_ARG;
    for (int j = 0; j < D->n_cells[i]; ++j)
      if (!(D->edges[i][j + 1] > D->edges[i][j]) || !std::isfinite(D->edges[i][j + 1])) return GPFVM_ERR_INVALID_ARG;
    if (D->n_pred[i] < 1 || D->n_pred[i] > 65536 || !D->pred[i]) return GPFVM_ERR_INVALID_ARG;
    for (int j = 0; j < D->n_pred[i]; ++j)
      if (!std::isfinite(D->pred[i][j])) return GPFVM_ERR_INVALID_ARG;
    N *= D->n_cells[i];
    P *= D->n_pred[i];
  }
  if (N > (i64)1 << 28 || P > (i64)1 << 28) return GPFVM_ERR_INVALID_ARG;
  bool any = false;
  for (int k = 0; k < D->n_terms; ++k) {
    if (!std::isfinite(D->coef[k])) return GPFVM_ERR_INVALID_ARG;
    any = any || D->coef[k] != 0.0;
    for (int i = 0; i < D->ndim; ++i)
      if (D->alpha[k][i] < 0 || D->alpha[k][i] > 2) return GPFVM_ERR_INVALID_ARG;
  }
  if (!any) return GPFVM_ERR_INVALID_ARG;
  i64 M = 0;
  for (int s = 0; s < D->n_sets; ++s) {
    const gpfvm_point_set& S = D->sets[s];
    if (!(S.noise_var >= 0) || !std::isfinite(S.noise_var)) return GPFVM_ERR_INVALID_ARG;
    i64 n = 1;
    for (int i = 0; i < D->ndim; ++i) {
      if (S.order[i] < 0 || S.order[i] > 1) return GPFVM_ERR_INVALID_ARG;
      if (S.n_pts[i] < 1 || S.n_pts[i] > 65536 || !S.coords[i]) return GPFVM_ERR_INVALID_ARG;
      for (int j = 0; j < S.n_pts[i]; ++j)
        if (!std::isfinite(S.coords[i][j])) return GPFVM_ERR_INVALID_ARG;
      n *= S.n_pts[i];
    }
    if (S.values)
      for (i64 j = 0; j < n; ++j)
        if (!std::isfinite(S.values[j])) return GPFVM_ERR_INVALID_ARG;
    M += n;
  }
  if (M > 65536) return GPFVM_ERR_INVALID_ARG;
  if (D->rhs)
    for (i64 j = 0; j < N; ++j)
      if (!std::isfinite(D->rhs[j])) return GPFVM_ERR_INVALID_ARG;
  for (int k = 0; k < D->n_terms; ++k)
    if (D->coef_field[k])
      for (i64 j = 0; j < N; ++j)
        if (!std::isfinite(D->coef_field[k][j])) return GPFVM_ERR_INVALID_ARG;
  for (int k = D->n_terms; k < GPFVM_MAX_TERMS; ++k)
    if (D->coef_field[k]) return GPFVM_ERR_INVALID_ARG;
  return GPFVM_OK;
}

}  // namespace

namespace {

cudaStream_t pick_stream(gpfvm_problem* p, void* s);

}  // namespace

static std::map<const gpfvm_problem*, cudaStream_t>& own_streams() {
  static std::map<const gpfvm_problem*, cudaStream_t> m;
  return m;
}

namespace {

cudaStream_t pick_stream(gpfvm_problem* p, void* s) {
  if (s) return (cudaStream_t)s;
  auto& m = own_streams();
  auto it = m.find(p);
  if (it != m.end()) return it->second;
  cudaStream_t st;
  GPFVM_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  m[p] = st;
  return st;
}

void alloc_all(gpfvm_problem* p) {
  const i64 N = p->N, M = p->M, P = p->P;
  DevBuf& m = p->mem;
  // coordinates
  std::vector<double> coords;
  for (int i = 0; i < p->d; ++i) {
    p->off_edges[i] = (i64)coords.size();
    coords.insert(coords.end(), p->edges[i].begin(), p->edges[i].end());
  }
  for (int s = 0; s < p->nsets; ++s)
    for (int i = 0; i < p->d; ++i) {
      p->off_set[s][i] = (i64)coords.size();
      coords.insert(coords.end(), p->sets[s].coords[i].begin(), p->sets[s].coords[i].end());
    }
  for (int i = 0; i < p->d; ++i) {
    p->off_pred[i] = (i64)coords.size();
    coords.insert(coords.end(), p->pred[i].begin(), p->pred[i].end());
  }
  for (int i = 0; i < p->d; ++i) {  // cell centres (the collocation points)
    p->off_mid[i] = (i64)coords.size();
    for (int j = 0; j < p->nc[i]; ++j) coords.push_back(0.5 * (p->edges[i][j] + p->edges[i][j + 1]));
  }
  p->d_coords = m.alloc<double>((i64)coords.size());
  GPFVM_CUDA(cudaMemcpy(p->d_coords, coords.data(), coords.size() * sizeof(double), cudaMemcpyHostToDevice));
  // factors
  i64 nfac = 0;
  for (auto& j : p->jobs) nfac += (i64)j.n_a * j.n_b;
  p->d_fac = m.alloc<double>(std::max<i64>(nfac, 1));
  for (auto& key_off : p->fac_off) {
    int ax, ka, aa, kb, ab;
    std::tie(ax, ka, aa, kb, ab) = key_off.first;
    for (auto& J : p->jobs)
      if ((i64)(intptr_t)J.out == key_off.second && (intptr_t)J.ca == ka * 1000 + aa && (intptr_t)J.cb == kb * 1000 + ab) {
        auto cptr = [&](int k, int a) -> const double* {
          if (k == 0) return p->d_coords + (p->colloc ? p->off_mid[ax] : p->off_edges[ax]);
          if (k == 1) return p->d_coords + p->off_set[a][ax];
          return p->d_coords + p->off_pred[ax];
        };
        J.ca = cptr(ka, aa);
        J.cb = cptr(kb, ab);
        J.out = p->d_fac + key_off.second;
        break;
      }
  }
  p->d_jobs = m.alloc<FactorJob>((i64)p->jobs.size());
  GPFVM_CUDA(cudaMemcpy(p->d_jobs, p->jobs.data(), p->jobs.size() * sizeof(FactorJob), cudaMemcpyHostToDevice));
  // IC/BC matrices: the structured stage needs set 0 to be the largest set,
  // to carry noise, and to have at most 96 points per axis (Jacobi in shared
  // memory); GPFVM_ICBC=dense forces the dense Cholesky of all of G_BB.
  p->sicbc = false;
  if (M > 0) {
    const char* env = getenv("GPFVM_ICBC");
    bool ok = !(env && std::strcmp(env, "dense") == 0) && p->sets[0].noise > 0 &&
              (p->sets[0].order2 < 0 || p->sets[0].noise2 > 0) && !p->multi;
    for (int s = 1; s < p->nsets; ++s) ok = ok && p->sets[s].size <= p->sets[0].size;
    for (int i = 0; i < p->d; ++i) ok = ok && p->sets[0].n[i] <= 96;
    p->sicbc = ok;
  }
  if (M > 0 && p->sicbc) {
    p->MK = (int)p->sets[0].size;
    p->MR = (int)(M - p->MK);
    const i64 MK = p->MK, MR = p->MR;
    p->d_A = m.alloc<double>(M * M);
    std::vector<JacobiJob> jobs(p->d);
    p->d_jac_sweeps = m.alloc<int>(2 * p->d);
    GPFVM_CUDA(cudaMemset(p->d_jac_sweeps, 0, sizeof(int) * 2 * p->d));
    for (int i = 0; i < p->d; ++i) {
      const int n = p->sets[0].n[i];
      p->nK[i] = n;
      p->d_QK[i] = m.alloc<double>((i64)n * n);
      p->d_lam[i] = m.alloc<double>(n);
      p->f_QK[i] = m.alloc<float>((i64)n * n);
      p->d_Hsq[i] = m.alloc<double>((i64)n * p->npred[i]);
      jobs[i] = JacobiJob{p->d_fac + p->fac_off.at(FKey(i, 1, 0, 1, 0)), p->d_QK[i], p->d_lam[i], n, 1e-14,
                          p->d_jac_sweeps + 2 * i};
    }
    p->d_jac = m.alloc<JacobiJob>(p->d);
    GPFVM_CUDA(cudaMemcpy(p->d_jac, jobs.data(), sizeof(JacobiJob) * p->d, cudaMemcpyHostToDevice));
    p->d_lt = m.alloc<double>(MK);
    p->d_ltinv = m.alloc<double>(MK);
    p->d_yBt = m.alloc<double>(M);
    p->facq_off.clear();
    i64 nq = 0;
    auto add_q = [&](const FKey& k, i64 size) {
      if (p->facq_off.count(k)) return;
      p->facq_off[k] = nq;
      nq += size;
    };
    for (int a = 0; a < p->nterms; ++a)
      for (int i = 0; i < p->d; ++i) add_q(FKey(i, 0, p->alpha[a][i], 1, 0), (i64)p->nc[i] * p->sets[0].n[i]);
    for (int i = 0; i < p->d; ++i) add_q(FKey(i, 1, 0, 2, 0), (i64)p->sets[0].n[i] * p->npred[i]);
    for (int s = 1; s < p->nsets; ++s)
      for (int i = 0; i < p->d; ++i) add_q(FKey(i, 1, s, 1, 0), (i64)p->sets[s].n[i] * p->sets[0].n[i]);
    p->nfacq = std::max<i64>(nq, 1);
    p->d_facq = m.alloc<double>(p->nfacq);
    p->f_facq = m.alloc<float>(p->nfacq);
    if (MR > 0) {
      p->d_Et = m.alloc<double>(MR * MK);
      p->d_EtT = m.alloc<double>(MR * MK);
      i64 maxms = 0;
      for (int s = 1; s < p->nsets; ++s) maxms = std::max<i64>(maxms, p->sets[s].size);
      p->d_Tsc = m.alloc<double>(MR * maxms);
      p->d_R = m.alloc<double>(MR * MK);
      p->d_Sc = m.alloc<double>(MR * MR);
      p->d_LS = m.alloc<double>(MR * MR);
      p->d_LSinv = m.alloc<double>(MR * MR);
      p->d_LSinvT = m.alloc<double>(MR * MR);
      p->d_sscr = m.alloc<double>(MR * MR / 4 + 64 * MR + 64);
      p->d_tR = m.alloc<double>(MR);
      p->d_uR = m.alloc<double>(MR);
      p->f_Et = m.alloc<float>(MR * MK);
      p->f_EtT = m.alloc<float>(MR * MK);
      p->f_LSinv = m.alloc<float>(MR * MR);
      p->f_LSinvT = m.alloc<float>(MR * MR);
      p->f_tR = m.alloc<float>(MR);
      p->f_uR = m.alloc<float>(MR);
    }
  }
  if (M > 0) {
    if (!p->sicbc) {
      p->d_A = m.alloc<double>(M * M);
      p->d_L = m.alloc<double>(M * M);
      p->d_Linv = m.alloc<double>(M * M);
      p->d_LinvT = m.alloc<double>(M * M);
      p->d_cscr = m.alloc<double>(M * M / 4 + 64 * M + 64);
    }
    if (p->oz_on) {  // window exponents of the digit-product dense GEMMs (rows x windows, per operand)
      const i64 big = std::max<i64>(M, p->MR);
      p->ozg_cap = big * ((big + OZ_KMAX - 1) / OZ_KMAX);
      p->d_ozgexp = m.alloc<int>(2 * p->ozg_cap);
    }
    p->d_yB = m.alloc<double>(M);
    p->d_g = m.alloc<double>(M);
    p->d_t = m.alloc<double>(M);
    p->d_w = m.alloc<double>(M);
    p->d_g2 = m.alloc<double>(M);
    p->d_win = m.alloc<double>(M);
    p->d_wout = m.alloc<double>(M);
    std::vector<double> y;
    for (int s = 0; s < p->nsets; ++s) y.insert(y.end(), p->sets[s].values.begin(), p->sets[s].values.end());
    GPFVM_CUDA(cudaMemcpy(p->d_yB, y.data(), M * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (!p->rhs.empty()) {
    p->d_rhs = m.alloc<double>(N);
    GPFVM_CUDA(cudaMemcpy(p->d_rhs, p->rhs.data(), N * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (p->nfield > 0) {
    p->d_field = m.alloc<double>((i64)p->nfield * N);
    p->f_field = m.alloc<float>((i64)p->nfield * N);
    GPFVM_CUDA(cudaMemcpy(p->d_field, p->fields.data(), sizeof(double) * p->nfield * N, cudaMemcpyHostToDevice));
    std::vector<float> f32(p->fields.begin(), p->fields.end());
    GPFVM_CUDA(cudaMemcpy(p->f_field, f32.data(), sizeof(float) * p->nfield * N, cudaMemcpyHostToDevice));
  }
  p->d_b = m.alloc<double>(N);
  p->d_x = m.alloc<double>(N);
  p->d_r = m.alloc<double>(N);
  p->d_p = m.alloc<double>(N);
  p->d_q = m.alloc<double>(N);
  p->d_vin = m.alloc<double>(N);
  p->d_vout = m.alloc<double>(N);
  p->d_u = m.alloc<double>(P);
  p->d_tbeta = m.alloc<double>(P);
  p->d_down = m.alloc<double>(P);
  p->d_mean = m.alloc<double>(P);
  p->d_var = m.alloc<double>(P);
  p->d_vB = m.alloc<double>(P);
  const int cap = p->cap;
  // the direction stores S, Q (FP64 and FP32) are allocated on first use, sized by need
  p->d_eta = m.alloc<double>(cap);
  p->d_part2 = m.alloc<double>((i64)cap * reorth_chunks(N));
  p->d_coef = m.alloc<double>(cap);
  if (M > 0) {
    // row chunks of the Cholesky-stage variance: rows x P FP64 (32 MB) stays in L2
    i64 R = std::max<i64>(1, std::min<i64>(M, ((i64)1 << 22) / std::max<i64>(P, 1)));
    p->vb_rows = (int)R;
    i64 maxms = 0;
    for (int s = 0; s < p->nsets; ++s) maxms = std::max(maxms, p->sets[s].size);
    p->d_vbchunk = m.alloc<double>(R * maxms);
    p->d_vbY = m.alloc<double>(R * P);
  }
  // mixed-precision buffers
  p->nfac = std::max<i64>(nfac, 1);
  p->f_fac = m.alloc<float>(p->nfac);
  if (M > 0) {
    if (!p->sicbc) {
      p->f_Linv = m.alloc<float>(M * M);
      p->f_LinvT = m.alloc<float>(M * M);
    }
    p->f_g = m.alloc<float>(M);
    p->f_t = m.alloc<float>(M);
    p->f_w = m.alloc<float>(M);
  }
  p->f_p = m.alloc<float>(N);
  p->f_q = m.alloc<float>(N);
  p->f_r = m.alloc<float>(N);
  p->f_d = m.alloc<float>(N);
  p->f_vin = m.alloc<float>(N);
  p->f_vout = m.alloc<float>(N);
  p->f_u = m.alloc<float>(P);
  p->d_eta32 = m.alloc<double>(cap);
  p->d_st = m.alloc<CGState>(1);
  p->d_st32 = m.alloc<CGState>(1);
  p->d_mctl = m.alloc<MixedCtl>(1);
  p->d_psync = m.alloc<unsigned int>(2);
  GPFVM_CUDA(cudaMemset(p->d_psync, 0, 2 * sizeof(unsigned int)));
  GPFVM_CUDA(cudaMemset(p->d_st, 0, sizeof(CGState)));
  GPFVM_CUDA(cudaMemset(p->d_st32, 0, sizeof(CGState)));
  GPFVM_CUDA(cudaMallocHost(&p->h_st, sizeof(CGState)));
  GPFVM_CUDA(cudaMallocHost(&p->h_st32, sizeof(CGState)));
  GPFVM_CUDA(cudaMallocHost(&p->h_mctl, sizeof(MixedCtl)));
  std::memset(p->h_mctl, 0, sizeof(MixedCtl));
  GPFVM_CUDA(cudaMemset(p->d_mctl, 0, sizeof(MixedCtl)));
  std::memset(p->h_st, 0, sizeof(CGState));
  std::memset(p->h_st32, 0, sizeof(CGState));
  GPFVM_CUDA(cudaMemset(p->d_down, 0, P * sizeof(double)));
  // plans: count scratch, allocate, build for real
  Builder B0{p};
  B0.scr.base = nullptr;
  B0.scr.cap = (i64)1 << 62;
  build_plans(p, B0);
  build_plans32(p, B0);
  p->f_tcsplit = m.alloc<float>(std::max<i64>(p->tc_split_total, 64));
  p->f_tcY = m.alloc<float>(std::max<i64>((i64)p->tc_nu * N, 64));
  p->f_tcZ = m.alloc<float>(std::max<i64>((i64)p->tc_nw * N, 64));
  p->f_tcpart = m.alloc<float>(std::max<i64>(p->tc_part_total, 64));
  p->d_tcops = m.alloc<TcOp>(std::max<i64>(p->tc_ops_total, 1));
  p->tc_jobs.clear();
  if (!p->ozx_ops.empty()) {
    p->ozx_ops_cap = (i64)p->ozx_ops.size();
    p->d_ozxops = m.alloc<OzOp>(p->ozx_ops_cap);
    p->d_ozximg = m.alloc<unsigned char>(std::max<i64>(p->ozx_img_n, 256));
    p->d_ozxfexp = m.alloc<int>(std::max<i64>(p->ozx_fexp_n, 64));
  }
  if (p->oz_ok) {
    p->d_ozops = m.alloc<OzOp>(std::max<i64>(p->oz_ops_total, 1));
    p->d_ozimg = m.alloc<unsigned char>(std::max<i64>(p->oz_img_total, 256));
    p->d_ozfexp = m.alloc<int>(std::max<i64>(p->oz_fexp_total, 64));
    p->d_ozexp = m.alloc<int>(std::max<i64>(p->oz_exp_total, 64));
    p->d_ozY = m.alloc<double>(std::max<i64>((i64)p->oz_nu * N, 64));
    p->d_ozZ = m.alloc<double>(std::max<i64>((i64)p->oz_nw * N, 64));
  }
  p->scratch_cap = std::max<i64>(B0.peak, 64);
  p->d_scratch = m.alloc<double>(p->scratch_cap);
  Builder B{p};
  B.scr.base = p->d_scratch;
  B.scr.cap = p->scratch_cap;
  build_plans(p, B);
  build_plans32(p, B);
  finalize_plans(p);
}

// Rebuilds every plan under the given mode-product policies (same scratch:
// intermediates do not depend on tile shapes); captured loops are dropped.
void rebuild_plans(gpfvm_problem* p, int tile, int tc_group) {
  set_tile_policy(tile);
  g_tc_group_policy = tc_group;
  try {
    p->tc_jobs.clear();
    Builder B{p};
    B.scr.base = p->d_scratch;
    B.scr.cap = p->scratch_cap;
    build_plans(p, B);
    build_plans32(p, B);
    finalize_plans(p);
  } catch (...) {
    set_tile_policy(-1);
    g_tc_group_policy = 0;
    throw;
  }
  set_tile_policy(-1);
  g_tc_group_policy = 0;
  p->tuned_tile = tile;
  p->tuned_tc = tc_group;
  if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; p->graph_key = -1; }
  if (p->graph32) { cudaGraphExecDestroy(p->graph32); p->graph32 = nullptr; p->graph32_key = -1; }
}

void copy_header_to_host(gpfvm_problem* p, cudaStream_t st) {
  GPFVM_CUDA(cudaMemcpyAsync(p->h_st, p->d_st, offsetof(CGState, part), cudaMemcpyDeviceToHost, st));
}

int run_assemble(gpfvm_problem* p, cudaStream_t st) {
  GPFVM_CUDA(cudaMemsetAsync(p->d_st, 0, offsetof(CGState, part), st));
  p->p_setup.run(st);
  if (p->M > 0) {
    p->p_chol.run(st);
    copy_header_to_host(p, st);
    GPFVM_CUDA(cudaStreamSynchronize(st));
    if (p->h_st->pad[0] & DEV_NOT_SPD) return GPFVM_ERR_NOT_SPD;
    if (p->h_st->pad[0] & DEV_TIMEOUT) return GPFVM_ERR_TIMEOUT;
  }
  p->p_rhs.run(st);
  if (p->oz_ok && p->d_ozimg)
    for (const auto& j : p->oz_jobs)
      oz_split_factor(p->d_fac + j.fac_off, j.n, 1, j.n, j.n, j.alpha, p->d_ozimg + j.img_off, p->d_ozfexp + j.fexp_off,
                      st);
  if (p->d_ozximg)
    for (const auto& j : p->ozx_jobs)
      oz_split_factor(j.F, j.rs, j.cs, j.N, j.K, j.alpha, p->d_ozximg + j.img_off, p->d_ozxfexp + j.fexp_off, st);
  convert_d2f(p->d_fac, p->f_fac, p->nfac, st);
  for (auto& j : p->tc_jobs) {
    const i64 n = std::get<2>(j), off = std::get<3>(j);
    tc_split(p->f_fac + std::get<0>(j), n, std::get<1>(j), p->f_tcsplit + off, p->f_tcsplit + off + (n + 63) / 64 * 64,
             st, std::get<4>(j));
  }
  if (p->M > 0 && !p->sicbc) {
    convert_d2f(p->d_Linv, p->f_Linv, p->M * p->M, st);
    convert_d2f(p->d_LinvT, p->f_LinvT, p->M * p->M, st);
  }
  GPFVM_CUDA(cudaStreamSynchronize(st));
  p->assembled = true;
  p->solved = false;
  p->vB_ready = false;
  return GPFVM_OK;
}

// Direction stores for the reorthogonalisation, allocated on first use.
void ensure_store64(gpfvm_problem* p, int need) {
  need = std::min(need, p->cap);
  if (p->cap64 >= need) return;
  const i64 ld = store_ld(p->N);
  if (p->d_S) { cudaFree(p->d_S); cudaFree(p->d_Q); p->mem.bytes -= 16LL * p->cap64 * ld; }
  p->d_S = p->d_Q = nullptr;
  p->cap64 = 0;
  if (cudaMalloc(&p->d_S, sizeof(double) * (size_t)need * ld) != cudaSuccess ||
      cudaMalloc(&p->d_Q, sizeof(double) * (size_t)need * ld) != cudaSuccess) {
    cudaGetLastError();
    if (p->d_S) cudaFree(p->d_S);
    p->d_S = p->d_Q = nullptr;
    throw CudaError{cudaErrorMemoryAllocation, "direction store"};
  }
  p->cap64 = need;
  p->mem.bytes += 16LL * need * ld;
  if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; p->graph_key = -1; }
}
// Grows the FP64 stores to `need` directions keeping the first `keep` rows.
void grow_store64(gpfvm_problem* p, int need, int keep) {
  need = std::min(need, p->cap);
  if (p->cap64 >= need) return;
  const i64 ld = store_ld(p->N);
  double *S = nullptr, *Q = nullptr;
  if (cudaMalloc(&S, sizeof(double) * (size_t)need * ld) != cudaSuccess ||
      cudaMalloc(&Q, sizeof(double) * (size_t)need * ld) != cudaSuccess) {
    cudaGetLastError();
    if (S) cudaFree(S);
    throw CudaError{cudaErrorMemoryAllocation, "direction store"};
  }
  if (keep > 0 && p->d_S) {
    GPFVM_CUDA(cudaMemcpy(S, p->d_S, sizeof(double) * (size_t)keep * ld, cudaMemcpyDeviceToDevice));
    GPFVM_CUDA(cudaMemcpy(Q, p->d_Q, sizeof(double) * (size_t)keep * ld, cudaMemcpyDeviceToDevice));
  }
  if (p->d_S) { cudaFree(p->d_S); cudaFree(p->d_Q); p->mem.bytes -= 16LL * p->cap64 * ld; }
  p->d_S = S;
  p->d_Q = Q;
  p->cap64 = need;
  p->mem.bytes += 16LL * need * ld;
  if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; p->graph_key = -1; }
}
// Grows the FP32 stores to at least `need` directions (geometric steps, at
// most p->cap) keeping the first `keep` rows; the captured inner loop graph
// addresses the stores, so it is rebuilt after a move.
void grow_store32(gpfvm_problem* p, int need, int keep) {
  need = std::min(need, p->cap);
  if (p->cap32 >= need) return;
  const int want = std::min(p->cap, std::max(need, p->cap32 + p->cap32 / 2));
  const i64 ld = store_ld(p->N);
  float *S = nullptr, *Q = nullptr;
  if (cudaMalloc(&S, sizeof(float) * (size_t)want * ld) != cudaSuccess ||
      cudaMalloc(&Q, sizeof(float) * (size_t)want * ld) != cudaSuccess) {
    cudaGetLastError();
    if (S) cudaFree(S);
    throw CudaError{cudaErrorMemoryAllocation, "direction store"};
  }
  if (keep > 0 && p->f_S) {
    GPFVM_CUDA(cudaMemcpy(S, p->f_S, sizeof(float) * (size_t)keep * ld, cudaMemcpyDeviceToDevice));
    GPFVM_CUDA(cudaMemcpy(Q, p->f_Q, sizeof(float) * (size_t)keep * ld, cudaMemcpyDeviceToDevice));
  }
  if (p->f_S) { cudaFree(p->f_S); cudaFree(p->f_Q); p->mem.bytes -= 8LL * p->cap32 * ld; }
  p->f_S = S;
  p->f_Q = Q;
  p->cap32 = want;
  p->mem.bytes += 8LL * want * ld;
  if (p->graph32) { cudaGraphExecDestroy(p->graph32); p->graph32 = nullptr; p->graph32_key = -1; }
}
void ensure_store32(gpfvm_problem* p, int need) {
  need = std::min(need, p->cap);
  if (p->cap32 >= need) return;
  const i64 ld = store_ld(p->N);
  if (p->f_S) { cudaFree(p->f_S); cudaFree(p->f_Q); p->mem.bytes -= 8LL * p->cap32 * ld; }
  p->f_S = p->f_Q = nullptr;
  p->cap32 = 0;
  if (cudaMalloc(&p->f_S, sizeof(float) * (size_t)need * ld) != cudaSuccess ||
      cudaMalloc(&p->f_Q, sizeof(float) * (size_t)need * ld) != cudaSuccess) {
    cudaGetLastError();
    if (p->f_S) cudaFree(p->f_S);
    p->f_S = p->f_Q = nullptr;
    throw CudaError{cudaErrorMemoryAllocation, "direction store"};
  }
  p->cap32 = need;
  p->mem.bytes += 8LL * need * ld;
  if (p->graph32) { cudaGraphExecDestroy(p->graph32); p->graph32 = nullptr; p->graph32_key = -1; }
}

void cg_iteration(gpfvm_problem* p, bool reorth, bool want_var, cudaStream_t st) {
  const i64 N = p->N;
  (want_var ? p->p_mvv_cg : p->p_mv_cg).run(st);
  cg_dot_eta(p->d_p, p->d_q, N, p->d_st, p->d_eta, st);
  if (want_var) cg_downdate(p->d_u, p->d_down, p->P, p->d_st, st);
  cg_update(p->d_x, p->d_r, p->d_p, p->d_q, N, p->d_st, reorth ? p->d_S : nullptr, reorth ? p->d_Q : nullptr, st);
  cg_pupdate(p->d_r, p->d_p, N, p->d_st, st);
  if (reorth) cg_reorth(p->d_S, p->d_Q, p->d_p, N, p->cap64, p->d_st, p->d_part2, p->d_coef, p->d_eta, st);
}

// The FP64 G^ of residuals and refinement: with the digit-product G_PP when the
// CG plans use it (the same operator as the captured refinement's p_res).
Plan& fp64_ghat(gpfvm_problem* p) { return (p->oz_ok && p->oz_on && p->d_ozops) ? p->p_op[5] : p->p_op[1]; }

double true_rel_residual(gpfvm_problem* p, const double* x, cudaStream_t st) {
  GPFVM_CUDA(cudaMemcpyAsync(p->d_vin, x, sizeof(double) * p->N, cudaMemcpyDeviceToDevice, st));
  fp64_ghat(p).run(st);
  axpby(p->d_b, p->d_vout, p->d_vout, 1.0, -1.0, p->N, st);
  norm2(p->d_vout, p->N, &p->d_st->aux[0], p->d_st, st);
  copy_header_to_host(p, st);
  GPFVM_CUDA(cudaStreamSynchronize(st));
  const double b2 = p->h_st->bnorm2;
  return b2 > 0 ? std::sqrt(p->h_st->aux[0] / b2) : 0.0;
}

// A graph whose only node is a WHILE loop over one captured CG iteration:
// the iteration kernels plus loop_ctl, which ends the loop once the device
// state reports done (or after max_iter + 2 passes).  One launch runs a whole
// CG run with no host round trips.  *body_kernels receives the kernels of one
// pass (the control kernel included).
// CG iterations per pass of a device-side loop (GPFVM_LOOP_UNROLL, 1 to 8; default 2)
int loop_unroll() {
  static const int u = [] {
    const char* e = getenv("GPFVM_LOOP_UNROLL");
    const int v = e ? std::atoi(e) : 2;
    return std::min(std::max(v, 1), 8);
  }();
  return u;
}

cudaGraphExec_t make_loop_graph(CGState* st_dev, cudaStream_t st, const std::function<void()>& body,
                                long long* body_kernels, bool host_loop) {
  if (host_loop) {  // one pass per launch; the host repeats it
    cudaGraph_t g = nullptr;
    const long long before = g_launches.load();
    GPFVM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      body();
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(st, &dummy);
      cudaGetLastError();
      throw;
    }
    GPFVM_CUDA(cudaStreamEndCapture(st, &g));
    *body_kernels = g_launches.load() - before;
    g_launches.fetch_sub(*body_kernels);
    cudaGraphExec_t ex = nullptr;
    GPFVM_CUDA(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    return ex;
  }
  cudaGraph_t g = nullptr;
  GPFVM_CUDA(cudaGraphCreate(&g, 0));
  try {
    cudaGraphConditionalHandle h;
    GPFVM_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    GPFVM_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    const long long before = g_launches.load();
    GPFVM_CUDA(cudaStreamBeginCaptureToGraph(st, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      // several iterations per pass (every kernel of an iteration does nothing
      // once the run is done), one condition update per pass
      const int unroll = loop_unroll();
      for (int u = 0; u < unroll; ++u) body();
      loop_ctl(st_dev, h, st);
    } catch (...) {
      cudaGraph_t dummy;
      cudaStreamEndCapture(st, &dummy);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t captured;
    GPFVM_CUDA(cudaStreamEndCapture(st, &captured));
    *body_kernels = g_launches.load() - before;
    g_launches.fetch_sub(*body_kernels);  // captured, not launched
    cudaGraphExec_t ex = nullptr;
    GPFVM_CUDA(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    return ex;
  } catch (...) {
    cudaGraphDestroy(g);
    throw;
  }
}

int mixed_solve(gpfvm_problem* p, const gpfvm_solve_opts* o, gpfvm_solve_info* info, cudaStream_t st);

struct SolveRun {
  gpfvm_solve_opts o{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int launched = 0;
  bool active = false;
};
std::map<const gpfvm_problem*, SolveRun>& runs() {
  static std::map<const gpfvm_problem*, SolveRun> m;
  return m;
}

// Multigrid warm start (appendix "Multigrid preconditioners"): the coarse FVM
// observations W^T y (a coarse volume is the union of f^d fine ones) are
// conditioned on exactly before CG.  With A_c = W^T G^ W = L_c L_c^T the
// columns of W L_c^-T are G^-orthonormal actions; they are written as the
// first n_c stored directions (eta = 1, their images G^ W L_c^-T beside them)
// with their downdate, so that the Galerkin projection at the start of the CG
// run is the exact coarse solve and every CG direction is made conjugate to
// them by the usual reorthogonalisation.  Two passes of n_c operator
// applications (A_c, then the directions); returns n_c or an error.
int multigrid_setup(gpfvm_problem* p, const gpfvm_solve_opts* o, cudaStream_t st) {
  const int f = o->coarse;
  CoarseGeom g{};
  g.d = p->d;
  g.f = f;
  i64 nc = 1;
  for (int i = 0; i < p->d; ++i) {
    if (p->nc[i] % f) return GPFVM_ERR_INVALID_ARG;
    g.n[i] = p->nc[i];
    g.nc[i] = p->nc[i] / f;
    nc *= g.nc[i];
  }
  if (nc > 4096 || nc + o->max_iter > p->cap64) return GPFVM_ERR_INVALID_ARG;
  const int n = (int)nc;
  const i64 N = p->N, ld = store_ld(N);
  double *Ac = nullptr, *Lc = nullptr, *Li = nullptr, *scr = nullptr;
  auto release = [&] {
    if (Ac) cudaFree(Ac);
    if (Lc) cudaFree(Lc);
    if (Li) cudaFree(Li);
    if (scr) cudaFree(scr);
  };
  try {
    GPFVM_CUDA(cudaMalloc(&Ac, sizeof(double) * nc * nc));
    GPFVM_CUDA(cudaMalloc(&Lc, sizeof(double) * nc * nc));
    GPFVM_CUDA(cudaMalloc(&Li, sizeof(double) * nc * nc));
    GPFVM_CUDA(cudaMalloc(&scr, sizeof(double) * (nc * nc / 4 + 64 * nc + 64)));
    GPFVM_CUDA(cudaMemsetAsync(&p->d_st->done, 0, sizeof(int), st));  // the operator plans run
    // pass 1: column c of A_c = W^T G^ (W e_c)
    for (int c = 0; c < n; ++c) {
      coarse_gather(p->d_p, N, g, nullptr, c, st);
      p->p_mv_cg.run(st);
      coarse_restrict(p->d_q, g, Ac + c, nc, st);
    }
    GPFVM_CUDA(cudaMemsetAsync(Lc, 0, sizeof(double) * nc * nc, st));
    GPFVM_CUDA(cudaMemsetAsync(Li, 0, sizeof(double) * nc * nc, st));
    GPFVM_CUDA(cudaMemsetAsync(&p->d_st->pad[0], 0, sizeof(int), st));
    {
      Plan ch;
      plan_chol_inverse(ch, Ac, Lc, Li, n, nc, scr, &p->d_st->pad[0]);
      ch.finalize();
      ch.fan = &p->fan;
      ch.run(st);
    }
    copy_header_to_host(p, st);
    GPFVM_CUDA(cudaStreamSynchronize(st));
    if (p->h_st->pad[0] & DEV_NOT_SPD) {
      release();
      return GPFVM_ERR_NOT_SPD;
    }
    // pass 2: s_c = W L_c^-T e_c (row c of L_c^-1 spread over the fine cells),
    // its image and its downdate (eta = 1)
    const bool want_var = o->want_var != 0;
    for (int c = 0; c < n; ++c) {
      coarse_gather(p->d_S + (i64)c * ld, N, g, Li + (i64)c * nc, -1, st);
      GPFVM_CUDA(cudaMemcpyAsync(p->d_p, p->d_S + (i64)c * ld, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      (want_var ? p->p_mvv_cg : p->p_mv_cg).run(st);
      GPFVM_CUDA(cudaMemcpyAsync(p->d_Q + (i64)c * ld, p->d_q, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      if (want_var) add_squares(p->d_down, p->d_u, p->P, st);
    }
    std::vector<double> ones((size_t)n, 1.0);
    GPFVM_CUDA(cudaMemcpyAsync(p->d_eta, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    GPFVM_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    release();
    throw;
  }
  release();
  return n;
}

int solve_begin(gpfvm_problem* p, const gpfvm_solve_opts* o, cudaStream_t st) {
  if (!p->assembled) return GPFVM_ERR_STATE;
  if (!o || o->max_iter < 1 || !(o->rtol >= 0)) return GPFVM_ERR_INVALID_ARG;
  if (o->precision != GPFVM_FP64) return GPFVM_ERR_INVALID_ARG;
  const bool reorth = o->reorth != 0, want_var = o->want_var != 0;
  if (reorth && o->max_iter > p->cap) return GPFVM_ERR_INVALID_ARG;
  SolveRun& R = runs()[p];
  R.o = *o;
  R.launched = 0;
  R.active = true;
  if (!R.e0) {
    GPFVM_CUDA(cudaEventCreate(&R.e0));
    GPFVM_CUDA(cudaEventCreate(&R.e1));
  }
  GPFVM_CUDA(cudaEventRecord(R.e0, st));
  // multigrid warm start: coarse actions stored ahead of the CG directions
  i64 ncoarse = 0;
  if (o->coarse > 1) {
    if (!reorth) return GPFVM_ERR_INVALID_ARG;
    ncoarse = 1;
    for (int i = 0; i < p->d; ++i) ncoarse *= p->nc[i] / o->coarse;
    if (ncoarse + o->max_iter > p->cap) return GPFVM_ERR_INVALID_ARG;
  }
  if (reorth) ensure_store64(p, (int)(o->max_iter + ncoarse));
  if (want_var) GPFVM_CUDA(cudaMemsetAsync(p->d_down, 0, sizeof(double) * p->P, st));
  int kb = 0;
  if (o->coarse > 1) {
    kb = multigrid_setup(p, o, st);
    if (kb < 0) return kb;
  }
  p->h_st->rtol2 = o->rtol * o->rtol;
  p->h_st->max_iter = o->max_iter + kb;  // the CG budget excludes the coarse actions
  p->h_st->cap = reorth ? p->cap64 : 0;
  p->h_st->kbase = kb;
  GPFVM_CUDA(cudaMemcpyAsync(&p->d_st->rtol2, &p->h_st->rtol2, sizeof(double), cudaMemcpyHostToDevice, st));
  GPFVM_CUDA(cudaMemcpyAsync(&p->d_st->max_iter, &p->h_st->max_iter, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
  GPFVM_CUDA(cudaMemcpyAsync(&p->d_st->kbase, &p->h_st->kbase, sizeof(int), cudaMemcpyHostToDevice, st));
  cg_init(p->d_b, p->d_x, p->d_r, p->d_p, p->N, p->d_st, st);
  if (kb > 0)  // x = the exact coarse solve, r and p projected
    cg_project<double>(p->d_S, p->d_Q, p->d_r, p->d_x, p->d_p, p->N, p->cap64, p->d_st, p->d_part2, p->d_coef,
                       p->d_eta, st);
  const int key = (reorth ? 1 : 0) + (want_var ? 2 : 0);
  if (!p->graph || p->graph_key != key) {
    if (p->graph) cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
    p->graph = make_loop_graph(p->d_st, st, [&] { cg_iteration(p, reorth, want_var, st); }, &p->graph_kernels,
                               p->host_loop);
    p->graph_key = key;
  }
  return GPFVM_OK;
}

// Host-driven form of a CG run (GPFVM_HOST_LOOP): replays the one-pass graph
// until the device state reports done; leaves the header copied to hst.
void host_loop_run(cudaGraphExec_t g, long long kernels, CGState* dst, CGState* hst, cudaStream_t st) {
  const int lim = std::max(dst ? hst->max_iter : 0, 0) + 2;
  for (int pass = 0; pass < lim; ++pass) {
    GPFVM_CUDA(cudaGraphLaunch(g, st));
    count_launch(kernels);
    GPFVM_CUDA(cudaMemcpyAsync(hst, dst, offsetof(CGState, part), cudaMemcpyDeviceToHost, st));
    GPFVM_CUDA(cudaStreamSynchronize(st));
    if (hst->done) break;
  }
  hst->loops = 0;  // launches already counted
}

// Enqueues the device-side CG loop (all iterations) and a copy of the scalar header.
void solve_launch(gpfvm_problem* p, int, cudaStream_t st) {
  SolveRun& R = runs()[p];
  if (R.launched > 0) return;
  if (p->host_loop) {
    host_loop_run(p->graph, p->graph_kernels, p->d_st, p->h_st, st);
    R.launched = R.o.max_iter;
    return;
  }
  GPFVM_CUDA(cudaGraphLaunch(p->graph, st));
  R.launched = R.o.max_iter;
  copy_header_to_host(p, st);
}

// True once the launched loop has ended; needs the stream to be synchronised.
bool solve_finished(gpfvm_problem* p) {
  SolveRun& R = runs()[p];
  return R.launched > 0;
}

int solve_end(gpfvm_problem* p, gpfvm_solve_info* info, cudaStream_t st) {
  SolveRun& R = runs()[p];
  GPFVM_CUDA(cudaEventRecord(R.e1, st));
  GPFVM_CUDA(cudaEventSynchronize(R.e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, R.e0, R.e1);
  R.active = false;
  const CGState& h = *p->h_st;
  count_launch((long long)h.loops * p->graph_kernels);
  int status = GPFVM_NOT_CONVERGED;
  if (h.status & DEV_TIMEOUT) status = GPFVM_ERR_TIMEOUT;
  else if (h.status & DEV_BREAKDOWN) status = GPFVM_ERR_BREAKDOWN;
  else if (h.converged) status = GPFVM_OK;
  gpfvm_solve_info I = p->last;
  I.iterations = h.k - h.kbase;  // CG iterations (coarse actions of a multigrid start excluded)
  I.status = status;
  I.rel_residual = h.bnorm2 > 0 ? std::sqrt(h.rr / h.bnorm2) : 0.0;
  I.t_solve_ms = ms;
  I.true_rel_residual = true_rel_residual(p, p->d_x, st);
  p->last = I;
  if (info) *info = I;
  p->solved = status >= 0;
  p->want_var_last = R.o.want_var != 0;
  p->last_store = R.o.reorth ? 1 : 0;
  p->last_kstore = R.o.reorth ? std::min(h.k, p->cap64) : 0;
  return status;
}

int run_solve(gpfvm_problem* p, const gpfvm_solve_opts* o, gpfvm_solve_info* info, cudaStream_t st) {
  if (p->multi && o && (o->precision != GPFVM_FP64 || o->coarse > 1)) return GPFVM_ERR_INVALID_ARG;
  if (o && o->precision != GPFVM_FP64) return mixed_solve(p, o, info, st);
  const int b = solve_begin(p, o, st);
  if (b != GPFVM_OK) return b;
  solve_launch(p, 0, st);
  GPFVM_CUDA(cudaStreamSynchronize(st));
  return solve_end(p, info, st);
}

int run_query(gpfvm_problem* p, double* mean, double* var, cudaStream_t st) {
  if (!p->solved) return GPFVM_ERR_STATE;
  if (var && !p->want_var_last) return GPFVM_ERR_STATE;
  p->p_mean.run(st);
  if (mean) GPFVM_CUDA(cudaMemcpyAsync(mean, p->d_mean, sizeof(double) * p->P, cudaMemcpyDeviceToDevice, st));
  if (var) {
    if (p->M > 0 && !p->vB_ready) {
      p->p_vB.run(st);
      p->vB_ready = true;
    }
    var_final(p->M > 0 ? p->d_vB : nullptr, p->d_down, p->d_var, p->s2, p->P, st);
    GPFVM_CUDA(cudaMemcpyAsync(var, p->d_var, sizeof(double) * p->P, cudaMemcpyDeviceToDevice, st));
  }
  return GPFVM_OK;
}

// One inner CG iteration of the mixed solver (FP32 operator and vectors, FP64 scalars).
void cg_iteration32(gpfvm_problem* p, bool want_var, bool reorth, cudaStream_t st) {
  const i64 N = p->N;
  if (p->tc_mode >= 0) (want_var ? p->p_mvv32tc[p->tc_mode] : p->p_mv32tc[p->tc_mode]).run(st);
  else (want_var ? p->p_mvv32 : p->p_mv32).run(st);
  cg_dot_eta<float>(p->f_p, p->f_q, N, p->d_st32, p->d_eta32, st);
  if (want_var) cg_downdate<float>(p->f_u, p->d_down, p->P, p->d_st32, st);
  cg_update<float>(p->f_d, p->f_r, p->f_p, p->f_q, N, p->d_st32, reorth ? p->f_S : nullptr,
                   reorth ? p->f_Q : nullptr, st);
  cg_pupdate<float>(p->f_r, p->f_p, N, p->d_st32, st);
  if (reorth)
    cg_reorth<float>(p->f_S, p->f_Q, p->f_p, N, p->cap32, p->d_st32, p->d_part2, p->d_coef, p->d_eta32, st);
}

// Mixed precision (Sec. 4.1 CG with an inexact operator, FP64 residual replacement):
//   r = b - G^ x            FP64 operator, FP64 vectors (x = 0: r = b)
//   inner CG on G^_32 d ~= r/|r|   FP32 (or tensor-core) operator, FP32 vectors, FP64 scalars
//   x += |r| d              (the unit right-hand side keeps FP32 in range for any data scale)
// until ||r|| / ||b|| <= rtol or max_iter inner iterations in total.
// With reorth the runs form ONE conjugate-direction sequence: every run keeps
// the stored directions of all earlier runs, starts with the Galerkin
// projection of its residual onto them (d = S c, r -= Q c, c_j = s_j.r/eta_j;
// zero in exact arithmetic) and makes each new direction G^-conjugate to all
// stored ones.  With an exact operator this is the FP64 CG recurrence itself
// (the restart direction r - (q_last.r/eta) s_last is the continued CG
// direction), so after k iterations the actions span the same Krylov space;
// the IterGP downdate sum_j u_j^2/eta_j runs over the directions of all runs.
// Each run's tolerance is max(inner_rtol, rtol |b|/|r|), so the last run stops
// where the continued recurrence reaches rtol, as the FP64 path does.
// Without reorth the runs are independent refinement steps and the downdate
// uses the first run's directions only (conjugate within that run).
// The solve is a resumable state machine so that batched and served execution
// can interleave many problems:
//   0 residual wanted -> 1 residual enqueued -> 2 inner CG running -> 0 ... -> 3 done
struct MixedRun {
  gpfvm_solve_opts o{};
  int mstate = 3, outer = 0, total = 0, launched = 0, lim = 0, status = 0;
  int kstore = 0;  // directions stored by the runs so far (conjugate continuation)
  int idle = 0;    // consecutive runs that took no iteration
  double tscale = 1.0;  // fraction of rtol the next run aims at
  double rel = 1.0, itol = 1e-2, rel_prev = 1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};
std::map<const gpfvm_problem*, MixedRun>& mruns() {
  static std::map<const gpfvm_problem*, MixedRun> m;
  return m;
}

int mixed_begin(gpfvm_problem* p, const gpfvm_solve_opts* o, cudaStream_t st) {
  if (!p->assembled) return GPFVM_ERR_STATE;
  if (!o || o->max_iter < 1 || !(o->rtol >= 0)) return GPFVM_ERR_INVALID_ARG;
  if (o->precision < GPFVM_MIXED_FP32 || o->precision > GPFVM_MIXED_BF16) return GPFVM_ERR_INVALID_ARG;
  if (o->coarse > 1) return GPFVM_ERR_INVALID_ARG;  // the multigrid start is an FP64-path option
  MixedRun& R = mruns()[p];
  R.o = *o;
  R.itol = o->inner_rtol > 0 ? o->inner_rtol : 1e-2;
  if (o->reorth < 0 || o->reorth > 2 || (o->reorth == 1 && o->max_iter > p->cap)) return GPFVM_ERR_INVALID_ARG;
  const int icap = std::min(p->cap, o->inner_max_iter > 0 ? o->inner_max_iter : p->cap);
  const int want_tc = o->precision == GPFVM_MIXED_TF32X3 ? TC_TF32X3
                      : o->precision == GPFVM_MIXED_BF16X3 ? TC_BF16X3
                      : o->precision == GPFVM_MIXED_BF16  ? TC_BF16
                                                          : -1;
  if (want_tc >= 0 && !p->tc_ok) return GPFVM_ERR_INVALID_ARG;
  // one run's worth unless the runs continue one direction set (reorth 1),
  // whose stores grow run by run (every run's directions: up to max_iter)
  if (o->reorth != 1) ensure_store32(p, icap);
  if (want_tc != p->tc_mode) {  // the captured inner iteration depends on the operator
    p->tc_mode = want_tc;
    if (p->graph32) cudaGraphExecDestroy(p->graph32);
    p->graph32 = nullptr;
    p->graph32_key = -1;
  }
  if (!R.e0) {
    GPFVM_CUDA(cudaEventCreate(&R.e0));
    GPFVM_CUDA(cudaEventCreate(&R.e1));
  }
  GPFVM_CUDA(cudaEventRecord(R.e0, st));
  p->h_st32->pad[1] = 0;
  GPFVM_CUDA(cudaMemcpyAsync(&p->d_st32->pad[1], &p->h_st32->pad[1], sizeof(int), cudaMemcpyHostToDevice, st));
  GPFVM_CUDA(cudaMemsetAsync(&p->d_st->status, 0, sizeof(int), st));
  GPFVM_CUDA(cudaMemsetAsync(p->d_x, 0, sizeof(double) * p->N, st));
  if (o->want_var) GPFVM_CUDA(cudaMemsetAsync(p->d_down, 0, sizeof(double) * p->P, st));
  norm2(p->d_b, p->N, &p->d_st->aux[1], p->d_st, st);
  R.mstate = 0;
  R.outer = 0;
  R.total = 0;
  R.kstore = 0;
  R.idle = 0;
  R.tscale = 1.0;
  R.rel_prev = 1.0;
  R.status = GPFVM_NOT_CONVERGED;
  R.rel = 1.0;
  return GPFVM_OK;
}

// Enqueues the next piece of work (the FP64 residual, or up to n inner iterations).
void mixed_launch(gpfvm_problem* p, int, cudaStream_t st) {
  MixedRun& R = mruns()[p];
  const i64 N = p->N;
  if (R.mstate == 0) {
    if (R.outer == 0) {  // x = 0 (mixed_begin): r = b
      GPFVM_CUDA(cudaMemcpyAsync(p->d_r, p->d_b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    } else {
      GPFVM_CUDA(cudaMemcpyAsync(p->d_vin, p->d_x, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      fp64_ghat(p).run(st);
      axpby(p->d_b, p->d_vout, p->d_r, 1.0, -1.0, N, st);
    }
    norm2(p->d_r, N, &p->d_st->aux[0], p->d_st, st);
    copy_header_to_host(p, st);
    R.mstate = 1;
  } else if (R.mstate == 2 && R.launched == 0 && p->host_loop) {
    host_loop_run(p->graph32, p->graph32_kernels, p->d_st32, p->h_st32, st);
    R.launched = R.lim;
  } else if (R.mstate == 2 && R.launched == 0) {
    GPFVM_CUDA(cudaGraphLaunch(p->graph32, st));  // the whole inner run
    R.launched = R.lim;
    GPFVM_CUDA(cudaMemcpyAsync(p->h_st32, p->d_st32, offsetof(CGState, part), cudaMemcpyDeviceToHost, st));
  }
}

// Advances the state machine after the stream has been synchronised; may enqueue work.
void mixed_poll(gpfvm_problem* p, cudaStream_t st) {
  MixedRun& R = mruns()[p];
  const gpfvm_solve_opts* o = &R.o;
  const i64 N = p->N;
  if (R.mstate == 1) {
    if (p->h_st->status & DEV_TIMEOUT) { R.status = GPFVM_ERR_TIMEOUT; R.mstate = 3; return; }
    const double b2 = p->h_st->aux[1];
    R.rel = b2 > 0 ? std::sqrt(p->h_st->aux[0] / b2) : 0.0;
    if (!std::isfinite(R.rel)) { R.status = GPFVM_ERR_BREAKDOWN; R.mstate = 3; return; }
    // divergence guard: a run that raised the FP64 residual tenfold (operator
    // error times conditioning above one; CG residuals are not monotone, so
    // smaller rises are left alone) is undone, and the solve stops with the
    // previous iterate
    if (R.outer > 0 && R.rel > 10.0 * R.rel_prev) {
      add_f2d(p->d_x, p->f_d, N, st, &p->d_st32->aux[7], -1.0);
      R.rel = R.rel_prev;
      R.status = GPFVM_NOT_CONVERGED;
      R.mstate = 3;
      return;
    }
    R.rel_prev = R.rel;
    const bool cont = o->reorth == 1;  // conjugate continuation across runs
    // The last run stops where its FP32 recurrence estimates rtol; the FP64
    // residual then confirms it within a factor 2 (the estimate's error), else
    // the next run aims at half the remaining distance.
    if (R.rel <= o->rtol || (cont && R.outer > 0 && R.tscale >= 1.0 && R.rel <= 2.0 * o->rtol)) {
      R.status = GPFVM_OK;
      R.mstate = 3;
      return;
    }
    if (R.total >= o->max_iter || R.idle >= 3) { R.status = GPFVM_NOT_CONVERGED; R.mstate = 3; return; }
    if (R.outer > 0 && R.rel <= 2.0 * o->rtol) R.tscale *= 0.5;
    const bool var_now = o->want_var && (cont || R.outer == 0);
    const bool reorth_now = o->reorth != 0;  // 2: within each run only
    const int kbase = cont ? R.kstore : 0;
    const int run_cap = std::min(o->inner_max_iter > 0 ? o->inner_max_iter : p->cap, o->max_iter - R.total);
    if (cont) grow_store32(p, kbase + run_cap, kbase);
    const int icap = std::min(p->cap32 - kbase, run_cap);
    // stop the run where the continued recurrence reaches the outer tolerance
    const double itol = std::max(R.itol, R.rel > 0 ? R.tscale * o->rtol / R.rel : R.itol);
    p->h_st32->rtol2 = itol * itol;
    p->h_st32->max_iter = kbase + icap;
    p->h_st32->cap = p->cap32;
    p->h_st32->kbase = kbase;
    GPFVM_CUDA(cudaMemcpyAsync(&p->d_st32->rtol2, &p->h_st32->rtol2, sizeof(double), cudaMemcpyHostToDevice, st));
    GPFVM_CUDA(
        cudaMemcpyAsync(&p->d_st32->max_iter, &p->h_st32->max_iter, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
    GPFVM_CUDA(cudaMemcpyAsync(&p->d_st32->kbase, &p->h_st32->kbase, sizeof(int), cudaMemcpyHostToDevice, st));
    // the inner run solves for the normalised residual r / ||r||: FP32 then
    // sees unit-norm data whatever the scale of y (no under- or overflow)
    cg_init<double, float>(p->d_r, p->f_d, p->f_r, p->f_p, N, p->d_st32, st, &p->d_st->aux[0]);
    if (cont && kbase > 0)
      cg_project<float>(p->f_S, p->f_Q, p->f_r, p->f_d, p->f_p, N, p->cap32, p->d_st32, p->d_part2, p->d_coef,
                        p->d_eta32, st);
    const int key = (var_now ? 1 : 0) + (reorth_now ? 2 : 0);
    if (!p->graph32 || p->graph32_key != key) {
      if (p->graph32) cudaGraphExecDestroy(p->graph32);
      p->graph32 = nullptr;
      p->graph32 = make_loop_graph(p->d_st32, st, [&] { cg_iteration32(p, var_now, reorth_now, st); },
                                   &p->graph32_kernels, p->host_loop);
      p->graph32_key = key;
    }
    R.launched = 0;
    R.lim = p->h_st32->max_iter - kbase;
    R.mstate = 2;
  } else if (R.mstate == 2) {
    if (R.launched == 0) return;  // the inner run has not been launched yet
    count_launch((long long)p->h_st32->loops * p->graph32_kernels);
    const int k = p->h_st32->k - p->h_st32->kbase;  // iterations of this run
    R.total += k;
    if (o->reorth == 1) R.kstore = std::min(p->h_st32->k, p->cap32);
    if (p->h_st32->pad[1] & DEV_TIMEOUT) { R.status = GPFVM_ERR_TIMEOUT; R.mstate = 3; return; }
    // a breakdown inside a run ends that run (its stored directions stay
    // conjugate: the failed direction is never stored); none at all is an error
    if (k == 0 && !p->h_st32->converged) { R.status = GPFVM_ERR_BREAKDOWN; R.mstate = 3; return; }
    R.idle = k == 0 ? R.idle + 1 : 0;
    add_f2d(p->d_x, p->f_d, N, st, &p->d_st32->aux[7]);
    R.outer++;
    R.mstate = 0;
  }
}

bool mixed_finished(gpfvm_problem* p) { return mruns()[p].mstate == 3; }

int mixed_end(gpfvm_problem* p, gpfvm_solve_info* info, cudaStream_t st) {
  MixedRun& R = mruns()[p];
  GPFVM_CUDA(cudaEventRecord(R.e1, st));
  GPFVM_CUDA(cudaEventSynchronize(R.e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, R.e0, R.e1);
  gpfvm_solve_info I = p->last;
  I.iterations = R.total;
  I.status = R.status;
  I.rel_residual = R.rel;
  I.true_rel_residual = R.rel;
  I.t_solve_ms = ms;
  p->last = I;
  p->last_outer = R.outer;
  if (info) *info = I;
  p->solved = R.status >= 0;
  p->want_var_last = R.o.want_var != 0;
  p->last_store = R.o.reorth == 1 ? 2 : 0;
  p->last_kstore = R.o.reorth == 1 ? R.kstore : 0;
  return R.status;
}

int mixed_solve(gpfvm_problem* p, const gpfvm_solve_opts* o, gpfvm_solve_info* info, cudaStream_t st) {
  const int b = mixed_begin(p, o, st);
  if (b != GPFVM_OK) return b;
  const int chunk = o->check_every > 0 ? o->check_every : 16;
  while (!mixed_finished(p)) {
    mixed_launch(p, chunk, st);
    GPFVM_CUDA(cudaStreamSynchronize(st));
    mixed_poll(p, st);
  }
  return mixed_end(p, info, st);
}

// Precision-independent resumable solve, used by the batch and server drivers.
bool is_mixed(const gpfvm_solve_opts* o) { return o && o->precision != GPFVM_FP64; }
int any_begin(gpfvm_problem* p, const gpfvm_solve_opts* o, cudaStream_t st) {
  return is_mixed(o) ? mixed_begin(p, o, st) : solve_begin(p, o, st);
}
void any_launch(gpfvm_problem* p, const gpfvm_solve_opts* o, int n, cudaStream_t st) {
  if (is_mixed(o)) mixed_launch(p, n, st);
  else solve_launch(p, n, st);
}
bool any_poll_finished(gpfvm_problem* p, const gpfvm_solve_opts* o, cudaStream_t st) {
  if (is_mixed(o)) {
    mixed_poll(p, st);
    return mixed_finished(p);
  }
  return solve_finished(p);
}
int any_end(gpfvm_problem* p, const gpfvm_solve_opts* o, gpfvm_solve_info* info, cudaStream_t st) {
  return is_mixed(o) ? mixed_end(p, info, st) : solve_end(p, info, st);
}

}  // namespace

#define GPFVM_GUARD_BEGIN try {
#define GPFVM_GUARD_END                  \
  }                                      \
  catch (const CudaError& e) {           \
    return map_error(e);                 \
  }                                      \
  catch (const std::bad_alloc&) {        \
    return GPFVM_ERR_OUT_OF_MEMORY;      \
  }                                      \
  catch (...) {                          \
    return GPFVM_ERR_DEVICE;             \
  }

extern "C" {

int gpfvm_create(const gpfvm_desc* D, int max_iter, gpfvm_problem** out) {
  if (!out) return GPFVM_ERR_INVALID_ARG;
  *out = nullptr;
  const int v = validate(D);
  if (v != GPFVM_OK) return v;
  std::unique_ptr<gpfvm_problem> p(new gpfvm_problem());
  GPFVM_GUARD_BEGIN
  p->d = D->ndim;
  p->N = 1;
  p->P = 1;
  for (int i = 0; i < p->d; ++i) {
    p->nc[i] = D->n_cells[i];
    p->edges[i].assign(D->edges[i], D->edges[i] + D->n_cells[i] + 1);
    p->ell[i] = D->lengthscale[i];
    p->npred[i] = D->n_pred[i];
    p->pred[i].assign(D->pred[i], D->pred[i] + D->n_pred[i]);
    p->N *= p->nc[i];
    p->P *= p->npred[i];
  }
  p->Nc = p->N;
  p->Pp = p->P;
  if (D->n_outputs > 0) {
    p->nout = D->n_outputs;
    p->neq = 0;
    for (int k = 0; k < D->n_terms; ++k) {
      p->teq[k] = D->term_eq[k];
      p->tout[k] = D->term_out[k];
      p->neq = std::max(p->neq, p->teq[k] + 1);
    }
    p->multi = p->nout > 1 || p->neq > 1;
  }
  if (p->multi) {
    p->N = p->Nc * p->neq;
    p->P = p->Pp * p->nout;
  } else {
    p->neq = p->nout = 1;
    for (int k = 0; k < D->n_terms; ++k) p->teq[k] = p->tout[k] = 0;
  }
  p->s2 = D->outputscale;
  p->jitter = D->jitter;
  p->colloc = D->observe == 1;
  p->oz_on = D->fp64_products == 0;
  p->nterms = D->n_terms;
  for (int k = 0; k < GPFVM_MAX_TERMS; ++k) p->fclass[k] = -1;
  {
    std::vector<const double*> seen;
    for (int k = 0; k < D->n_terms; ++k) {
      const double* f = D->coef_field[k];
      if (!f) continue;
      int c = -1;
      for (size_t j = 0; j < seen.size(); ++j)
        if (seen[j] == f) c = (int)j;
      if (c < 0) {
        c = (int)seen.size();
        seen.push_back(f);
        i64 n = 1;
        for (int i = 0; i < D->ndim; ++i) n *= D->n_cells[i];
        p->fields.insert(p->fields.end(), f, f + n);
      }
      p->fclass[k] = c;
    }
    p->nfield = (int)seen.size();
  }
  for (int k = 0; k < p->nterms; ++k) {
    p->coef[k] = D->coef[k];
    for (int i = 0; i < p->d; ++i) p->alpha[k][i] = D->alpha[k][i];
  }
  if (D->rhs) p->rhs.assign(D->rhs, D->rhs + p->N);
  p->nsets = D->n_sets;
  i64 off = 0;
  for (int s = 0; s < p->nsets; ++s) {
    SetC& S = p->sets[s];
    S.size = 1;
    for (int i = 0; i < p->d; ++i) {
      S.order[i] = D->sets[s].order[i];
      S.n[i] = D->sets[s].n_pts[i];
      S.coords[i].assign(D->sets[s].coords[i], D->sets[s].coords[i] + S.n[i]);
      S.size *= S.n[i];
    }
    if (D->sets[s].values) S.values.assign(D->sets[s].values, D->sets[s].values + S.size);
    else S.values.assign(S.size, 0.0);
    S.noise = D->sets[s].noise_var;
    S.comp = p->multi ? D->set_out[s] : 0;
    S.off = off;
    off += S.size;
    p->uset[s] = s;
    p->uslice[s] = -1;
  }
  p->nusets = p->nsets;
  p->M = off;
  stack_sets(p.get());
  p->cap = max_iter > 0 ? max_iter : 2000;
  // register the 1D factors the problem needs
  for (int a = 0; a < p->nterms; ++a)
    for (int b = 0; b < p->nterms; ++b)
      for (int i = 0; i < p->d; ++i) need_factor(p.get(), i, 0, p->alpha[a][i], 0, p->alpha[b][i]);
  for (int s = 0; s < p->nsets; ++s) {
    for (int a = 0; a < p->nterms; ++a)
      for (int i = 0; i < p->d; ++i) need_factor(p.get(), i, 0, p->alpha[a][i], 1, s);
    for (int s2 = 0; s2 < p->nsets; ++s2)
      for (int i = 0; i < p->d; ++i) need_factor(p.get(), i, 1, s, 1, s2);
    for (int i = 0; i < p->d; ++i) need_factor(p.get(), i, 1, s, 2, 0);
  }
  for (int a = 0; a < p->nterms; ++a)
    for (int i = 0; i < p->d; ++i) need_factor(p.get(), i, 0, p->alpha[a][i], 2, 0);
  {
    const char* e = std::getenv("GPFVM_HOST_LOOP");
    p->host_loop = e && std::atoi(e) != 0;
  }
  alloc_all(p.get());
  *out = p.release();
  return GPFVM_OK;
  GPFVM_GUARD_END
}

void gpfvm_destroy(gpfvm_problem* p) {
  if (!p) return;
  {
    auto it = runs().find(p);
    if (it != runs().end()) {
      if (it->second.e0) cudaEventDestroy(it->second.e0);
      if (it->second.e1) cudaEventDestroy(it->second.e1);
      runs().erase(it);
    }
    auto jt = mruns().find(p);
    if (jt != mruns().end()) {
      if (jt->second.e0) cudaEventDestroy(jt->second.e0);
      if (jt->second.e1) cudaEventDestroy(jt->second.e1);
      mruns().erase(jt);
    }
  }
  auto& m = own_streams();
  auto it = m.find(p);
  if (it != m.end()) {
    cudaStreamSynchronize(it->second);
    cudaStreamDestroy(it->second);
    m.erase(it);
  }
  delete p;
}

int gpfvm_sizes(const gpfvm_problem* p, int64_t out[4]) {
  if (!p || !out) return GPFVM_ERR_INVALID_ARG;
  out[0] = p->N;
  out[1] = p->M;
  out[2] = p->P;
  out[3] = p->cap;
  return GPFVM_OK;
}

int gpfvm_assemble(gpfvm_problem* p, void* stream) {
  if (!p) return GPFVM_ERR_INVALID_ARG;
  GPFVM_GUARD_BEGIN
  cudaStream_t st = pick_stream(p, stream);
  cudaEvent_t e0, e1;
  GPFVM_CUDA(cudaEventCreate(&e0));
  GPFVM_CUDA(cudaEventCreate(&e1));
  GPFVM_CUDA(cudaEventRecord(e0, st));
  const int r = run_assemble(p, st);
  GPFVM_CUDA(cudaEventRecord(e1, st));
  GPFVM_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  p->last.t_assemble_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
  GPFVM_GUARD_END
}

}  // extern "C"

namespace {
// The FP32 operators of gpfvm_gram_matvec: op -> plan and whether it maps the
// inner CG vectors f_p -> f_q (else f_vin -> f_vout); nullptr for FP64 ops.
//   4 G_PP FP32 SIMT, 5 G_PP split TF32, 6 G^ FP32, 7 G^ split TF32,
//   8 G_PP split BF16, 9 G^ split BF16, 10 G_PP BF16, 11 G^ BF16
const Plan* op32_plan(gpfvm_problem* p, int op, bool* inner) {
  *inner = (op == 6 || op == 7 || op == 9 || op == 11);
  switch (op) {
    case 4: return &p->p_pp32;
    case 5: return &p->p_pp32tc[TC_TF32X3];
    case 6: return &p->p_mv32;
    case 7: return &p->p_mv32tc[TC_TF32X3];
    case 8: return &p->p_pp32tc[TC_BF16X3];
    case 9: return &p->p_mv32tc[TC_BF16X3];
    case 10: return &p->p_pp32tc[TC_BF16];
    case 11: return &p->p_mv32tc[TC_BF16];
    default: return nullptr;
  }
}
bool op_uses_tc(int op) { return op == 5 || op >= 7; }
}  // namespace

extern "C" {

int gpfvm_gram_matvec(gpfvm_problem* p, int op, const double* v, double* out, void* stream) {
  if (!p || !v || !out || op < 0 || op > 13) return GPFVM_ERR_INVALID_ARG;
  if (!p->assembled) return GPFVM_ERR_STATE;
  if ((op == 2 || op == 3) && p->M == 0) return GPFVM_ERR_INVALID_ARG;
  if (op_uses_tc(op) && !p->tc_ok) return GPFVM_ERR_INVALID_ARG;
  if (op >= 12 && !p->oz_ok) return GPFVM_ERR_INVALID_ARG;
  if (p->multi && op > 3) return GPFVM_ERR_INVALID_ARG;  // systems: the FP64 operators 0-3
  GPFVM_GUARD_BEGIN
  cudaStream_t st = pick_stream(p, stream);
  bool inner = false;
  if (const Plan* pl = op32_plan(p, op, &inner)) {
    // FP32 operators: the inner ones are gated by the inner "done" flag
    p->h_st32->done = 0;
    p->h_st32->pad[1] = 0;
    GPFVM_CUDA(cudaMemcpyAsync(&p->d_st32->done, &p->h_st32->done, sizeof(int), cudaMemcpyHostToDevice, st));
    GPFVM_CUDA(cudaMemcpyAsync(&p->d_st32->pad[1], &p->h_st32->pad[1], sizeof(int), cudaMemcpyHostToDevice, st));
    convert_d2f(v, inner ? p->f_p : p->f_vin, p->N, st);
    pl->run(st);
    f2d(inner ? p->f_q : p->f_vout, out, p->N, st);
    GPFVM_CUDA(cudaMemcpyAsync(p->h_st32, p->d_st32, offsetof(CGState, part), cudaMemcpyDeviceToHost, st));
    GPFVM_CUDA(cudaStreamSynchronize(st));
    return (p->h_st32->pad[1] & DEV_TIMEOUT) ? GPFVM_ERR_TIMEOUT : GPFVM_OK;
  }
  const i64 nin = (op == 3) ? p->M : p->N;
  const i64 nout = (op == 2) ? p->M : p->N;
  double* in = (op == 3) ? p->d_win : p->d_vin;
  double* res = (op == 2) ? p->d_wout : p->d_vout;
  GPFVM_CUDA(cudaMemcpyAsync(in, v, sizeof(double) * nin, cudaMemcpyDeviceToDevice, st));
  if (op >= 12) GPFVM_CUDA(cudaMemsetAsync(&p->d_st->status, 0, sizeof(int), st));
  p->p_op[op >= 12 ? op - 8 : op].run(st);
  GPFVM_CUDA(cudaMemcpyAsync(out, res, sizeof(double) * nout, cudaMemcpyDeviceToDevice, st));
  if (op >= 12) GPFVM_CUDA(cudaMemcpyAsync(p->h_st, p->d_st, offsetof(CGState, part), cudaMemcpyDeviceToHost, st));
  GPFVM_CUDA(cudaStreamSynchronize(st));
  if (op >= 12 && (p->h_st->status & DEV_TIMEOUT)) return GPFVM_ERR_TIMEOUT;
  return GPFVM_OK;
  GPFVM_GUARD_END
}

int gpfvm_gram_matvec_bench(gpfvm_problem* p, int op, const double* v, double* out, int reps, void* stream,
                            double* ms_per_application) {
  if (!p || !v || !out || !ms_per_application || reps < 1 || op < 0 || op > 13) return GPFVM_ERR_INVALID_ARG;
  if (!p->assembled) return GPFVM_ERR_STATE;
  if ((op == 2 || op == 3) && p->M == 0) return GPFVM_ERR_INVALID_ARG;
  if (op_uses_tc(op) && !p->tc_ok) return GPFVM_ERR_INVALID_ARG;
  if (op >= 12 && !p->oz_ok) return GPFVM_ERR_INVALID_ARG;
  if (p->multi && op > 3) return GPFVM_ERR_INVALID_ARG;  // systems: the FP64 operators 0-3
  GPFVM_GUARD_BEGIN
  cudaStream_t st = pick_stream(p, stream);
  bool inner = false;
  const Plan* plan = op32_plan(p, op, &inner);
  if (plan) {
    p->h_st32->done = 0;
    p->h_st32->pad[1] = 0;
    GPFVM_CUDA(cudaMemcpyAsync(&p->d_st32->done, &p->h_st32->done, sizeof(int), cudaMemcpyHostToDevice, st));
    GPFVM_CUDA(cudaMemcpyAsync(&p->d_st32->pad[1], &p->h_st32->pad[1], sizeof(int), cudaMemcpyHostToDevice, st));
  }
  const i64 nin = (op == 3) ? p->M : p->N;
  const i64 nout = (op == 2) ? p->M : p->N;
  if (plan) {
    convert_d2f(v, inner ? p->f_p : p->f_vin, p->N, st);
  } else {
    GPFVM_CUDA(cudaMemcpyAsync(op == 3 ? p->d_win : p->d_vin, v, sizeof(double) * nin, cudaMemcpyDeviceToDevice, st));
    plan = &p->p_op[op >= 12 ? op - 8 : op];
  }
  const bool is32 = op >= 4 && op <= 11;
  // one application as a CUDA graph, replayed reps times between events
  cudaGraph_t g = nullptr;
  const long long before = g_launches.load();
  GPFVM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  try {
    plan->run(st);
  } catch (...) {
    cudaGraph_t dummy;
    cudaStreamEndCapture(st, &dummy);
    cudaGetLastError();
    throw;
  }
  GPFVM_CUDA(cudaStreamEndCapture(st, &g));
  const long long kernels = g_launches.load() - before;
  g_launches.fetch_sub(kernels);
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  GPFVM_CUDA(e);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  try {
    GPFVM_CUDA(cudaEventCreate(&e0));
    GPFVM_CUDA(cudaEventCreate(&e1));
    for (int i = 0; i < 2; ++i) GPFVM_CUDA(cudaGraphLaunch(ex, st));  // warm-up
    GPFVM_CUDA(cudaEventRecord(e0, st));
    for (int i = 0; i < reps; ++i) GPFVM_CUDA(cudaGraphLaunch(ex, st));
    GPFVM_CUDA(cudaEventRecord(e1, st));
    count_launch((long long)(reps + 2) * kernels);
    GPFVM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    GPFVM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *ms_per_application = (double)ms / reps;
    if (is32) f2d(inner ? p->f_q : p->f_vout, out, p->N, st);
    else GPFVM_CUDA(cudaMemcpyAsync(out, op == 2 ? p->d_wout : p->d_vout, sizeof(double) * nout,
                                    cudaMemcpyDeviceToDevice, st));
    GPFVM_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGraphExecDestroy(ex);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(ex);
  return GPFVM_OK;
  GPFVM_GUARD_END
}

int gpfvm_solve(gpfvm_problem* p, const gpfvm_solve_opts* opts, gpfvm_solve_info* info, void* stream) {
  if (!p) return GPFVM_ERR_INVALID_ARG;
  GPFVM_GUARD_BEGIN
  return run_solve(p, opts, info, pick_stream(p, stream));
  GPFVM_GUARD_END
}

int gpfvm_query(gpfvm_problem* p, double* mean, double* var, void* stream) {
  if (!p || (!mean && !var)) return GPFVM_ERR_INVALID_ARG;
  GPFVM_GUARD_BEGIN
  cudaStream_t st = pick_stream(p, stream);
  cudaEvent_t e0, e1;
  GPFVM_CUDA(cudaEventCreate(&e0));
  GPFVM_CUDA(cudaEventCreate(&e1));
  GPFVM_CUDA(cudaEventRecord(e0, st));
  const int r = run_query(p, mean, var, st);
  GPFVM_CUDA(cudaEventRecord(e1, st));
  GPFVM_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  p->last.t_query_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
  GPFVM_GUARD_END
}

int gpfvm_autotune(gpfvm_problem* p, int precision, void* stream, double* report, int report_cap) {
  if (!p || precision < GPFVM_FP64 || precision > GPFVM_MIXED_BF16) return GPFVM_ERR_INVALID_ARG;
  if (!p->assembled) return GPFVM_ERR_STATE;
  static const int op_of[5] = {1, 6, 7, 9, 11};  // the solver's operator of each precision
  const int op = op_of[precision];
  const bool tc = precision >= GPFVM_MIXED_TF32X3;
  if (tc && !p->tc_ok) return GPFVM_ERR_INVALID_ARG;
  GPFVM_GUARD_BEGIN
  cudaStream_t st = pick_stream(p, stream);
  // cache key: precision, operator terms and the axis sizes rounded up to 16
  auto up16 = [](int n) { return (n + 15) / 16 * 16; };
  std::vector<int> key = {precision, p->d, p->nterms, p->M > 0, up16(p->nc[0]), p->d > 1 ? up16(p->nc[1]) : 1,
                          p->d > 2 ? up16(p->nc[2]) : 1};
  for (int a = 0; a < p->nterms; ++a)
    for (int i = 0; i < p->d; ++i) key.push_back(p->alpha[a][i]);
  static std::mutex mu;
  static std::map<std::vector<int>, std::pair<int, int>> cache;
  std::pair<int, int> best{-1, 0};
  bool hit = false;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) { best = it->second; hit = true; }
  }
  int nrep = 0;
  if (!hit) {
    double *v = nullptr, *out = nullptr;
    GPFVM_CUDA(cudaMalloc(&v, sizeof(double) * p->N));
    if (cudaMalloc(&out, sizeof(double) * p->N) != cudaSuccess) {
      cudaFree(v);
      return GPFVM_ERR_OUT_OF_MEMORY;
    }
    double best_ms = 1e300;
    try {
      GPFVM_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * p->N, st));
      for (int tcg = 0; tcg < (tc ? 2 : 1); ++tcg)
        for (int tile = -1; tile <= 2; ++tile) {
          rebuild_plans(p, tile, tcg);
          double ms = 0.0;
          const int r = gpfvm_gram_matvec_bench(p, op, v, out, 8, stream, &ms);
          if (r != GPFVM_OK) throw CudaError{cudaErrorUnknown, "autotune timing"};
          if (report && nrep < report_cap) report[nrep] = ms;
          ++nrep;
          if (ms < best_ms) { best_ms = ms; best = {tile, tcg}; }
        }
    } catch (...) {
      cudaFree(v);
      cudaFree(out);
      rebuild_plans(p, -1, 0);
      throw;
    }
    cudaFree(v);
    cudaFree(out);
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best;
  }
  if (p->tuned_tile != best.first || p->tuned_tc != best.second) rebuild_plans(p, best.first, best.second);
  if (report && nrep < report_cap) report[nrep] = 3 * (best.first + 1) + best.second;  // the choice
  return hit ? 1 : 0;
  GPFVM_GUARD_END
}

int gpfvm_target(gpfvm_problem* p, const double* beta, int n_actions, void* stream) {
  if (!p || !beta || n_actions < 1 || p->multi) return GPFVM_ERR_INVALID_ARG;
  GPFVM_GUARD_BEGIN
  cudaStream_t st = pick_stream(p, stream);
  if (!p->solved || p->last_store != 1 || !p->want_var_last) return GPFVM_ERR_STATE;
  const int k0 = p->last_kstore;
  if (k0 + n_actions > p->cap) return GPFVM_ERR_INVALID_ARG;
  const i64 N = p->N, P = p->P;
  grow_store64(p, k0 + n_actions, k0);
  // the scalar header of the finished CG run: never "converged" (rtol2 < 0),
  // k0 + n_actions iterations in all, stores of cap64 directions
  CGState& h = *p->h_st;
  h.rtol2 = -1.0;
  h.max_iter = k0 + n_actions;
  h.cap = p->cap64;
  h.done = 0;
  GPFVM_CUDA(cudaMemcpyAsync(&p->d_st->rtol2, &h.rtol2, sizeof(double), cudaMemcpyHostToDevice, st));
  GPFVM_CUDA(cudaMemcpyAsync(&p->d_st->max_iter, &h.max_iter, 2 * sizeof(int), cudaMemcpyHostToDevice, st));
  GPFVM_CUDA(cudaMemcpyAsync(&p->d_st->done, &h.done, sizeof(int), cudaMemcpyHostToDevice, st));
  for (int a = 0; a < n_actions; ++a) {
    GPFVM_CUDA(cudaMemcpyAsync(p->d_tbeta, beta + (i64)a * P, sizeof(double) * P, cudaMemcpyDeviceToDevice, st));
    p->p_tgt.run(st);  // p = Lhat k(X*) beta
    // action s = t - G^ C t, direction d = s - C G^ s (conjugate to every stored one)
    cg_residual_wrt(p->d_S, p->d_Q, p->d_p, N, p->cap64, p->d_st, p->d_part2, p->d_coef, p->d_eta, st);
    cg_reorth(p->d_S, p->d_Q, p->d_p, N, p->cap64, p->d_st, p->d_part2, p->d_coef, p->d_eta, st);
    p->p_mvv_cg.run(st);  // q = G^ d, u = Lhat k(X*)^T d
    cg_dot_eta_pr(p->d_p, p->d_q, p->d_r, N, p->d_st, p->d_eta, st);
    cg_downdate(p->d_u, p->d_down, P, p->d_st, st);
    cg_update(p->d_x, p->d_r, p->d_p, p->d_q, N, p->d_st, p->d_S, p->d_Q, st, true);
  }
  copy_header_to_host(p, st);
  GPFVM_CUDA(cudaStreamSynchronize(st));
  p->last_kstore = std::min(h.k, p->cap64);
  if (h.status & DEV_BREAKDOWN) return GPFVM_ERR_BREAKDOWN;
  return GPFVM_OK;
  GPFVM_GUARD_END
}

int gpfvm_solve_host(gpfvm_problem* p, const double* values_host, const gpfvm_solve_opts* opts, double* mean_host,
                     double* var_host, gpfvm_solve_info* info, void* stream) {
  if (!p || !opts || !mean_host) return GPFVM_ERR_INVALID_ARG;
  GPFVM_GUARD_BEGIN
  cudaStream_t st = pick_stream(p, stream);
  if (values_host && p->M > 0)
    GPFVM_CUDA(cudaMemcpyAsync(p->d_yB, values_host, sizeof(double) * p->M, cudaMemcpyHostToDevice, st));
  int r;
  if (!p->assembled) {
    r = run_assemble(p, st);
    if (r != GPFVM_OK) return r;
  } else {
    p->p_rhs.run(st);
  }
  r = run_solve(p, opts, info, st);
  if (r < 0) return r;
  const int q = run_query(p, p->d_mean, var_host ? p->d_var : nullptr, st);
  if (q != GPFVM_OK) return q;
  GPFVM_CUDA(cudaMemcpyAsync(mean_host, p->d_mean, sizeof(double) * p->P, cudaMemcpyDeviceToHost, st));
  if (var_host) GPFVM_CUDA(cudaMemcpyAsync(var_host, p->d_var, sizeof(double) * p->P, cudaMemcpyDeviceToHost, st));
  GPFVM_CUDA(cudaStreamSynchronize(st));
  return r;
  GPFVM_GUARD_END
}

int64_t gpfvm_export(gpfvm_problem* p, int what, double* host_out, int64_t capacity, void* stream) {
  if (!p || !host_out) return GPFVM_ERR_INVALID_ARG;
  GPFVM_GUARD_BEGIN
  cudaStream_t st = pick_stream(p, stream);
  const double* src = nullptr;
  i64 n = 0;
  switch (what) {
    case 0: src = p->d_b; n = p->N; break;
    case 1: src = p->d_x; n = p->N; break;
    case 2: src = p->d_A; n = p->M * p->M; break;
    case 3: src = p->d_Linv; n = p->M * p->M; break;
    case 5: src = p->d_down; n = p->P; break;
    case 6: src = p->d_eta; n = p->last.iterations; break;
    case 8: {  // refinement steps of the last mixed-precision solve
      host_out[0] = p->last_outer;
      return 1;
    }
    case 10: {  // IC/BC stage: structured (1) or dense (0), rows of the structured set, other rows
      if (capacity < 3) return GPFVM_ERR_INVALID_ARG;
      host_out[0] = p->sicbc ? 1.0 : 0.0;
      host_out[1] = p->sicbc ? p->MK : 0;
      host_out[2] = p->sicbc ? p->MR : (double)p->M;
      return 3;
    }
    case 9: {  // eigensolver sweeps (FP32, FP64) per axis of the structured IC/BC stage
      if (!p->d_jac_sweeps) return 0;
      if (capacity < 2 * p->d) return GPFVM_ERR_INVALID_ARG;
      int sw[2 * GPFVM_MAX_DIM] = {};
      GPFVM_CUDA(cudaMemcpyAsync(sw, p->d_jac_sweeps, sizeof(int) * 2 * p->d, cudaMemcpyDeviceToHost, st));
      GPFVM_CUDA(cudaStreamSynchronize(st));
      for (int i = 0; i < 2 * p->d; ++i) host_out[i] = sw[i];
      return 2 * p->d;
    }
    case 11: {  // stored directions p_j of the last solve (k rows of N), k = what 12's count
      const i64 k = p->last_kstore, ld = store_ld(p->N);
      if (k * p->N > capacity) return GPFVM_ERR_INVALID_ARG;
      if (p->last_store == 1) {
        GPFVM_CUDA(cudaMemcpy2DAsync(host_out, sizeof(double) * p->N, p->d_S, sizeof(double) * ld,
                                     sizeof(double) * p->N, k, cudaMemcpyDeviceToHost, st));
        GPFVM_CUDA(cudaStreamSynchronize(st));
      } else if (p->last_store == 2) {
        std::vector<float> tmp((size_t)(k * p->N));
        GPFVM_CUDA(cudaMemcpy2DAsync(tmp.data(), sizeof(float) * p->N, p->f_S, sizeof(float) * ld,
                                     sizeof(float) * p->N, k, cudaMemcpyDeviceToHost, st));
        GPFVM_CUDA(cudaStreamSynchronize(st));
        for (i64 i = 0; i < k * p->N; ++i) host_out[i] = tmp[(size_t)i];
      }
      return p->last_store ? k * p->N : 0;
    }
    case 12: {  // eta_j = p_j^T G^ p_j of the stored directions (the operator of their precision)
      const i64 k = p->last_kstore;
      if (k > capacity) return GPFVM_ERR_INVALID_ARG;
      if (p->last_store && k > 0) {
        GPFVM_CUDA(cudaMemcpyAsync(host_out, p->last_store == 1 ? p->d_eta : p->d_eta32, sizeof(double) * k,
                                   cudaMemcpyDeviceToHost, st));
        GPFVM_CUDA(cudaStreamSynchronize(st));
      }
      return p->last_store ? k : 0;
    }
    case 7: {  // timing of the last assemble / solve / query (ms)
      if (capacity < 3) return GPFVM_ERR_INVALID_ARG;
      host_out[0] = p->last.t_assemble_ms;
      host_out[1] = p->last.t_solve_ms;
      host_out[2] = p->last.t_query_ms;
      return 3;
    }
    default: return GPFVM_ERR_INVALID_ARG;
  }
  if (n > capacity) return GPFVM_ERR_INVALID_ARG;
  if (n > 0 && !src) return GPFVM_ERR_STATE;  // e.g. L^-1 under the structured IC/BC stage
  if (what == 2) {
    // G_BB is overwritten by the Cholesky recursion: rebuild it
    p->p_setup.run(st);
  }
  if (n > 0) GPFVM_CUDA(cudaMemcpyAsync(host_out, src, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  GPFVM_CUDA(cudaStreamSynchronize(st));
  return n;
  GPFVM_GUARD_END
}

int64_t gpfvm_factor(gpfvm_problem* p, int axis, int kind_a, int arg_a, int kind_b, int arg_b, double* host_out,
                     int64_t capacity, void* stream) {
  if (!p || !host_out || axis < 0 || axis >= p->d) return GPFVM_ERR_INVALID_ARG;
  // the caller's set numbers -> internal sets (and the axis-0 point of a stacked set)
  int ia = arg_a, ib = arg_b, sa = -1, sb = -1;
  if (kind_a == 1) {
    if (arg_a < 0 || arg_a >= p->nusets) return GPFVM_ERR_NOT_FOUND;
    ia = p->uset[arg_a];
    if (axis == 0) sa = p->uslice[arg_a];
  }
  if (kind_b == 1) {
    if (arg_b < 0 || arg_b >= p->nusets) return GPFVM_ERR_NOT_FOUND;
    ib = p->uset[arg_b];
    if (axis == 0) sb = p->uslice[arg_b];
  }
  auto it = p->fac_off.find(FKey(axis, kind_a, ia, kind_b, ib));
  if (it == p->fac_off.end()) return GPFVM_ERR_NOT_FOUND;
  GPFVM_GUARD_BEGIN
  cudaStream_t st = pick_stream(p, stream);
  const i64 na = fam_n(p, axis, kind_a, ia), nb = fam_n(p, axis, kind_b, ib);
  const i64 ra = sa >= 0 ? 1 : na, rb = sb >= 0 ? 1 : nb;
  if (ra * rb > capacity) return GPFVM_ERR_INVALID_ARG;
  p->p_setup.run(st);
  std::vector<double> full(sa >= 0 || sb >= 0 ? na * nb : 0);
  double* dst = full.empty() ? host_out : full.data();
  GPFVM_CUDA(cudaMemcpyAsync(dst, p->d_fac + it->second, sizeof(double) * na * nb, cudaMemcpyDeviceToHost, st));
  GPFVM_CUDA(cudaStreamSynchronize(st));
  if (!full.empty())
    for (i64 i = 0; i < ra; ++i)
      for (i64 j = 0; j < rb; ++j) host_out[i * rb + j] = full[(sa >= 0 ? sa : i) * nb + (sb >= 0 ? sb : j)];
  return ra * rb;
  GPFVM_GUARD_END
}

int gpfvm_set_values(gpfvm_problem* p, const double* values, void* stream) {
  if (!p || (!values && p->M > 0)) return GPFVM_ERR_INVALID_ARG;
  if (!p->assembled) return GPFVM_ERR_STATE;
  GPFVM_GUARD_BEGIN
  cudaStream_t st = pick_stream(p, stream);
  if (p->M > 0) GPFVM_CUDA(cudaMemcpyAsync(p->d_yB, values, sizeof(double) * p->M, cudaMemcpyDeviceToDevice, st));
  p->p_rhs.run(st);
  p->solved = false;
  return GPFVM_OK;
  GPFVM_GUARD_END
}

int64_t gpfvm_launch_count(void) { return g_launches.load(); }

const char* gpfvm_strerror(int code) {
  switch (code) {
    case GPFVM_OK: return "ok";
    case GPFVM_NOT_CONVERGED: return "iteration budget exhausted before the tolerance";
    case GPFVM_ERR_INVALID_ARG: return "invalid argument";
    case GPFVM_ERR_OUT_OF_MEMORY: return "out of device memory";
    case GPFVM_ERR_NOT_SPD: return "IC/BC Gram matrix not positive definite (Cholesky pivot <= 0)";
    case GPFVM_ERR_BREAKDOWN: return "CG breakdown (p^T G p <= 0 or not finite)";
    case GPFVM_ERR_DEVICE: return "CUDA error";
    case GPFVM_ERR_TIMEOUT: return "bounded device wait timed out";
    case GPFVM_ERR_STATE: return "call out of order";
    case GPFVM_ERR_NOT_FOUND: return "not found";
    case GPFVM_ERR_TOO_LARGE: return "request exceeds the static scratch capacity of the allocation-free path";
    default: return "unknown status";
  }
}

const char* gpfvm_version(void) { return "gpfvm 0.1 sm_103a"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched solves: every problem runs on its own stream, each CG run as one
// device-side loop (a graph WHILE node), so the problems' kernels overlap on
// the device; the host only advances the mixed-precision refinement steps of
// problems whose streams have gone idle.
// ---------------------------------------------------------------------------
extern "C" int gpfvm_solve_batch(gpfvm_problem** ps, int n, const gpfvm_solve_opts* opts, gpfvm_solve_info* infos,
                                 void* stream) {
  if (!ps || n < 0 || !opts) return GPFVM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!ps[i] || ps[i]->multi) return GPFVM_ERR_INVALID_ARG;  // (systems: one at a time)
  GPFVM_GUARD_BEGIN
  cudaEvent_t ev;
  GPFVM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  if (stream) GPFVM_CUDA(cudaEventRecord(ev, (cudaStream_t)stream));
  std::vector<cudaStream_t> sts(n);
  std::vector<int> active(n, 1);
  int worst = GPFVM_OK;
  for (int i = 0; i < n; ++i) {
    sts[i] = pick_stream(ps[i], nullptr);
    if (stream) GPFVM_CUDA(cudaStreamWaitEvent(sts[i], ev, 0));
    const int b = any_begin(ps[i], opts, sts[i]);
    if (b != GPFVM_OK) {
      active[i] = 0;
      worst = std::min(worst, b);
      if (infos) infos[i].status = b;
    }
  }
  // every problem runs its own device-side loops on its own stream; the host
  // advances whichever problem's stream has gone idle
  int left = 0;
  for (int i = 0; i < n; ++i) left += active[i];
  std::vector<char> pending(n, 0);
  while (left > 0) {
    bool progressed = false;
    for (int i = 0; i < n; ++i) {
      if (!active[i]) continue;
      if (!pending[i]) {
        any_launch(ps[i], opts, 0, sts[i]);
        pending[i] = 1;
      }
      const cudaError_t q = cudaStreamQuery(sts[i]);
      if (q == cudaErrorNotReady) continue;
      GPFVM_CUDA(q);
      pending[i] = 0;
      progressed = true;
      if (any_poll_finished(ps[i], opts, sts[i])) {
        const int r = any_end(ps[i], opts, infos ? &infos[i] : nullptr, sts[i]);
        if (r < 0) worst = std::min(worst, r);
        else if (r == GPFVM_NOT_CONVERGED && worst == GPFVM_OK) worst = r;
        active[i] = 0;
        --left;
      }
    }
    if (!progressed) std::this_thread::yield();
  }
  cudaEventDestroy(ev);
  return worst;
  GPFVM_GUARD_END
}

// ---------------------------------------------------------------------------
// Batched solves as ONE graph launch.  Every problem's whole solve is a
// device-driven loop: a WHILE node whose body computes the FP64 residual,
// takes the refinement decision on the device (mixed_ctl), runs the inner CG
// as a nested WHILE node and applies the correction (mixed_post); an FP64
// problem's body is its CG iteration.  All problems' loops are independent
// branches of one graph, launched once; the host only sets them up before
// and reads their states after.  The direction stores cannot grow inside a
// graph, so they are allocated up front: every run's directions with reorth 1
// (up to max_iter), one run's with reorth 0 or 2.
// ---------------------------------------------------------------------------
namespace {

struct CaptureGuard {  // ends a failed capture so that the stream stays usable
  cudaStream_t st;
  bool active = true;
  ~CaptureGuard() {
    if (active) {
      cudaGraph_t dummy = nullptr;
      cudaStreamEndCapture(st, &dummy);
      if (dummy) cudaGraphDestroy(dummy);
      cudaGetLastError();
    }
  }
};

// Adds to `g` the WHILE node of one problem's device-driven solve (handle
// created on g); *k_outer / *k_inner receive the kernels of one outer / inner
// pass (for the launch count).
void add_solve_loop(gpfvm_problem* p, const gpfvm_solve_opts* o, cudaGraph_t g, cudaStream_t st, cudaStream_t st2,
                    long long* k_outer, long long* k_inner) {
  const i64 N = p->N;
  const bool mixed = o->precision != GPFVM_FP64;
  cudaGraphConditionalHandle ho;
  GPFVM_CUDA(cudaGraphConditionalHandleCreate(&ho, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = ho;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t wo;
  GPFVM_CUDA(cudaGraphAddNode(&wo, g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  const int unroll = loop_unroll();
  if (!mixed) {  // FP64: the CG iteration itself, as in make_loop_graph
    const bool reorth = o->reorth != 0, want_var = o->want_var != 0;
    const long long before = g_launches.load();
    GPFVM_CUDA(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    {
      CaptureGuard cg{st};
      for (int u = 0; u < unroll; ++u) cg_iteration(p, reorth, want_var, st);
      loop_ctl(p->d_st, ho, st);
      cudaGraph_t out;
      cg.active = false;
      GPFVM_CUDA(cudaStreamEndCapture(st, &out));
    }
    *k_inner = g_launches.load() - before;
    g_launches.fetch_sub(*k_inner);
    *k_outer = 0;
    return;
  }
  MixedCtl* c = p->d_mctl;
  const bool reorth = o->reorth != 0, cont = o->reorth == 1, want_var = o->want_var != 0;
  // segment A: FP64 residual, decision, start of the next run
  const long long before = g_launches.load();
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  std::vector<cudaGraphNode_t> tail;
  cudaGraphConditionalHandle hi;
  GPFVM_CUDA(cudaGraphConditionalHandleCreate(&hi, body, 0, 0));
  GPFVM_CUDA(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  {
    CaptureGuard cg{st};
    axpby(p->d_x, p->d_x, p->d_vin, 1.0, 0.0, N, st);  // vin = x (a kernel node)
    p->p_res.run(st);  // skipped on the first pass (x = 0)
    mixed_resid(p->d_b, p->d_vout, p->d_r, N, c, st);
    norm2(p->d_r, N, &p->d_st->aux[0], p->d_st, st);
    mixed_ctl(c, p->d_st, p->d_st32, ho, hi, st);
    cg_init<double, float>(p->d_r, p->f_d, p->f_r, p->f_p, N, p->d_st32, st, &p->d_st->aux[0], &c->stop);
    if (cont)
      cg_project<float>(p->f_S, p->f_Q, p->f_r, p->f_d, p->f_p, N, p->cap32, p->d_st32, p->d_part2, p->d_coef,
                        p->d_eta32, st);
    cudaStreamCaptureStatus cs;
    GPFVM_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
    tail.assign(deps, deps + ndeps);
    cudaGraph_t out;
    cg.active = false;
    GPFVM_CUDA(cudaStreamEndCapture(st, &out));
  }
  // the inner CG run: a nested WHILE node after segment A
  cudaGraphNodeParams ip{};
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hi;
  ip.conditional.type = cudaGraphCondTypeWhile;
  ip.conditional.size = 1;
  cudaGraphNode_t wi;
  GPFVM_CUDA(cudaGraphAddNode(&wi, body, tail.data(), nullptr, tail.size(), &ip));
  cudaGraph_t ibody = ip.conditional.phGraph_out[0];
  const long long mid = g_launches.load();
  GPFVM_CUDA(cudaStreamBeginCaptureToGraph(st2, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  {
    CaptureGuard cg{st2};
    for (int u = 0; u < unroll; ++u) cg_iteration32(p, want_var, reorth, st2);
    loop_ctl(p->d_st32, hi, st2);
    cudaGraph_t out;
    cg.active = false;
    GPFVM_CUDA(cudaStreamEndCapture(st2, &out));
  }
  *k_inner = g_launches.load() - mid;
  // segment B: bookkeeping and the correction, after the inner loop
  const long long mid2 = g_launches.load();
  GPFVM_CUDA(cudaStreamBeginCaptureToGraph(st, body, &wi, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  {
    CaptureGuard cg{st};
    mixed_post(c, p->d_st32, p->d_x, p->f_d, N, ho, st);
    cudaGraph_t out;
    cg.active = false;
    GPFVM_CUDA(cudaStreamEndCapture(st, &out));
  }
  *k_outer = (mid - before) + (g_launches.load() - mid2);
  g_launches.fetch_sub(g_launches.load() - before);
}

// Host-side set-up of one problem's device-driven solve (enqueued on st).
int graph_begin(gpfvm_problem* p, const gpfvm_solve_opts* o, cudaStream_t st) {
  if (!p->assembled) return GPFVM_ERR_STATE;
  if (!o || o->max_iter < 1 || !(o->rtol >= 0) || o->reorth < 0 || o->reorth > 2) return GPFVM_ERR_INVALID_ARG;
  if (o->precision == GPFVM_FP64) {
    const int b = solve_begin(p, o, st);  // stores, scalar header, x = 0, r = p = b
    if (b != GPFVM_OK) return b;
    runs()[p].launched = o->max_iter;  // the graph is launched by the batch
    return GPFVM_OK;
  }
  if (o->precision < GPFVM_MIXED_FP32 || o->precision > GPFVM_MIXED_BF16) return GPFVM_ERR_INVALID_ARG;
  if (o->coarse > 1) return GPFVM_ERR_INVALID_ARG;  // the multigrid start is an FP64-path option
  if (o->reorth == 1 && o->max_iter > p->cap) return GPFVM_ERR_INVALID_ARG;
  const int want_tc = o->precision == GPFVM_MIXED_TF32X3 ? TC_TF32X3
                      : o->precision == GPFVM_MIXED_BF16X3 ? TC_BF16X3
                      : o->precision == GPFVM_MIXED_BF16  ? TC_BF16
                                                          : -1;
  if (want_tc >= 0 && !p->tc_ok) return GPFVM_ERR_INVALID_ARG;
  if (want_tc != p->tc_mode) {
    p->tc_mode = want_tc;
    if (p->graph32) cudaGraphExecDestroy(p->graph32);
    p->graph32 = nullptr;
    p->graph32_key = -1;
  }
  const int icap = std::min(p->cap, o->inner_max_iter > 0 ? o->inner_max_iter : p->cap);
  ensure_store32(p, o->reorth == 1 ? std::min(o->max_iter, p->cap) : icap);
  MixedCtl& h = *p->h_mctl;
  std::memset(&h, 0, sizeof(MixedCtl));
  h.rtol = o->rtol;
  h.itol = o->inner_rtol > 0 ? o->inner_rtol : 1e-2;
  h.max_iter = o->max_iter;
  h.icap_opt = icap;
  h.cap32 = p->cap32;
  h.cont = o->reorth == 1;
  h.want_var = o->want_var != 0;
  h.max_outer = o->max_iter + 4;
  h.rel = h.rel_prev = 1.0;
  h.tscale = 1.0;
  h.first = 1;
  GPFVM_CUDA(cudaMemcpyAsync(p->d_mctl, &h, sizeof(MixedCtl), cudaMemcpyHostToDevice, st));
  GPFVM_CUDA(cudaMemsetAsync(&p->d_st->status, 0, sizeof(int), st));
  GPFVM_CUDA(cudaMemsetAsync(&p->d_st32->pad[1], 0, sizeof(int), st));
  GPFVM_CUDA(cudaMemsetAsync(p->d_x, 0, sizeof(double) * p->N, st));
  if (o->want_var) GPFVM_CUDA(cudaMemsetAsync(p->d_down, 0, sizeof(double) * p->P, st));
  norm2(p->d_b, p->N, &p->d_st->aux[1], p->d_st, st);
  return GPFVM_OK;
}

// Reads the final state of one problem's device-driven solve.
int graph_end(gpfvm_problem* p, const gpfvm_solve_opts* o, gpfvm_solve_info* info, long long k_outer,
              long long k_inner, cudaStream_t st) {
  if (o->precision == GPFVM_FP64) {
    copy_header_to_host(p, st);
    GPFVM_CUDA(cudaStreamSynchronize(st));
    p->graph_kernels = k_inner;
    return solve_end(p, info, st);
  }
  GPFVM_CUDA(cudaMemcpyAsync(p->h_mctl, p->d_mctl, sizeof(MixedCtl), cudaMemcpyDeviceToHost, st));
  GPFVM_CUDA(cudaStreamSynchronize(st));
  const MixedCtl& h = *p->h_mctl;
  count_launch((long long)(h.outer + 1) * k_outer + h.inner_passes * k_inner);
  int status = h.stop ? h.status : GPFVM_NOT_CONVERGED;
  gpfvm_solve_info I = p->last;
  I.iterations = h.total;
  I.status = status;
  I.rel_residual = h.rel;
  I.true_rel_residual = h.rel;
  I.t_solve_ms = 0.0;
  p->last = I;
  p->last_outer = h.outer;
  if (info) *info = I;
  p->solved = status >= 0;
  p->want_var_last = o->want_var != 0;
  p->last_store = o->reorth == 1 ? 2 : 0;
  p->last_kstore = o->reorth == 1 ? h.kstore : 0;
  return status;
}

}  // namespace

extern "C" int gpfvm_solve_batch_graph(gpfvm_problem** ps, int n, const gpfvm_solve_opts* opts,
                                       gpfvm_solve_info* infos, void* stream, int64_t* launches_out) {
  if (!ps || n < 0 || !opts) return GPFVM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!ps[i] || ps[i]->multi) return GPFVM_ERR_INVALID_ARG;  // (systems: one at a time)
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (ps[i] == ps[j]) return GPFVM_ERR_INVALID_ARG;  // one loop per problem
  GPFVM_GUARD_BEGIN
  // set-up and launch on a stream of our own (capture is not possible on the
  // legacy default stream), ordered after the caller's stream
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  GPFVM_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  struct StreamOwner {
    cudaStream_t s;
    cudaEvent_t& e;
    ~StreamOwner() {
      if (e) cudaEventDestroy(e);
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } owner{st, ev};
  GPFVM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  GPFVM_CUDA(cudaEventRecord(ev, (cudaStream_t)stream));
  GPFVM_CUDA(cudaStreamWaitEvent(st, ev, 0));
  std::vector<int> ok(n, 0);
  int worst = GPFVM_OK;
  for (int i = 0; i < n; ++i) {
    const int b = graph_begin(ps[i], opts, st);
    ok[i] = b == GPFVM_OK;
    if (!ok[i]) {
      worst = std::min(worst, b);
      if (infos) infos[i].status = b;
    }
  }
  cudaStream_t cap_st = nullptr, cap_st2 = nullptr;
  GPFVM_CUDA(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
  if (cudaStreamCreateWithFlags(&cap_st2, cudaStreamNonBlocking) != cudaSuccess) {
    cudaStreamDestroy(cap_st);
    throw CudaError{cudaErrorUnknown, "stream"};
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  std::vector<long long> ko(n, 0), ki(n, 0);
  const long long l0 = g_launches.load();
  try {
    GPFVM_CUDA(cudaGraphCreate(&g, 0));
    for (int i = 0; i < n; ++i)
      if (ok[i]) add_solve_loop(ps[i], opts, g, cap_st, cap_st2, &ko[i], &ki[i]);
    GPFVM_CUDA(cudaGraphInstantiate(&ex, g, 0));
    GPFVM_CUDA(cudaGraphLaunch(ex, st));  // the whole batch
    GPFVM_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    if (ex) cudaGraphExecDestroy(ex);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap_st);
    cudaStreamDestroy(cap_st2);
    throw;
  }
  cudaGraphExecDestroy(ex);
  cudaGraphDestroy(g);
  cudaStreamDestroy(cap_st);
  cudaStreamDestroy(cap_st2);
  for (int i = 0; i < n; ++i) {
    if (!ok[i]) continue;
    const int r = graph_end(ps[i], opts, infos ? &infos[i] : nullptr, ko[i], ki[i], st);
    if (r < 0) worst = std::min(worst, r);
    else if (r == GPFVM_NOT_CONVERGED && worst == GPFVM_OK) worst = r;
  }
  if (launches_out) *launches_out = g_launches.load() - l0;
  return worst;
  GPFVM_GUARD_END
}

// ---------------------------------------------------------------------------
// Serving loop with continuous batching.
// ---------------------------------------------------------------------------
namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t ticket = 0;
  gpfvm_desc desc{};
  std::vector<std::vector<double>> store;  // owned copies of every descriptor array
  gpfvm_problem* p = nullptr;
  int state = 0;  // 0 queued, 1 running, 2 done
  bool pending = false;  // work enqueued on the request's stream and not yet polled
  int code = 0;
  std::vector<double> mean, var;
  gpfvm_solve_info info{};
  double t_submit = 0;
};

const double* own_copy(Request& R, const double* src, i64 n) {
  if (!src) return nullptr;
  R.store.emplace_back(src, src + n);
  return R.store.back().data();
}

}  // namespace

struct gpfvm_server {
  gpfvm_server_opts o{};
  std::deque<Request*> queue;
  std::vector<Request*> running;
  std::map<int64_t, std::unique_ptr<Request>> all;
  int64_t next = 0;
  int64_t used = 0, budget = 0;
};

extern "C" int gpfvm_server_create(const gpfvm_server_opts* o, gpfvm_server** out) {
  if (!o || !out || o->max_slots < 1 || o->steps_per_tick < 1 || o->solve.max_iter < 1) return GPFVM_ERR_INVALID_ARG;
  GPFVM_GUARD_BEGIN
  auto* s = new gpfvm_server();
  s->o = *o;
  s->budget = o->memory_budget;
  if (s->budget <= 0) {
    size_t fr = 0, tot = 0;
    GPFVM_CUDA(cudaMemGetInfo(&fr, &tot));
    s->budget = (int64_t)(0.9 * (double)fr);
  }
  *out = s;
  return GPFVM_OK;
  GPFVM_GUARD_END
}

extern "C" int gpfvm_server_submit(gpfvm_server* s, const gpfvm_desc* d, int64_t* ticket) {
  if (!s || !d || !ticket) return GPFVM_ERR_INVALID_ARG;
  const int v = validate(d);
  if (v != GPFVM_OK) return v;
  if (d->n_outputs > 0) {  // (systems: one at a time, FP64)
    for (int k = 0; k < d->n_terms; ++k)
      if (d->term_eq[k] != 0 || d->term_out[k] != 0) return GPFVM_ERR_INVALID_ARG;
    if (d->n_outputs > 1) return GPFVM_ERR_INVALID_ARG;
  }
  auto R = std::make_unique<Request>();
  R->desc = *d;
  R->store.reserve(4 + 3 * GPFVM_MAX_SETS + 8);
  i64 N = 1;
  for (int i = 0; i < d->ndim; ++i) {
    R->desc.edges[i] = own_copy(*R, d->edges[i], d->n_cells[i] + 1);
    R->desc.pred[i] = own_copy(*R, d->pred[i], d->n_pred[i]);
    N *= d->n_cells[i];
  }
  R->desc.rhs = own_copy(*R, d->rhs, N);
  for (int k = 0; k < d->n_sets; ++k) {
    i64 n = 1;
    for (int i = 0; i < d->ndim; ++i) {
      R->desc.sets[k].coords[i] = own_copy(*R, d->sets[k].coords[i], d->sets[k].n_pts[i]);
      n *= d->sets[k].n_pts[i];
    }
    R->desc.sets[k].values = own_copy(*R, d->sets[k].values, n);
  }
  R->ticket = s->next++;
  R->t_submit = now_ms();
  *ticket = R->ticket;
  s->queue.push_back(R.get());
  s->all[R->ticket] = std::move(R);
  return GPFVM_OK;
}

static void finish_request(gpfvm_server* s, Request* R, int code) {
  R->code = code;
  R->state = 2;
  R->info.latency_ms = now_ms() - R->t_submit;
  if (R->p) {
    s->used -= R->p->mem.bytes;
    gpfvm_destroy(R->p);
    R->p = nullptr;
  }
}

extern "C" int gpfvm_server_step(gpfvm_server* s) {
  if (!s) return GPFVM_ERR_INVALID_ARG;
  GPFVM_GUARD_BEGIN
  // admit queued requests while slots and memory allow (FIFO)
  while (!s->queue.empty() && (int)s->running.size() < s->o.max_slots) {
    Request* R = s->queue.front();
    gpfvm_problem* p = nullptr;
    int r = gpfvm_create(&R->desc, s->o.solve.max_iter, &p);
    // admission counts the direction stores the solve will allocate
    i64 store = 0;
    if (r == GPFVM_OK) {
      const gpfvm_solve_opts& so = s->o.solve;
      const i64 ld = store_ld(p->N);
      if (so.precision == GPFVM_FP64) store = so.reorth ? 16LL * ld * std::min(so.max_iter, p->cap) : 0;
      else if (so.reorth == 1) store = 8LL * ld * std::min(so.max_iter, p->cap);  // every run's directions
      else store = 8LL * ld * std::min(p->cap, so.inner_max_iter > 0 ? so.inner_max_iter : p->cap);
    }
    if (r == GPFVM_ERR_OUT_OF_MEMORY || (r == GPFVM_OK && s->used + p->mem.bytes + store > s->budget)) {
      if (p) gpfvm_destroy(p);
      if (s->running.empty()) {  // can never fit: fail it rather than stall the queue
        s->queue.pop_front();
        finish_request(s, R, GPFVM_ERR_OUT_OF_MEMORY);
        continue;
      }
      break;
    }
    s->queue.pop_front();
    if (r != GPFVM_OK) {
      finish_request(s, R, r);
      continue;
    }
    R->p = p;
    cudaStream_t st = pick_stream(p, nullptr);
    r = run_assemble(p, st);
    if (r == GPFVM_OK) r = any_begin(p, &s->o.solve, st);
    s->used += p->mem.bytes;
    if (r != GPFVM_OK) {
      finish_request(s, R, r);
      continue;
    }
    R->state = 1;
    s->running.push_back(R);
  }
  // advance every resident request whose stream is idle; the device-side
  // loops of the others keep running meanwhile
  bool progressed = false;
  std::vector<Request*> still;
  for (Request* R : s->running) {
    cudaStream_t st = pick_stream(R->p, nullptr);
    if (!R->pending) {
      any_launch(R->p, &s->o.solve, 0, st);
      R->pending = true;
    }
    const cudaError_t q = cudaStreamQuery(st);
    if (q == cudaErrorNotReady) {
      still.push_back(R);
      continue;
    }
    GPFVM_CUDA(q);
    R->pending = false;
    progressed = true;
    if (!any_poll_finished(R->p, &s->o.solve, st)) {
      still.push_back(R);
      continue;
    }
    int r = any_end(R->p, &s->o.solve, &R->info, st);
    if (r >= 0) {
      R->mean.resize(R->p->P);
      if (s->o.solve.want_var) R->var.resize(R->p->P);
      const int q2 = run_query(R->p, R->p->d_mean, s->o.solve.want_var ? R->p->d_var : nullptr, st);
      if (q2 == GPFVM_OK) {
        GPFVM_CUDA(cudaMemcpyAsync(R->mean.data(), R->p->d_mean, sizeof(double) * R->p->P, cudaMemcpyDeviceToHost, st));
        if (s->o.solve.want_var)
          GPFVM_CUDA(cudaMemcpyAsync(R->var.data(), R->p->d_var, sizeof(double) * R->p->P, cudaMemcpyDeviceToHost, st));
        GPFVM_CUDA(cudaStreamSynchronize(st));
      } else {
        r = q2;
      }
    }
    finish_request(s, R, r);
  }
  if (!progressed && !still.empty()) std::this_thread::sleep_for(std::chrono::microseconds(50));
  s->running.swap(still);
  return (int)(s->queue.size() + s->running.size());
  GPFVM_GUARD_END
}

extern "C" int gpfvm_server_poll(gpfvm_server* s, int64_t ticket, double* mean, double* var, gpfvm_solve_info* info) {
  if (!s) return GPFVM_ERR_INVALID_ARG;
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return GPFVM_ERR_NOT_FOUND;
  Request* R = it->second.get();
  if (R->state != 2) return 2;
  if (info) *info = R->info;
  if (R->code >= 0) {
    if (mean) std::memcpy(mean, R->mean.data(), R->mean.size() * sizeof(double));
    if (var && !R->var.empty()) std::memcpy(var, R->var.data(), R->var.size() * sizeof(double));
  }
  return R->code;
}

extern "C" void gpfvm_server_destroy(gpfvm_server* s) {
  if (!s) return;
  for (auto& kv : s->all)
    if (kv.second->p) gpfvm_destroy(kv.second->p);
  delete s;
}
