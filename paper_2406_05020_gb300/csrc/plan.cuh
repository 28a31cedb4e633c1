// A "plan" is a fixed sequence of kernel launches whose argument tables live
// in device memory.  Plans are built once per problem (at create/assemble)
// and replayed every CG iteration, so they can be captured in CUDA graphs.
#pragma once
#include <functional>

#include "kernels.cuh"

namespace gpfvm {

struct PlanOp {
  enum Kind { GEMM, GEMV, GEMV32, FUNC } kind;
  GemmDesc g;
  int seg0 = 0, group0 = 0;
  // GEMV
  int m = 0, n = 0, tri = 0;
  const double* A = nullptr;
  i64 lda = 0;
  const double* x = nullptr;
  double* y = nullptr;
  double alpha = 1.0, beta = 0.0;
  std::function<void(cudaStream_t)> fn;
};

class Plan {
 public:
  std::vector<GemmSeg> segs;
  std::vector<GemmGroup> groups;
  std::vector<PlanOp> ops;
  GemmSeg* d_segs = nullptr;
  GemmGroup* d_groups = nullptr;
  const int* skip = nullptr;  // device flag: when set, every GEMM/GEMV of the plan is a no-op

  ~Plan() { release(); }
  void release() {
    if (d_segs) cudaFree(d_segs);
    if (d_groups) cudaFree(d_groups);
    d_segs = nullptr;
    d_groups = nullptr;
  }
  // Adds a GEMM; `gs` lists the groups, each with its segments.
  void gemm(GemmDesc g, const std::vector<std::pair<GemmGroup, std::vector<GemmSeg>>>& gs) {
    PlanOp op;
    op.kind = PlanOp::GEMM;
    op.group0 = (int)groups.size();
    for (auto& pr : gs) {
      GemmGroup G = pr.first;
      G.seg0 = (int)segs.size();
      G.nseg = (int)pr.second.size();
      for (auto& s : pr.second) segs.push_back(s);
      groups.push_back(G);
    }
    g.n_groups = (int)gs.size();
    op.g = g;
    ops.push_back(op);
  }
  void gemv(int m, int n, const double* A, i64 lda, const double* x, double* y, double alpha,
            double beta, int tri) {
    PlanOp op;
    op.kind = PlanOp::GEMV;
    op.m = m; op.n = n; op.A = A; op.lda = lda; op.x = x; op.y = y;
    op.alpha = alpha; op.beta = beta; op.tri = tri;
    ops.push_back(op);
  }
  void gemv32(int m, int n, const float* A, i64 lda, const float* x, float* y, int tri, double alpha = 1.0,
              double beta = 0.0) {
    PlanOp op;
    op.kind = PlanOp::GEMV32;
    op.m = m; op.n = n; op.A = (const double*)A; op.lda = lda; op.x = (const double*)x; op.y = (double*)y;
    op.alpha = alpha; op.beta = beta; op.tri = tri;
    ops.push_back(op);
  }
  void func(std::function<void(cudaStream_t)> f) {
    PlanOp op;
    op.kind = PlanOp::FUNC;
    op.fn = std::move(f);
    ops.push_back(op);
  }
  void append(const Plan& o) {
    const int s0 = (int)segs.size(), g0 = (int)groups.size();
    for (auto s : o.segs) segs.push_back(s);
    for (auto G : o.groups) { G.seg0 += s0; groups.push_back(G); }
    for (auto op : o.ops) { op.group0 += g0; ops.push_back(op); }
  }
  void finalize() {
    release();
    if (!segs.empty()) {
      GPFVM_CUDA(cudaMalloc(&d_segs, segs.size() * sizeof(GemmSeg)));
      GPFVM_CUDA(cudaMemcpy(d_segs, segs.data(), segs.size() * sizeof(GemmSeg), cudaMemcpyHostToDevice));
    }
    if (!groups.empty()) {
      GPFVM_CUDA(cudaMalloc(&d_groups, groups.size() * sizeof(GemmGroup)));
      GPFVM_CUDA(cudaMemcpy(d_groups, groups.data(), groups.size() * sizeof(GemmGroup),
                            cudaMemcpyHostToDevice));
    }
    for (auto& op : ops)
      if (op.kind == PlanOp::GEMM) {
        op.g.segs = d_segs;
        op.g.groups = d_groups + op.group0;
        op.g.skip = skip;
      }
  }
  void run(cudaStream_t st) const {
    for (auto& op : ops) {
      if (op.kind == PlanOp::GEMM) launch_gemm64(op.g, st);
      else if (op.kind == PlanOp::GEMV)
        launch_gemv64(op.m, op.n, op.A, op.lda, op.x, op.y, op.alpha, op.beta, op.tri, st, skip);
      else if (op.kind == PlanOp::GEMV32)
        launch_gemv32(op.m, op.n, (const float*)op.A, op.lda, (const float*)op.x, (float*)op.y, (float)op.alpha,
                      (float)op.beta, op.tri, st, skip);
      else op.fn(st);
    }
  }
  int launches() const { return (int)ops.size(); }
};

// Builds the recursive Cholesky + inverse of an n x n SPD matrix A (lower
// triangle read, lda) into L and Linv (lower, row-major, lda); scratch must
// hold n*n/4 + 64 doubles.  status receives DEV_NOT_SPD on a pivot <= 0.
void plan_chol_inverse(Plan& plan, double* A, double* L, double* Linv, int n, i64 lda,
                       double* scratch, int* status);

}  // namespace gpfvm
