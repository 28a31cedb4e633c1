// Plans for Kronecker-structured products (see kron.cu).
#pragma once
#include "plan.cuh"

namespace gpfvm {

// A dense matrix view: element (i, j) at p + i*rs + j*cs.
struct MatRef {
  const double* p;
  i64 rs, cs;
};

// One term  c * (F[0] (x) F[1] (x) F[2]);  F[i] maps axis i from din[i] to dout[i].
struct KTerm {
  double c;
  MatRef f[GPFVM_MAX_DIM];
};

// A bump allocator over a device buffer for plan intermediates.
struct Scratch {
  double* base = nullptr;
  i64 cap = 0, used = 0;
  double* take(i64 n) {
    n = (n + 31) / 32 * 32;
    if (used + n > cap) throw CudaError{cudaErrorMemoryAllocation, "plan scratch exhausted"};
    double* p = base + used;
    used += n;
    return p;
  }
};

// Appends to `plan` the launches computing
//   out = scale * sum_t c_t (F_t0 (x) ... ) in  + beta*out + gamma*D
// for `batch` contiguous tensors (in: prod din, out: prod dout doubles each).
// Intermediates come from `scratch`.  n_modeprods (optional) accumulates the
// number of mode products issued.  With f32 every pointer (factors, in, out,
// D) addresses float data and the GEMMs run in FP32.
void plan_kron(Plan& plan, Scratch& scratch, int d, const int* din, const int* dout, i64 batch,
               const std::vector<KTerm>& terms, double scale, const double* in, double* out, double beta,
               const double* D, double gamma, int* n_modeprods, bool f32 = false);

// Row-tile policy of the mode-product GEMMs built by plan_kron on this host
// thread: -1 = the size heuristic (default), 0/1/2 = always 64/32/16 rows
// (the autotuner's candidates).
void set_tile_policy(int policy);
int tile_policy();

}  // namespace gpfvm
