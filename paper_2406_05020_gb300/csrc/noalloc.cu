// Kronecker Gram matvec that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a Gram
// product: frameworks whose allocator owns the whole device and refuse
// foreign allocations, or real-time loops that must not enter the driver's
// allocator (a cudaMalloc can synchronise the device and take milliseconds).
// This entry point keeps the intermediates of the three-level mode-product
// chain and the GEMM argument tables in file-scope __device__ arrays instead:
// every GPU that loads the library holds them (about 32 MiB) until the
// process exits.  The argument tables reach the device as the by-value
// parameter of a small fill kernel, so no host memory is read after the call
// returns.
#include <string.h>

#include <mutex>

#include "kernels.cuh"

namespace gpfvm {

// Maximum number of doubles of intermediates (32 MiB).
constexpr long long NOALLOC_SCRATCH_DOUBLES = 4LL * 1024 * 1024;
constexpr int NOALLOC_MAX_SEGS = 256;
constexpr int NOALLOC_MAX_GROUPS = 160;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];
static __device__ __align__(256) GemmSeg g_noalloc_segs[NOALLOC_MAX_SEGS];
static __device__ __align__(256) GemmGroup g_noalloc_groups[NOALLOC_MAX_GROUPS];

struct NoallocAddrs {
  double* scratch;
  GemmSeg* segs;
  GemmGroup* groups;
};

// Device addresses of the static arrays, looked up once per device with that
// device current (a host-side reference to the array names is only a host
// stand-in, not a device address).  The lookup is serialised by a mutex, so
// host threads making their first calls at the same time are safe.
static int noalloc_setup(NoallocAddrs* out) {
  static std::mutex mu;
  static NoallocAddrs cache[NOALLOC_MAX_DEVICES];
  static bool ready[NOALLOC_MAX_DEVICES] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return GPFVM_ERR_DEVICE;
  std::lock_guard<std::mutex> lock(mu);
  if (!ready[dev]) {
    NoallocAddrs a{};
    if (cudaGetSymbolAddress((void**)&a.scratch, g_noalloc_scratch) != cudaSuccess) return GPFVM_ERR_DEVICE;
    if (cudaGetSymbolAddress((void**)&a.segs, g_noalloc_segs) != cudaSuccess) return GPFVM_ERR_DEVICE;
    if (cudaGetSymbolAddress((void**)&a.groups, g_noalloc_groups) != cudaSuccess) return GPFVM_ERR_DEVICE;
    cache[dev] = a;
    ready[dev] = true;
  }
  *out = cache[dev];
  return GPFVM_OK;
}

// The GEMM argument tables of one call, passed BY VALUE as a kernel parameter
// (about 12.5 KB, within the 32 KB parameter limit): the launch copies them,
// so nothing on the host stack is read once the call has returned.
struct NoallocTables {
  int ns, ng;
  GemmSeg segs[NOALLOC_MAX_SEGS];
  GemmGroup groups[NOALLOC_MAX_GROUPS];
};
static_assert(sizeof(NoallocTables) < 32000, "kernel parameter too large");

__global__ void noalloc_fill_kernel(const NoallocTables t) {
  for (int i = threadIdx.x; i < t.ns; i += blockDim.x) g_noalloc_segs[i] = t.segs[i];
  for (int i = threadIdx.x; i < t.ng; i += blockDim.x) g_noalloc_groups[i] = t.groups[i];
}

}  // namespace gpfvm

using namespace gpfvm;

extern "C" int gpfvm_kron_matvec_noalloc(int ndim, const int* n, int n_terms, const double* const* factors,
                                         const double* coef, double scale, double diag, const double* v,
                                         double* out, void* stream) {
  if (ndim < 1 || ndim > 3 || !n || n_terms < 1 || n_terms > 64 || !factors || !coef || !v || !out)
    return GPFVM_ERR_INVALID_ARG;
  long long N = 1;
  for (int i = 0; i < ndim; ++i) {
    if (n[i] < 1 || n[i] > 65536) return GPFVM_ERR_INVALID_ARG;
    N *= n[i];
  }
  for (int k = 0; k < n_terms * ndim; ++k)
    if (!factors[k]) return GPFVM_ERR_INVALID_ARG;
  // distinct factors on the last axis (level 1, 3 axes only) and on axis 0
  int u_of[64], w_of[64], nu = 0, nw = 0;
  const double* U[64];
  const double* Wf[64];
  for (int k = 0; k < n_terms; ++k) {
    const double* fl = factors[k * ndim + ndim - 1];
    const double* f0 = factors[k * ndim + 0];
    u_of[k] = -1;
    if (ndim == 3) {
      for (int j = 0; j < nu; ++j)
        if (U[j] == fl) u_of[k] = j;
      if (u_of[k] < 0) { U[nu] = fl; u_of[k] = nu++; }
    }
    w_of[k] = -1;
    for (int j = 0; j < nw; ++j)
      if (Wf[j] == f0) w_of[k] = j;
    if (w_of[k] < 0) { Wf[nw] = f0; w_of[k] = nw++; }
  }
  const long long need = (ndim == 1) ? 0 : (long long)(nu + nw) * N;
  if (need > NOALLOC_SCRATCH_DOUBLES) return GPFVM_ERR_TOO_LARGE;
  NoallocAddrs A;
  const int st_ok = noalloc_setup(&A);
  if (st_ok != GPFVM_OK) return st_ok;
  cudaStream_t st = (cudaStream_t)stream;

  static thread_local NoallocTables tab;  // large: kept off the stack
  memset(&tab, 0, sizeof(tab));
  GemmSeg* segs = tab.segs;
  GemmGroup* groups = tab.groups;
  int ns = 0, ng = 0;
  GemmDesc L[3];
  int nl = 0;
  double* Y = A.scratch;
  double* Z = A.scratch + (long long)nu * N;
  try {
    if (ndim == 1) {
      GemmDesc g{};
      g.m = 1; g.n = n[0]; g.k = n[0];
      g.a_rs = n[0]; g.a_cs = 1; g.b_rs = 1; g.b_cs = n[0]; g.c_rs = n[0]; g.d_rs = n[0];
      g.batch = 1; g.tile = 2;
      g.groups = A.groups + ng; g.segs = A.segs;
      groups[ng] = GemmGroup{out, v, 0.0, diag, ns, n_terms};
      for (int k = 0; k < n_terms; ++k) segs[ns++] = GemmSeg{v, factors[k], scale * coef[k]};
      g.n_groups = 1;
      ++ng;
      L[nl++] = g;
    } else {
      const int n0 = n[0], n1 = n[1], n2 = (ndim == 3) ? n[2] : 1;
      if (ndim == 3) {
        // level 1: Y[u] = v x_2 U[u]  (right multiplication, rows = n0*n1)
        GemmDesc g{};
        g.m = n0 * n1; g.n = n2; g.k = n2;
        g.a_rs = n2; g.a_cs = 1; g.b_rs = 1; g.b_cs = n2; g.c_rs = n2; g.d_rs = n2;
        g.batch = 1; g.tile = 0;
        g.groups = A.groups + ng; g.segs = A.segs; g.n_groups = nu;
        for (int j = 0; j < nu; ++j) {
          groups[ng++] = GemmGroup{Y + (long long)j * N, nullptr, 0.0, 0.0, ns, 1};
          segs[ns++] = GemmSeg{v, U[j], 1.0};
        }
        L[nl++] = g;
        // level 2: Z[w] = sum_k coef_k Y[u_k] x_1 F_k1 (left multiplication, batch over axis 0)
        GemmDesc h{};
        h.m = n1; h.n = n2; h.k = n1;
        h.a_rs = n1; h.a_cs = 1; h.b_rs = n2; h.b_cs = 1; h.b_bs = (long long)n1 * n2;
        h.c_rs = n2; h.c_bs = (long long)n1 * n2; h.d_rs = n2;
        h.batch = n0; h.tile = 0;
        h.groups = A.groups + ng; h.segs = A.segs; h.n_groups = nw;
        for (int j = 0; j < nw; ++j) {
          const int s0 = ns;
          for (int k = 0; k < n_terms; ++k)
            if (w_of[k] == j) segs[ns++] = GemmSeg{factors[k * ndim + 1], Y + (long long)u_of[k] * N, coef[k]};
          groups[ng++] = GemmGroup{Z + (long long)j * N, nullptr, 0.0, 0.0, s0, ns - s0};
        }
        L[nl++] = h;
      } else {
        // 2 axes: Z[w] = sum_k coef_k v x_1 F_k1 (right multiplication)
        GemmDesc h{};
        h.m = n0; h.n = n1; h.k = n1;
        h.a_rs = n1; h.a_cs = 1; h.b_rs = 1; h.b_cs = n1; h.c_rs = n1; h.d_rs = n1;
        h.batch = 1; h.tile = 2;
        h.groups = A.groups + ng; h.segs = A.segs; h.n_groups = nw;
        for (int j = 0; j < nw; ++j) {
          const int s0 = ns;
          for (int k = 0; k < n_terms; ++k)
            if (w_of[k] == j) segs[ns++] = GemmSeg{v, factors[k * ndim + 1], coef[k]};
          groups[ng++] = GemmGroup{Z + (long long)j * N, nullptr, 0.0, 0.0, s0, ns - s0};
        }
        L[nl++] = h;
      }
      // level 3: out = scale * sum_w W[w] x_0 Z[w] + diag * v
      const long long post = (long long)n1 * n2;
      GemmDesc g{};
      g.m = n0; g.n = (int)post; g.k = n0;
      g.a_rs = n0; g.a_cs = 1; g.b_rs = post; g.b_cs = 1; g.c_rs = post; g.d_rs = post;
      g.batch = 1; g.tile = (n0 <= 16) ? 2 : (n0 <= 32 ? 1 : 2);
      g.groups = A.groups + ng; g.segs = A.segs; g.n_groups = 1;
      groups[ng++] = GemmGroup{out, v, 0.0, diag, ns, nw};
      for (int j = 0; j < nw; ++j) segs[ns++] = GemmSeg{Wf[j], Z + (long long)j * N, scale};
      L[nl++] = g;
    }
    // argument tables into the static arrays: by-value kernel parameter, stream ordered
    tab.ns = ns;
    tab.ng = ng;
    noalloc_fill_kernel<<<1, 256, 0, st>>>(tab);
    if (cudaGetLastError() != cudaSuccess) return GPFVM_ERR_DEVICE;
    count_launch(1);
    for (int l = 0; l < nl; ++l) launch_gemm64(L[l], st);
  } catch (const CudaError&) {
    return GPFVM_ERR_DEVICE;
  }
  return GPFVM_OK;
}
