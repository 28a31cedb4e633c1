// Kernel interfaces of the GP-FVM GPU library.
#pragma once
#include "common.cuh"

namespace gpfvm {

// ---- 1D factor assembly (factors.cu) -------------------------------------
// kind 0: cell family over edges ca[0..n] with derivative order ord (0..2);
// kind 1: point family at ca[0..n) with derivative order ord (0..1).
// A point family made of two stacked sets (two points at one coordinate of
// axis 0, see SetC in api.cu) gives its point 1 the order ord2 when has2 is set.
struct FactorJob {
  int kind_a, ord_a, n_a;
  int kind_b, ord_b, n_b;
  int has2_a, ord2_a, has2_b, ord2_b;
  const double* ca;
  const double* cb;
  double ell;
  double* out;  // n_a x n_b row-major
};
void launch_factors(const FactorJob* d_jobs, int n_jobs, i64 max_entries, cudaStream_t st);

struct GbbParams {
  int M, ndim, n_sets;
  int off[GPFVM_MAX_SETS + 1];
  int dims[GPFVM_MAX_SETS][GPFVM_MAX_DIM];
  double noise[GPFVM_MAX_SETS];
  double noise2[GPFVM_MAX_SETS];  // noise of the points with axis-0 index >= 1 (stacked sets)
  int comp[GPFVM_MAX_SETS];       // output component of each set (different: uncorrelated)
  double outputscale;
  const double* fac[GPFVM_MAX_SETS][GPFVM_MAX_SETS][GPFVM_MAX_DIM];
};
void launch_gbb(const GbbParams& P, double* G, cudaStream_t st);

// ---- grouped, segmented, batched, strided FP64 GEMM (gemm64.cu) -----------
// For every group g and batch entry b:
//   C_g[b](i,j) = beta_g C_g[b](i,j) + gamma_g D_g[b](i,j)
//               + sum_{s in segs of g} alpha_s sum_kk A_s[b](i,kk) B_s[b](kk,j)
// with A(i,kk) at A + b*a_bs + i*a_rs + kk*a_cs, B(kk,j) at B + b*b_bs +
// kk*b_rs + j*b_cs, C(i,j) at C + b*c_bs + i*c_rs + j, D likewise with d_rs.
struct GemmSeg {
  const double* A;
  const double* B;
  double alpha;
};
struct GemmGroup {
  double* C;
  const double* D;
  double beta, gamma;
  int seg0, nseg;
};
enum GemmTri {
  TRI_A_LOWER = 1,  // A(i,kk) = 0 for kk > i
  TRI_A_UPPER = 2,  // A(i,kk) = 0 for kk < i
  TRI_B_UPPER = 4,  // B(kk,j) = 0 for kk > j
  TRI_B_LOWER = 8,  // B(kk,j) = 0 for kk < j
  TRI_C_LOWER = 16  // only tiles touching the lower triangle of C are computed
};
struct GemmDesc {
  int m, n, k;
  i64 a_rs, a_cs, b_rs, b_cs, c_rs, d_rs;
  i64 a_bs, b_bs, c_bs, d_bs;
  int batch, n_groups, tri, tile;  // tile: 0 = 64x64, 1 = 32x64, 2 = 16x64 (rows x cols)
  const GemmSeg* segs;
  const GemmGroup* groups;
  const int* skip;  // if non-null and *skip != 0 the launch does nothing (converged CG)
  int f32;          // 1: every A/B/C/D pointer of the launch addresses float data (FP32 FFMA)
};
void launch_gemm64(const GemmDesc& g, cudaStream_t st);

// A GEMM op inside a multi-op launch (tile grid of the op and its first tile).
struct MOp {
  GemmDesc g;
  int tiles_x, tiles_y;
  i64 tile_begin;
};
void launch_multi_gemm(const MOp* d_ops, int nops, i64 total_tiles, int f32, int bm, cudaStream_t st);

// A GEMV op inside a multi-op launch: y = alpha A x + beta z (tri as launch_gemv64).
struct MGemv {
  const void* A;
  const void* x;
  const void* z;
  void* y;
  i64 lda, row_begin;
  int m, n, tri, pad;
  double alpha, beta;
  const int* skip;
  const double* zs;  // optional per-row scale of z: y = alpha A x + beta zs .* z
};
// Warps per row of a merged multi-GEMV: split long rows until about 4096
// warps are in flight (chunks of at least 256 columns).
inline int mgemv_split(i64 rows, int maxn) {
  int S = 1;
  while (S < 4 && rows * S < 4096 && maxn / (2 * S) >= 256) S *= 2;
  return S;
}

// S warps per output row (1, 2 or 4; see mgemv_item)
void launch_multi_gemv(const MGemv* d_ops, int nops, i64 total_rows, int f32, int S, cudaStream_t st);

// y(i) = alpha * sum_{j in tri range} A(i,j) x(j) + beta y(i); A row-major lda.
// tri: 0 full, 1 lower (j <= i), 2 upper (j >= i).
void launch_gemv64(int m, int n, const double* A, i64 lda, const double* x, double* y, double alpha,
                   double beta, int tri, cudaStream_t st, const int* skip = nullptr);
// FP32 variant (float A, x, y; FP32 accumulation)
void launch_gemv32(int m, int n, const float* A, i64 lda, const float* x, float* y, float alpha, float beta, int tri,
                   cudaStream_t st, const int* skip = nullptr);
// float <-> double conversions
void convert_d2f(const double* in, float* out, i64 n, cudaStream_t st);

// ---- IC/BC stage base case (chol.cu) ---------------------------------------
// One CTA factorises an n <= 64 diagonal block: L = chol(A) and Linv = L^-1.
void launch_chol_base(const double* A, double* L, double* Linv, int n, i64 lda, int* status,
                      cudaStream_t st);

// ---- structured IC/BC stage (icbc.cu) ---------------------------------------
struct JacobiJob {
  const double* A;  // n x n symmetric PSD, row-major
  double* Q;        // n x n eigenvectors (columns), row-major
  double* lam;      // n eigenvalues
  int n;
  double tol;
  int* sweeps;      // out: sweeps of the FP32 and of the FP64 phase (may be null)
};
void launch_jacobi(const JacobiJob* d_jobs, int n_jobs, int max_n, cudaStream_t st);
// lt[i0, i1, i2] = s2 l0[i0] l1[i1] l2[i2] + noise, the noise of eigenvector
// i0 of axis 0 being nu, or with q0 (the n0 = 2 eigenvectors of a stacked
// axis 0, row-major) nu q0[0][i0]^2 + nu_b q0[1][i0]^2
void lambda_tensor(const double* l0, const double* l1, const double* l2, int n0, int n1, int n2, double s2, double nu,
                   const double* q0, double nu_b, double* lt, cudaStream_t st);
// One launch of a merged table of face-set ops (face.cuh): kind 0 ContrOp,
// 1 BilOp, 2 ExpAddOp; `items` CTAs in total, `smem` dynamic shared bytes.
void launch_face(int kind, const void* table, int nops, i64 items, int f32, int smem, cudaStream_t st);
void recip(const double* lt, double* out, i64 n, cudaStream_t st);
// Sets 1.. of the structured IC/BC stage (row offsets relative to the first
// of them, dims, and per axis C_i = F_i(s, 0) Q_i, null for a missing axis)
struct EtildeSets {
  int ns;
  int off[GPFVM_MAX_SETS];
  int n[GPFVM_MAX_SETS][3];
  const double* c[GPFVM_MAX_SETS][3];
};
// Et (MR x MK) = sigma^2 (x)_i C_i[s] rows, times ltinv per column (k_etilde)
void etilde(const EtildeSets& S, int nk0, int nk1, int nk2, double s2, const double* ltinv, double* Et, int MR,
            cudaStream_t st);
// D[r ldd + c] += alpha S[r lds + c]
void axpy_block(double* D, i64 ldd, const double* S, i64 lds, int rows, int cols, double alpha, cudaStream_t st);
void square(const double* in, double* out, i64 n, cudaStream_t st);

}  // namespace gpfvm
