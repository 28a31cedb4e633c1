// IC/BC stage of the Cholesky deflation (Sec. 4.2): G_BB = L L^T and the
// explicit inverse factor L^-1, so that every CG iteration applies
// G_BB^-1 = L^-T L^-1 with two parallel triangular GEMVs instead of two
// sequential triangular solves.
//
// Recursive 2x2 block form (all blocks aligned to 64):
//   L11, L11^-1 = chol_inv(A11)
//   L21 = A21 L11^-T
//   A22 <- A22 - L21 L21^T                     (lower tiles only)
//   L22, L22^-1 = chol_inv(A22)
//   (L^-1)21 = -L22^-1 (L21 L11^-1)
// The base case (n <= 64) runs in one CTA from shared memory.
#include "oz.cuh"
#include "plan.cuh"

namespace gpfvm {

__global__ void __launch_bounds__(256) chol_base_kernel(const double* __restrict__ A, double* __restrict__ L,
                                                        double* __restrict__ Linv, int n, i64 lda,
                                                        int* status) {
  extern __shared__ double sm[];
  constexpr int LD = 65;
  double* Ls = sm;            // 64 x 65
  double* Xs = sm + 64 * LD;  // 64 x 65
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) bad = 0;
  for (int e = tid; e < 64 * 64; e += blockDim.x) {
    const int i = e / 64, j = e % 64;
    Ls[i * LD + j] = (i < n && j <= i) ? A[(i64)i * lda + j] : 0.0;
    Xs[i * LD + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // Right-looking Cholesky; X = L^-1 is eliminated alongside: X starts as I,
  // and once column j of L is final, row j of X is divided by L[j][j] and
  // X[i][c] -= L[i][j] X[j][c] for the rows i > j (columns c <= j; X stays
  // lower triangular).  Rows go to warps, columns to lanes.
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double d = Ls[j * LD + j];
      if (!(d > 0.0)) {
        bad = 1;
        Ls[j * LD + j] = 1.0;
      } else {
        Ls[j * LD + j] = sqrt(d);
      }
    }
    __syncthreads();
    const double piv = Ls[j * LD + j];
    for (int i = j + 1 + tid; i < n; i += blockDim.x) Ls[i * LD + j] /= piv;
    for (int c = tid; c <= j; c += blockDim.x) Xs[j * LD + c] /= piv;
    __syncthreads();
    for (int i = j + 1 + warp; i < n; i += nw) {
      const double lij = Ls[i * LD + j];
      for (int l = j + 1 + lane; l <= i; l += 32) Ls[i * LD + l] -= lij * Ls[l * LD + j];
      for (int c = lane; c <= j; c += 32) Xs[i * LD + c] -= lij * Xs[j * LD + c];
    }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    L[(i64)i * lda + j] = (j <= i) ? Ls[i * LD + j] : 0.0;
    Linv[(i64)i * lda + j] = (j <= i) ? Xs[i * LD + j] : 0.0;
  }
  if (tid == 0 && bad) atomicOr(status, (int)DEV_NOT_SPD);
}

void launch_chol_base(const double* A, double* L, double* Linv, int n, i64 lda, int* status,
                      cudaStream_t st) {
  const int smem = 2 * 64 * 65 * (int)sizeof(double);
  static bool attr = false;
  if (!attr) {
    GPFVM_CUDA(cudaFuncSetAttribute(chol_base_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = true;
  }
  chol_base_kernel<<<1, 256, smem, st>>>(A, L, Linv, n, lda, status);
  GPFVM_LAUNCH_CHECK();
}

// Row tile for a dense FP64 GEMM: the FP64 pipe needs several CTAs per SM, so
// take the tallest tile that still gives about two CTAs for each of the 152 SMs.
int dense_tile(int m, int n) {
  const i64 cols = (n + 63) / 64;
  if ((i64)((m + 63) / 64) * cols >= 304) return 0;
  if ((i64)((m + 31) / 32) * cols >= 304) return 1;
  return 2;
}

static GemmDesc gdesc(int m, int n, int k, i64 a_rs, i64 a_cs, i64 b_rs, i64 b_cs, i64 c_rs, int tri) {
  GemmDesc g{};
  g.m = m; g.n = n; g.k = k;
  g.a_rs = a_rs; g.a_cs = a_cs; g.b_rs = b_rs; g.b_cs = b_cs; g.c_rs = c_rs; g.d_rs = 0;
  g.batch = 1; g.tri = tri; g.tile = dense_tile(m, n);
  return g;
}

// One dense FP64 GEMM (one group, one segment): digit products for the large
// ones (both sizes >= 128 and a contraction of at least 128) when `oz` is
// given, else the FP64 FMA kernel.
void plan_dense_gemm(Plan& plan, const GemmDesc& g, const GemmGroup& G, const GemmSeg& S, const OzChol* oz) {
  const i64 nwin = (g.k + OZ_KMAX - 1) / OZ_KMAX;
  if (oz && g.m >= 128 && g.n >= 128 && g.k >= 128 && g.a_cs == 1 && (g.b_rs == 1 || g.b_cs == 1) &&
      (i64)g.m * nwin <= oz->cap && (i64)g.n * nwin <= oz->cap) {
    OzGemm o{};
    o.m = g.m; o.n = g.n; o.k = g.k;
    o.A = S.A; o.a_rs = g.a_rs;
    o.B = S.B; o.b_rs = g.b_rs; o.b_cs = g.b_cs;
    o.C = G.C; o.c_rs = g.c_rs;
    o.D = G.D; o.d_rs = g.d_rs;
    o.alpha = S.alpha; o.beta = G.beta; o.gamma = G.gamma;
    o.tri = g.tri;
    int *ea = oz->Aexp, *eb = oz->Bexp, *st = oz->status;
    plan.func([=](cudaStream_t s) { oz_gemm(o, ea, eb, st, s); });
  } else {
    plan.gemm(g, {{G, {S}}});
  }
}

void plan_chol_inverse(Plan& plan, double* A, double* L, double* Linv, int n, i64 lda,
                       double* scratch, int* status, const OzChol* oz) {
  if (n <= 0) return;
  if (n <= 64) {
    plan.func([=](cudaStream_t st) { launch_chol_base(A, L, Linv, n, lda, status, st); });
    return;
  }
  const int nb = (n + 63) / 64;
  const int n1 = 64 * ((nb + 1) / 2);
  const int n2 = n - n1;
  double* A21 = A + (i64)n1 * lda;
  double* A22 = A21 + n1;
  double* L21 = L + (i64)n1 * lda;
  double* L22 = L21 + n1;
  double* Li21 = Linv + (i64)n1 * lda;
  double* Li22 = Li21 + n1;
  plan_chol_inverse(plan, A, L, Linv, n1, lda, scratch, status, oz);
  // L21 = A21 * Linv11^T ; B(kk, j) = Linv11[j][kk] is upper triangular in (kk, j)
  plan_dense_gemm(plan, gdesc(n2, n1, n1, lda, 1, 1, lda, lda, TRI_B_UPPER), GemmGroup{L21, nullptr, 0.0, 0.0, 0, 0},
            GemmSeg{A21, Linv, 1.0}, oz);
  // A22 -= L21 * L21^T (lower tiles)
  plan_dense_gemm(plan, gdesc(n2, n2, n1, lda, 1, 1, lda, lda, TRI_C_LOWER), GemmGroup{A22, nullptr, 1.0, 0.0, 0, 0},
            GemmSeg{L21, L21, -1.0}, oz);
  plan_chol_inverse(plan, A22, L22, Li22, n2, lda, scratch, status, oz);
  // T = L21 * Linv11 (Linv11 lower: B(kk, j) = 0 for kk < j)
  plan_dense_gemm(plan, gdesc(n2, n1, n1, lda, 1, lda, 1, n1, TRI_B_LOWER), GemmGroup{scratch, nullptr, 0.0, 0.0, 0, 0},
            GemmSeg{L21, Linv, 1.0}, oz);
  // Linv21 = -Linv22 * T (Linv22 lower: A(i, kk) = 0 for kk > i)
  plan_dense_gemm(plan, gdesc(n2, n1, n2, lda, 1, n1, 1, lda, TRI_A_LOWER), GemmGroup{Li21, nullptr, 0.0, 0.0, 0, 0},
            GemmSeg{Li22, scratch, -1.0}, oz);
}

}  // namespace gpfvm
