// FP64 Kronecker mode products on the bf16 tensor cores by exact digit
// products, see oz.cu.
#pragma once
#include "kernels.cuh"

namespace gpfvm {

constexpr int OZ_MAXSEG = 16;
constexpr int OZ_DIGITS = 8;                          // balanced 7-bit digits per operand
constexpr int OZ_ROWS = 128;                          // tensor rows per tile (MMA M)
constexpr int OZ_COLS = 64;                           // output columns per tile (MMA N)
constexpr int OZ_KB = 32;                             // K per stage (bf16: 64-byte rows)
constexpr int OZ_KMAX = 128;                          // largest K of one segment (exactness bound)
constexpr int OZ_A_PLANE = OZ_ROWS * 64;              // bytes of one A digit plane of a stage
constexpr int OZ_B_PLANE = OZ_COLS * 64;              // bytes of one B digit plane of a stage
constexpr int OZ_IMG_STAGE = OZ_DIGITS * OZ_B_PLANE;  // 32 KB: B digit planes of one (K block, column half)

// out[j * R + r] = sum_s sum_k A_s[r * K + k] * B_s[j][k]  (+ gamma D[j * R + r]) (+ beta out[j * R + r])
// in FP64, with A_s an R x K row-major FP64 tensor view, Aexp_s[r] the largest
// biased exponent field of its row r (oz_row_exponents), and B_s = alpha_s F_s
// given by its digit image and per-row exponent fields (oz_split_factor).
// K <= OZ_KMAX, N <= 128.
struct OzOp {
  int R, K, N, nseg;
  const double* A[OZ_MAXSEG];
  const int* Aexp[OZ_MAXSEG];
  const unsigned char* Bimg[OZ_MAXSEG];
  const int* Bexp[OZ_MAXSEG];
  double* out;
  const double* D;
  double gamma, beta;
  i64 tile_begin;   // first tile of this op in the launch
  const int* skip;  // op does nothing if *skip
};

// Row-exponent jobs of one launch (all with the same R x K shape).
struct OzExpJobs {
  const double* A[OZ_MAXSEG];
  int* ex[OZ_MAXSEG];
  int n, R, K;
  const int* skip;
};

// bytes of the digit image of an N x K factor (zero padded to 64-row halves and 32-wide K blocks)
i64 oz_image_bytes(int N, int K);
// digit image and per-row exponent fields of alpha * F (F: N x K FP64, element
// (j, k) at F[j * rs + k * cs])
void oz_split_factor(const double* F, i64 rs, i64 cs, int N, int K, double alpha, unsigned char* img, int* fexp,
                     cudaStream_t st);
void oz_row_exponents(const OzExpJobs& jobs, cudaStream_t st);
// the tall tiling (all outputs of a tile on the MMA's M side) for 64 < N <= 128
bool oz_tall(int N);
// tiles of one op (row tiles x column halves, or row tiles of 64 when tall)
i64 oz_tiles(int R, int N);
// one level of ops, all with N outputs (the same tiling for the whole launch)
void launch_oz_modes(const OzOp* d_ops, int nops, i64 total_tiles, int n, int* status, cudaStream_t st);

// C = beta C + gamma D + alpha A B in FP64 by digit products for long K:
// A(i, kk) = A[i a_rs + kk] (m x k), B(kk, j) = B[kk b_rs + j b_cs] with
// b_rs == 1 or b_cs == 1, C(i, j) = C[i c_rs + j], D likewise with d_rs;
// tri: GemmTri flags (zero triangles of A / B are masked, TRI_C_LOWER skips
// the tiles above the diagonal).  Aexp / Bexp: device scratch of m and n
// times ceil(k / 128) ints (the per-window exponents, written here).
struct OzGemm {
  int m, n, k, nwin;
  const double* A;
  i64 a_rs;
  const double* B;
  i64 b_rs, b_cs;
  double* C;
  i64 c_rs;
  const double* D;
  i64 d_rs;
  double alpha, beta, gamma;
  int tri;
  const int* Aexp;
  const int* Bexp;
  const int* skip;
};
void oz_gemm(const OzGemm& g, int* Aexp, int* Bexp, int* status, cudaStream_t st);

}  // namespace gpfvm
