// Tensor-core (tcgen05) mode products, see tc.cu.
#pragma once
#include "kernels.cuh"

namespace gpfvm {

constexpr int TC_MAXSEG = 16;

// Operand formats of a tensor-core mode product (every operand x is split as
// x = hi + lo):
//   TC_TF32X3  hi = tf32(x), lo = x - hi; kind::tf32, hi*hi + hi*lo + lo*hi
//   TC_BF16X3  hi = bf16(x), lo = bf16(x - hi); kind::f16 (bf16), the same three products
//   TC_BF16    hi = bf16(x); kind::f16 (bf16), hi*hi only
enum TcMode { TC_TF32X3 = 0, TC_BF16X3 = 1, TC_BF16 = 2 };

// out[j * R + r] = sum_s sum_k A_s[r * K + k] * (Bhi_s + Blo_s)[j * K + k]
//                  (+ gamma * D[j * R + r]) (+ beta * out[j * R + r])
// A_s: R x K row-major (FP32, split on the fly); B_s: N x K row-major, already
// scaled and split into tf32 hi / FP32 lo parts.  N <= 256.
struct TcOp {
  int R, K, N, nseg;
  const float* A[TC_MAXSEG];
  const float* Bhi[TC_MAXSEG];
  const float* Blo[TC_MAXSEG];
  float* out;
  const float* D;
  float gamma, beta;
  i64 tile_begin;   // first tile of this op in the launch
  const int* skip;  // op does nothing if *skip
  // Segment groups: with sgroups > 1 the segments are split into sgroups
  // contiguous groups, one tile per (128 rows, group), each writing its
  // partial sum to part + group * N * R; tc_sum then adds the groups in order
  // (and gamma D, beta out) into out.
  int sgroups;
  float* part;
  int mode;  // TcMode (uniform over the ops of one launch)
};

// Runs the tiles of one level; with any_split the partial sums of split ops
// are then reduced (a second, elementwise launch).
void launch_tc_modes(const TcOp* d_ops, int nops, i64 total_tiles, int max_n, int* status, cudaStream_t st,
                     int any_split = 0);
// hi / lo parts of alpha * F for the given TcMode (kept as FP32 values that
// are exactly representable in the mode's operand type)
void tc_split(const float* F, i64 n, float alpha, float* hi, float* lo, cudaStream_t st, int mode = TC_TF32X3);
int tc_smem_bytes(int ncols, int nbuf);

}  // namespace gpfvm
