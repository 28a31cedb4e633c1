// Shared device/host helpers of the GP-FVM GPU library (not shared with the oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/gpfvm.h"

namespace gpfvm {

typedef long long i64;

// Status words written by device code (bounded waits, breakdown, pivots).
enum DevStatus : int {
  DEV_OK = 0,
  DEV_NOT_SPD = 1,
  DEV_BREAKDOWN = 2,
  DEV_TIMEOUT = 4,
  DEV_BADPTR = 8,
};

struct CudaError {
  cudaError_t err;
  const char* where;
};

#define GPFVM_CUDA(call)                                                   \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) throw ::gpfvm::CudaError{e_, #call};            \
  } while (0)

// Every kernel launch of the library is followed by this check, which also
// counts the launch (see gpfvm_launch_count).
void count_launch(long long n = 1);
#define GPFVM_LAUNCH_CHECK()             \
  do {                                   \
    GPFVM_CUDA(cudaGetLastError());      \
    ::gpfvm::count_launch();             \
  } while (0)

// Launch with programmatic dependent launch allowed: the grid may be scheduled
// while its stream predecessor drains.  Every kernel launched this way calls
// pdl_wait() before it touches memory that an earlier kernel writes.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  GPFVM_CUDA(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
  count_launch();
}
// Waits until the grids this one depends on have completed and their memory
// operations are visible (a no-op for a grid launched without that dependency).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }


inline int ceil_div(i64 a, i64 b) { return (int)((a + b - 1) / b); }

// Fixed-order block reduction of doubles (deterministic for a fixed blockDim).
template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* smem) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = (lane < THREADS / 32) ? smem[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

}  // namespace gpfvm
