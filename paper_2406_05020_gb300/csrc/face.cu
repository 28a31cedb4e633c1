// Launches of the face-set operations (see face.cuh): one CTA per item of a
// merged table of ops.
#include "face.cuh"
#include "kernels.cuh"

namespace gpfvm {

template <typename T>
__global__ void __launch_bounds__(FACE_THREADS) contr_kernel(const ContrOp* __restrict__ ops, int nops) {
  __shared__ T red[FACE_THREADS * FACE_MAXF];
  const ContrOp& op = face_find(ops, nops, (i64)blockIdx.x);
  pdl_wait();
  if (op.skip && *op.skip) return;
  contr_item<T>(op, (i64)blockIdx.x - op.item_begin, red);
}

template <typename T>
__global__ void __launch_bounds__(FACE_THREADS) bilin_kernel(const BilOp* __restrict__ ops, int nops) {
  extern __shared__ __align__(16) unsigned char face_smem[];
  T* sm = reinterpret_cast<T*>(face_smem);
  const BilOp& op = face_find(ops, nops, (i64)blockIdx.x);
  pdl_wait();
  if (op.skip && *op.skip) return;
  bilin_item<T>(op, (i64)blockIdx.x - op.item_begin, sm);
}

template <typename T>
__global__ void __launch_bounds__(FACE_THREADS) expadd_kernel(const ExpAddOp* __restrict__ ops, int nops) {
  const ExpAddOp& op = face_find(ops, nops, (i64)blockIdx.x);
  pdl_wait();
  if (op.skip && *op.skip) return;
  expadd_item<T>(op, (i64)blockIdx.x - op.item_begin);
}

void launch_face(int kind, const void* table, int nops, i64 items, int f32, int smem, cudaStream_t st) {
  if (nops <= 0 || items <= 0) return;
  const int grid = (int)items;
  static bool attr = false;
  if (!attr) {
    GPFVM_CUDA(cudaFuncSetAttribute(bilin_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, FACE_SMEM_MAX));
    GPFVM_CUDA(cudaFuncSetAttribute(bilin_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, FACE_SMEM_MAX));
    attr = true;
  }
  if (kind == 0) {
    if (f32) launch_pdl(contr_kernel<float>, grid, FACE_THREADS, 0, st, (const ContrOp*)table, nops);
    else launch_pdl(contr_kernel<double>, grid, FACE_THREADS, 0, st, (const ContrOp*)table, nops);
  } else if (kind == 1) {
    if (f32) launch_pdl(bilin_kernel<float>, grid, FACE_THREADS, smem, st, (const BilOp*)table, nops);
    else launch_pdl(bilin_kernel<double>, grid, FACE_THREADS, smem, st, (const BilOp*)table, nops);
  } else {
    if (f32) launch_pdl(expadd_kernel<float>, grid, FACE_THREADS, 0, st, (const ExpAddOp*)table, nops);
    else launch_pdl(expadd_kernel<double>, grid, FACE_THREADS, 0, st, (const ExpAddOp*)table, nops);
  }
}

}  // namespace gpfvm
