// Persistent execution of a phased plan: one cooperative launch runs every
// phase of a structured Gram product (the zip levels of Eq. kronecker-structure
// mode products, the IC/BC products of Sec. 4.2) instead of one launch per
// phase and unit.  The CTAs (one per SM, all resident by the cooperative
// launch) take the work items of a phase grid-stride -- GEMM tiles, groups of
// GEMV rows, tensor-core tiles, element chunks -- and meet at a grid barrier
// before the next phase.  The per-item code is the same device code the
// separate kernels run (gemm_tiles.cuh, tc_tile.cuh), so results are
// bit-identical to the launch-by-launch execution.
//
// The grid barrier is a counter and a generation word in global memory; every
// wait is bounded (2^24 polls with a short sleep), after which the CTA sets
// DEV_TIMEOUT in *status and leaves, so a fault can not hang the device.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "gemm_tiles.cuh"
#include "persist.cuh"
#include <functional>

#include "face.cuh"
#include "plan.cuh"
#include "tc_tile.cuh"

namespace gpfvm {

enum PUnitKind { PU_MGEMM = 0, PU_MGEMV, PU_TC, PU_COPY, PU_GEMM, PU_GEMV, PU_TCSUM, PU_CONTR, PU_BILIN, PU_EXPADD };
constexpr int P_SUM_CHUNKS = 64;  // items per op of a segment-group reduction

constexpr int P_THREADS = 256;
constexpr int P_GEMV_ROWS = P_THREADS / 32;  // one warp per row
constexpr int P_ELEMS = 4 * P_THREADS;       // elements per COPY item

struct PUnit {
  int kind, f32, bm, nops;
  i64 items, item_begin;
  const void* table;  // MOp* / MGemv* / TcOp*
  i64 total;          // MGEMV rows
  // COPY (4-byte words)
  void* dst;
  const void* src;
  i64 words;
  // single GEMM
  GemmDesc g;
  int tiles_x, tiles_y;
  // single GEMV
  int m, n, tri;
  const void* A;
  i64 lda;
  const void* x;
  void* y;
  double alpha, beta;
  const int* skip;
};

struct PPhase {
  int unit0, nunits;
  i64 items;
};

struct PProgDev {
  const PPhase* phases;
  const PUnit* units;
  int nphases, tc_cols;
  unsigned int* sync;
  int* status;
  const int* skip;
};

struct PersistProg {
  PProgDev dev{};
  PPhase* d_phases = nullptr;
  PUnit* d_units = nullptr;
  int smem = 0, grid = 0;
};

// ---------------------------------------------------------------------------
// device side

template <typename T, int BM>
__device__ __forceinline__ void p_gemm_tile(const GemmDesc& g, int bx, int by, i64 zb, unsigned char* sm) {
  constexpr int S = GemmStages<T, BM>::value;
  T(*As)[16][BM + 1] = reinterpret_cast<T(*)[16][BM + 1]>(sm);
  constexpr size_t a_bytes = ((size_t)S * 16 * (BM + 1) * sizeof(T) + 15) / 16 * 16;
  T(*Bs)[16][65] = reinterpret_cast<T(*)[16][65]>(sm + a_bytes);
  gemm_tile<T, BM>(g, bx, by, zb, As, Bs);
}

__device__ __forceinline__ void p_gemm_dispatch(const GemmDesc& g, int f32, int bm, int bx, int by, i64 zb,
                                                unsigned char* sm) {
  if (f32) {
    if (bm == 64) p_gemm_tile<float, 64>(g, bx, by, zb, sm);
    else if (bm == 32) p_gemm_tile<float, 32>(g, bx, by, zb, sm);
    else p_gemm_tile<float, 16>(g, bx, by, zb, sm);
  } else {
    if (bm == 64) p_gemm_tile<double, 64>(g, bx, by, zb, sm);
    else if (bm == 32) p_gemm_tile<double, 32>(g, bx, by, zb, sm);
    else p_gemm_tile<double, 16>(g, bx, by, zb, sm);
  }
}

// tile t of a multi-GEMM unit (the mapping of multi_gemm_kernel)
__device__ __forceinline__ void p_mgemm_item(const PUnit& u, i64 t, unsigned char* sm) {
  const MOp* __restrict__ ops = static_cast<const MOp*>(u.table);
  int lo = 0, hi = u.nops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ops[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  const MOp& op = ops[lo];
  if (op.g.skip && *op.g.skip) return;
  const i64 r = t - op.tile_begin;
  const int bx = (int)(r % op.tiles_x);
  const int by = (int)((r / op.tiles_x) % op.tiles_y);
  const i64 zb = r / ((i64)op.tiles_x * op.tiles_y);
  p_gemm_dispatch(op.g, u.f32, u.bm, bx, by, zb, sm);
}

template <typename T>
__device__ __forceinline__ void p_gemv_row(const PUnit& u, int i, int lane) {
  int lo = 0, hi = u.n;
  if (u.tri == 1) hi = min(u.n, i + 1);
  if (u.tri == 2) lo = i;
  const T* row = reinterpret_cast<const T*>(u.A) + (i64)i * u.lda;
  const T s = warp_row_dot(row, reinterpret_cast<const T*>(u.x), lo, hi, lane);
  T* y = reinterpret_cast<T*>(u.y);
  if (lane == 0) y[i] = (T)u.alpha * s + ((T)u.beta != T(0) ? (T)u.beta * y[i] : T(0));
}

// Returns false if the barrier gave up (then *abort is set for the CTA).
__device__ __forceinline__ bool grid_barrier(unsigned int* sync, int* status, int* abort_sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = sync + 1;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(sync, 1u) == gridDim.x - 1) {
      atomicExch(sync, 0u);
      __threadfence();
      atomicAdd(sync + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (++spins > (1LL << 24)) {
          atomicOr(status, (int)DEV_TIMEOUT);
          *abort_sm = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *abort_sm == 0;
}

__global__ void __launch_bounds__(P_THREADS, 1) persist_kernel(PProgDev prog) {
  extern __shared__ __align__(1024) unsigned char p_smem[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)p_smem + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (prog.tc_cols > 0 && warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(prog.tc_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  TcCtx cx{};
  for (int b = 0; b < 2; ++b) {  // one operand set (the persistent kernel's shared memory budget)
    cx.sAhi[b] = sm;
    cx.sAlo[b] = sm + TC_A_BYTES;
    cx.sBhi[b] = sm + 2 * TC_A_BYTES;
    cx.sBlo[b] = sm + 2 * TC_A_BYTES + prog.tc_cols * 128;
    cx.bar[b] = &bar;
    cx.phase[b] = 0u;
  }
  cx.nbuf = 1;
  cx.tmem = prog.tc_cols > 0 ? tmem_slot : 0u;
  cx.abort_flag = &abort_flag;
  cx.status = prog.status;
  // a converged CG (the plan's skip flag, written before this launch) runs nothing
  const bool skip_all = prog.skip && *prog.skip;
  for (int ph = 0; ph < prog.nphases && !skip_all; ++ph) {
    const PPhase P = prog.phases[ph];
    for (i64 it = blockIdx.x; it < P.items && !abort_flag; it += gridDim.x) {
      int ui = P.unit0;
      while (ui + 1 < P.unit0 + P.nunits && prog.units[ui + 1].item_begin <= it) ++ui;
      const PUnit& u = prog.units[ui];
      const i64 local = it - u.item_begin;
      switch (u.kind) {
        case PU_MGEMM:
          p_mgemm_item(u, local, sm);
          break;
        case PU_MGEMV:
          if (u.f32)
            mgemv_item<float, false>(static_cast<const MGemv*>(u.table), u.nops, u.total, u.bm, local,
                                     reinterpret_cast<float*>(sm));
          else
            mgemv_item<double, false>(static_cast<const MGemv*>(u.table), u.nops, u.total, u.bm, local,
                                      reinterpret_cast<double*>(sm));
          break;
        case PU_TC:
          tc_tile(static_cast<const TcOp*>(u.table), u.nops, local, cx);
          break;
        case PU_CONTR: {
          const ContrOp& op = face_find(static_cast<const ContrOp*>(u.table), u.nops, local);
          if (op.skip && *op.skip) break;
          if (u.f32) contr_item<float>(op, local - op.item_begin, reinterpret_cast<float*>(sm));
          else contr_item<double>(op, local - op.item_begin, reinterpret_cast<double*>(sm));
          break;
        }
        case PU_BILIN: {
          const BilOp& op = face_find(static_cast<const BilOp*>(u.table), u.nops, local);
          if (op.skip && *op.skip) break;
          if (u.f32) bilin_item<float>(op, local - op.item_begin, reinterpret_cast<float*>(sm));
          else bilin_item<double>(op, local - op.item_begin, reinterpret_cast<double*>(sm));
          break;
        }
        case PU_EXPADD: {
          const ExpAddOp& op = face_find(static_cast<const ExpAddOp*>(u.table), u.nops, local);
          if (op.skip && *op.skip) break;
          if (u.f32) expadd_item<float>(op, local - op.item_begin);
          else expadd_item<double>(op, local - op.item_begin);
          break;
        }
        case PU_COPY: {
          const i64 w0 = local * P_ELEMS;
          const unsigned int* s = static_cast<const unsigned int*>(u.src);
          unsigned int* d = static_cast<unsigned int*>(u.dst);
          for (i64 e = w0 + tid; e < w0 + P_ELEMS && e < u.words; e += P_THREADS) d[e] = s[e];
          break;
        }
        case PU_GEMM: {
          if (u.g.skip && *u.g.skip) break;
          const int bx = (int)(local % u.tiles_x);
          const int by = (int)((local / u.tiles_x) % u.tiles_y);
          const i64 zb = local / ((i64)u.tiles_x * u.tiles_y);
          p_gemm_dispatch(u.g, u.f32, u.bm, bx, by, zb, sm);
          break;
        }
        case PU_TCSUM: {
          // out = sum of the segment groups in order (+ gamma D + beta out), as tc_sum_kernel
          const TcOp& op = static_cast<const TcOp*>(u.table)[local / P_SUM_CHUNKS];
          if (op.sgroups <= 1 || (op.skip && *op.skip)) break;
          const i64 n = (i64)op.N * op.R;
          for (i64 e = (local % P_SUM_CHUNKS) * P_THREADS + tid; e < n; e += (i64)P_SUM_CHUNKS * P_THREADS) {
            float v = 0.0f;
            for (int g = 0; g < op.sgroups; ++g) v += op.part[(i64)g * n + e];
            if (op.D) v += op.gamma * op.D[e];
            if (op.beta != 0.0f) v += op.beta * op.out[e];
            op.out[e] = v;
          }
          break;
        }
        case PU_GEMV: {
          if (u.skip && *u.skip) break;
          const i64 i = local * P_GEMV_ROWS + warp;
          if (i < u.m) {
            if (u.f32) p_gemv_row<float>(u, (int)i, lane);
            else p_gemv_row<double>(u, (int)i, lane);
          }
          break;
        }
        default:
          break;
      }
    }
    if (!grid_barrier(prog.sync, prog.status, &abort_flag)) break;
  }
  __syncthreads();
  if (prog.tc_cols > 0 && warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(cx.tmem), "r"(prog.tc_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// host side

static int gemm_smem_bytes() {
  // the largest ring among the six (type, row tile) variants, plus the B offset rounding
  auto ring = [](size_t es, int bm, int stages) {
    return ((size_t)stages * 16 * (bm + 1) * es + 15) / 16 * 16 + (size_t)stages * 16 * 65 * es;
  };
  size_t m = 0;
  m = std::max(m, ring(4, 64, GemmStages<float, 64>::value));
  m = std::max(m, ring(4, 32, GemmStages<float, 32>::value));
  m = std::max(m, ring(4, 16, GemmStages<float, 16>::value));
  m = std::max(m, ring(8, 64, GemmStages<double, 64>::value));
  m = std::max(m, ring(8, 32, GemmStages<double, 32>::value));
  m = std::max(m, ring(8, 16, GemmStages<double, 16>::value));
  return (int)m;
}

bool persist_enabled() {
  static const int on = [] {
    const char* e = std::getenv("GPFVM_PERSIST");
    return (e && std::atoi(e) != 0) ? 1 : 0;
  }();
  return on != 0;
}

PersistProg* persist_build(const Plan& plan, unsigned int* sync, int* status) {
  std::vector<PPhase> phases;
  std::vector<PUnit> units;
  int tc_maxn = 0;
  int face_smem = 0;  // largest bilinear item
  auto unit_of = [&](const Plan& plan, const PlanOp& op, PUnit& u) -> bool {
    u = PUnit{};
    switch (op.kind) {
      case PlanOp::TC:
        u.kind = PU_TC;
        u.table = op.tc_ops;
        u.nops = op.tc_nops;
        u.items = op.tc_tiles;
        tc_maxn = std::max(tc_maxn, op.tc_maxn);
        return true;
      case PlanOp::COPY:
        if (op.cp_bytes % 4) return false;
        u.kind = PU_COPY;
        u.dst = op.cp_dst;
        u.src = op.cp_src;
        u.words = op.cp_bytes / 4;
        u.items = (u.words + P_ELEMS - 1) / P_ELEMS;
        return true;
      case PlanOp::GEMM: {
        u.kind = PU_GEMM;
        u.g = op.g;
        u.f32 = op.g.f32;
        u.bm = op.g.tile == 2 ? 16 : (op.g.tile == 1 ? 32 : 64);
        u.tiles_x = (op.g.n + 63) / 64;
        u.tiles_y = (op.g.m + u.bm - 1) / u.bm;
        u.items = (i64)u.tiles_x * u.tiles_y * op.g.batch * op.g.n_groups;
        return true;
      }
      case PlanOp::GEMV:
      case PlanOp::GEMV32:
        u.kind = PU_GEMV;
        u.f32 = op.kind == PlanOp::GEMV32;
        u.m = op.m;
        u.n = op.n;
        u.tri = op.tri;
        u.A = op.A;
        u.lda = op.lda;
        u.x = op.x;
        u.y = op.y;
        u.alpha = op.alpha;
        u.beta = op.beta;
        u.skip = plan.skip;
        u.items = (op.m + P_GEMV_ROWS - 1) / P_GEMV_ROWS;
        return true;
      default:
        return false;  // host callbacks cannot run inside the kernel
    }
  };
  std::vector<PUnit> sums;  // reductions of split tensor-core levels of the current phase
  auto unit_of_sum = [&](const PlanOp& op) {
    if (op.kind == PlanOp::TC && op.tc_split) {
      PUnit u{};
      u.kind = PU_TCSUM;
      u.table = op.tc_ops;
      u.nops = op.tc_nops;
      u.items = (i64)op.tc_nops * P_SUM_CHUNKS;
      sums.push_back(u);
    }
  };
  // a background chain (FORK) runs in place: the kernel executes phases in order
  std::function<bool(const Plan&)> emit = [&](const Plan& plan) -> bool {
  const auto& ops = plan.ops;
  size_t i = 0;
  while (i < ops.size()) {
    if (ops[i].kind == PlanOp::FORK) {
      if (!emit(*plan.bgs[ops[i].bg])) return false;
      ++i;
      continue;
    }
    if (ops[i].kind == PlanOp::JOIN) {
      ++i;
      continue;
    }
    PPhase P{(int)units.size(), 0, 0};
    sums.clear();
    auto push = [&](PUnit u) {
      u.item_begin = P.items;
      P.items += u.items;
      units.push_back(u);
      P.nunits++;
    };
    if (ops[i].phase < 0) {
      PUnit u;
      if (!unit_of(plan, ops[i], u)) return false;
      if (u.items > 0) push(u);
      unit_of_sum(ops[i]);
      ++i;
    } else {
      const int ph = ops[i].phase;
      size_t j = i;
      while (j < ops.size() && ops[j].phase == ph) ++j;
      for (const LaunchUnit& lu : plan.phase_units[ph]) {
        PUnit u{};
        if (lu.kind == 0) {
          u.kind = PU_MGEMM;
          u.f32 = lu.f32;
          u.bm = lu.bm;
          u.nops = lu.nops;
          u.table = plan.d_tables + lu.offset;
          u.items = lu.total;
        } else if (lu.kind >= 2) {
          u.kind = lu.kind == 2 ? PU_CONTR : (lu.kind == 3 ? PU_BILIN : PU_EXPADD);
          face_smem = std::max(face_smem, lu.smem);
          u.f32 = lu.f32;
          u.nops = lu.nops;
          u.table = plan.d_tables + lu.offset;
          u.items = lu.total;
        } else {
          u.kind = PU_MGEMV;
          u.f32 = lu.f32;
          u.bm = lu.bm;  // warps per row
          u.nops = lu.nops;
          u.table = plan.d_tables + lu.offset;
          u.total = lu.total;
          u.items = (lu.total * lu.bm + 7) / 8;
        }
        if (u.items > 0) push(u);
      }
      for (size_t t = i; t < j; ++t) {
        if (!ops[t].func_like()) continue;
        PUnit u;
        if (!unit_of(plan, ops[t], u)) return false;
        if (u.items > 0) push(u);
        unit_of_sum(ops[t]);
      }
      i = j;
    }
    if (P.nunits > 0) phases.push_back(P);
    if (!sums.empty()) {  // the next phase may read what the split levels wrote
      PPhase S{(int)units.size(), 0, 0};
      for (PUnit u : sums) {
        u.item_begin = S.items;
        S.items += u.items;
        units.push_back(u);
        S.nunits++;
      }
      phases.push_back(S);
    }
  }
  return true;
  };
  if (!emit(plan) || phases.empty()) return nullptr;
  auto* pr = new PersistProg();
  int tc_cols = 0;
  if (tc_maxn > 0) {
    const int npad = (tc_maxn + 15) & ~15;
    tc_cols = 32;
    while (tc_cols < npad) tc_cols <<= 1;
  }
  const int tc_smem = tc_cols > 0 ? 2 * TC_A_BYTES + 2 * tc_cols * 128 : 0;
  pr->smem = std::max(std::max(gemm_smem_bytes(), tc_smem), face_smem) + 1024;
  GPFVM_CUDA(cudaMalloc(&pr->d_phases, sizeof(PPhase) * phases.size()));
  GPFVM_CUDA(cudaMalloc(&pr->d_units, sizeof(PUnit) * units.size()));
  GPFVM_CUDA(cudaMemcpy(pr->d_phases, phases.data(), sizeof(PPhase) * phases.size(), cudaMemcpyHostToDevice));
  GPFVM_CUDA(cudaMemcpy(pr->d_units, units.data(), sizeof(PUnit) * units.size(), cudaMemcpyHostToDevice));
  pr->dev = PProgDev{pr->d_phases, pr->d_units, (int)phases.size(), tc_cols, sync, status, plan.skip};
  // one CTA per SM (the kernel is register-heavy); all of them must be resident
  int dev = 0, nsm = 0, occ = 0;
  GPFVM_CUDA(cudaGetDevice(&dev));
  GPFVM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  GPFVM_CUDA(cudaFuncSetAttribute(persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pr->smem));
  GPFVM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persist_kernel, P_THREADS, pr->smem));
  pr->grid = occ >= 1 ? nsm : 0;
  return pr;
}

void persist_free(PersistProg* prog) {
  if (!prog) return;
  if (prog->d_phases) cudaFree(prog->d_phases);
  if (prog->d_units) cudaFree(prog->d_units);
  delete prog;
}

bool persist_run(const PersistProg* prog, cudaStream_t st) {
  if (!prog || prog->grid <= 0) return false;
  // the grid-barrier words start from zero on every launch (a launch that gave
  // up at a barrier leaves its arrival count behind)
  GPFVM_CUDA(cudaMemsetAsync(prog->dev.sync, 0, 2 * sizeof(unsigned int), st));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(prog->grid);
  cfg.blockDim = dim3(P_THREADS);
  cfg.dynamicSmemBytes = prog->smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  GPFVM_CUDA(cudaLaunchKernelEx(&cfg, persist_kernel, prog->dev));
  count_launch();
  return true;
}

}  // namespace gpfvm
