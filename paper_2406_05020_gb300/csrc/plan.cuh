// A "plan" is a fixed sequence of kernel launches whose argument tables live
// in device memory.  Plans are built once per problem (at create/assemble)
// and replayed every CG iteration, so they can be captured in CUDA graphs.
#pragma once
#include <algorithm>
#include <cstring>
#include <functional>
#include <memory>

#include "face.cuh"
#include "kernels.cuh"
#include "persist.cuh"
#include "tc.cuh"

namespace gpfvm {

struct PlanOp {
  // FUNC runs a host callback; TC and COPY are typed device ops that the
  // persistent plan kernel can also execute (they run like FUNC ops in run()).
  // FORK starts background chain `bg` of the plan on its own stream; JOIN
  // makes the plan's stream wait for it.
  // CONTR, BILIN and EXPADD are the face-set ops of face.cuh (phased only:
  // merged into one launch per kind, element type and phase).
  enum Kind { GEMM, GEMV, GEMV32, FUNC, TC, COPY, FORK, JOIN, CONTR, BILIN, EXPADD } kind;
  int phase = -1;  // ops sharing a phase id (>= 0, consecutive) are independent: merged launches
  GemmDesc g;
  int seg0 = 0, group0 = 0;
  // GEMV
  int m = 0, n = 0, tri = 0;
  const double* A = nullptr;
  i64 lda = 0;
  const double* x = nullptr;
  double* y = nullptr;
  const double* z = nullptr;   // phased GEMV only: y = alpha A x + beta zs .* z (z = y if null)
  const double* zs = nullptr;  // phased GEMV only: per-row scale of z (FP64)
  double alpha = 1.0, beta = 0.0;
  std::function<void(cudaStream_t)> fn;
  // TC: tensor-core mode products of one level (see tc.cu)
  const TcOp* tc_ops = nullptr;
  int tc_nops = 0, tc_maxn = 0;
  i64 tc_tiles = 0;
  int* tc_status = nullptr;
  int tc_split = 0;  // some op of the level sums segment groups (second launch)
  // COPY: device to device
  void* cp_dst = nullptr;
  const void* cp_src = nullptr;
  i64 cp_bytes = 0;
  int bg = -1;  // FORK: index into Plan::bgs
  int fc_f32 = 0;  // face ops: element type
  ContrOp fco{};
  BilOp fbo{};
  ExpAddOp feo{};
  bool face() const { return kind == CONTR || kind == BILIN || kind == EXPADD; }
  bool func_like() const { return kind == FUNC || kind == TC || kind == COPY; }
};

// One merged launch of a phase: a table of GEMM ops (same element type and
// row tile) or of GEMV ops (same element type).
struct LaunchUnit {
  int kind;  // 0 multi-GEMM, 1 multi-GEMV, 2 / 3 / 4 face CONTR / BILIN / EXPADD
  int f32, bm, nops;
  i64 total;
  size_t offset;  // byte offset of the op table in the plan's table buffer
  int smem = 0;   // dynamic shared memory of the launch (face BILIN)
};

// Auxiliary streams on which the independent launches of one phase run
// side by side (fork from the plan's stream at the phase start, join at its
// end); under stream capture they become parallel graph branches.
struct Fan {
  static constexpr int NAUX = 3;
  cudaStream_t aux[NAUX] = {};
  cudaEvent_t fork = nullptr, join[NAUX] = {};
  // the background chain of a plan (FORK .. JOIN) runs on bgs
  cudaStream_t bgs = nullptr;
  cudaEvent_t bg_fork = nullptr, bg_join = nullptr;
  void create() {
    for (int a = 0; a < NAUX; ++a) {
      GPFVM_CUDA(cudaStreamCreateWithFlags(&aux[a], cudaStreamNonBlocking));
      GPFVM_CUDA(cudaEventCreateWithFlags(&join[a], cudaEventDisableTiming));
    }
    GPFVM_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    GPFVM_CUDA(cudaStreamCreateWithFlags(&bgs, cudaStreamNonBlocking));
    GPFVM_CUDA(cudaEventCreateWithFlags(&bg_fork, cudaEventDisableTiming));
    GPFVM_CUDA(cudaEventCreateWithFlags(&bg_join, cudaEventDisableTiming));
  }
  void destroy() {
    for (int a = 0; a < NAUX; ++a) {
      if (aux[a]) cudaStreamDestroy(aux[a]);
      if (join[a]) cudaEventDestroy(join[a]);
      aux[a] = nullptr;
      join[a] = nullptr;
    }
    if (fork) cudaEventDestroy(fork);
    if (bgs) cudaStreamDestroy(bgs);
    if (bg_fork) cudaEventDestroy(bg_fork);
    if (bg_join) cudaEventDestroy(bg_join);
    fork = nullptr;
    bgs = nullptr;
    bg_fork = bg_join = nullptr;
  }
};

class Plan {
 public:
  std::vector<GemmSeg> segs;
  std::vector<GemmGroup> groups;
  std::vector<PlanOp> ops;
  GemmSeg* d_segs = nullptr;
  GemmGroup* d_groups = nullptr;
  char* d_tables = nullptr;
  std::vector<std::vector<LaunchUnit>> phase_units;  // indexed by phase id
  int n_phases = 0;
  const int* skip = nullptr;  // device flag: when set, every GEMM/GEMV of the plan is a no-op
  const Fan* fan = nullptr;    // optional: run the independent launches of a phase concurrently
  PersistProg* prog = nullptr; // optional: the whole plan as one cooperative launch (persist.cu)
  std::vector<std::shared_ptr<Plan>> bgs;  // background chains (FORK / JOIN)

  ~Plan() { release(); }
  void release() {
    persist_free(prog);
    prog = nullptr;
    if (d_segs) cudaFree(d_segs);
    if (d_groups) cudaFree(d_groups);
    if (d_tables) cudaFree(d_tables);
    d_segs = nullptr;
    d_groups = nullptr;
    d_tables = nullptr;
  }
  Plan() = default;
  Plan(const Plan&) = delete;
  Plan& operator=(const Plan&) = delete;
  Plan(Plan&& o) noexcept { *this = std::move(o); }
  Plan& operator=(Plan&& o) noexcept {
    if (this != &o) {
      release();
      segs = std::move(o.segs);
      groups = std::move(o.groups);
      ops = std::move(o.ops);
      phase_units = std::move(o.phase_units);
      bgs = std::move(o.bgs);
      n_phases = o.n_phases;
      skip = o.skip;
      fan = o.fan;
      prog = o.prog;
      o.prog = nullptr;
      d_segs = o.d_segs; d_groups = o.d_groups; d_tables = o.d_tables;
      o.d_segs = nullptr; o.d_groups = nullptr; o.d_tables = nullptr;
    }
    return *this;
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
  // y = alpha A x + beta zs .* z (zs may be null), FP64 or FP32 (f32) data; only inside zipped chains
  void gemvz(bool f32, int m, int n, const void* A, i64 lda, const void* x, void* y, double alpha, double beta,
             const void* z, const double* zs, int tri = 0) {
    PlanOp op;
    op.kind = f32 ? PlanOp::GEMV32 : PlanOp::GEMV;
    op.m = m; op.n = n; op.A = (const double*)A; op.lda = lda; op.x = (const double*)x; op.y = (double*)y;
    op.alpha = alpha; op.beta = beta; op.tri = tri;
    op.z = (const double*)z; op.zs = zs;
    ops.push_back(op);
  }
  void func(std::function<void(cudaStream_t)> f) {
    PlanOp op;
    op.kind = PlanOp::FUNC;
    op.fn = std::move(f);
    ops.push_back(op);
  }
  void tc(const TcOp* d_ops, int nops, i64 tiles, int maxn, int* status, int split = 0) {
    PlanOp op;
    op.kind = PlanOp::TC;
    op.tc_ops = d_ops; op.tc_nops = nops; op.tc_tiles = tiles; op.tc_maxn = maxn; op.tc_status = status;
    op.tc_split = split;
    ops.push_back(op);
  }
  void copy(void* dst, const void* src, i64 bytes) {
    PlanOp op;
    op.kind = PlanOp::COPY;
    op.cp_dst = dst; op.cp_src = src; op.cp_bytes = bytes;
    ops.push_back(op);
  }
  void contr(const ContrOp& o, bool f32) {
    PlanOp op;
    op.kind = PlanOp::CONTR;
    op.fco = o;
    op.fc_f32 = f32 ? 1 : 0;
    ops.push_back(op);
  }
  void bilin(const BilOp& o, bool f32) {
    PlanOp op;
    op.kind = PlanOp::BILIN;
    op.fbo = o;
    op.fc_f32 = f32 ? 1 : 0;
    ops.push_back(op);
  }
  void expadd(const ExpAddOp& o, bool f32) {
    PlanOp op;
    op.kind = PlanOp::EXPADD;
    op.feo = o;
    op.fc_f32 = f32 ? 1 : 0;
    ops.push_back(op);
  }
  // Runs `chain` concurrently with the ops that follow, up to the next join():
  // they must neither write what the chain reads nor touch what it writes.
  void fork(Plan&& chain) {
    bgs.push_back(std::make_shared<Plan>(std::move(chain)));
    PlanOp op;
    op.kind = PlanOp::FORK;
    op.bg = (int)bgs.size() - 1;
    ops.push_back(op);
  }
  void join() {
    PlanOp op;
    op.kind = PlanOp::JOIN;
    ops.push_back(op);
  }
  void append(const Plan& o) {
    const int s0 = (int)segs.size(), g0 = (int)groups.size();
    for (auto s : o.segs) segs.push_back(s);
    for (auto G : o.groups) { G.seg0 += s0; groups.push_back(G); }
    for (auto op : o.ops) { op.group0 += g0; op.phase = -1; ops.push_back(op); }
  }
  // Appends independent chains level by level: op l of every chain shares one
  // phase (they read only what earlier levels or earlier plan ops wrote).
  void zip(const std::vector<const Plan*>& chains, size_t max_levels = (size_t)-1) {
    const int s0 = (int)segs.size(), g0 = (int)groups.size();
    std::vector<int> sbase, gbase;
    int so = s0, go = g0;
    for (const Plan* c : chains) {
      sbase.push_back(so);
      gbase.push_back(go);
      for (auto x : c->segs) segs.push_back(x);
      for (auto G : c->groups) { G.seg0 += so - s0 + s0; groups.push_back(G); }
      so += (int)c->segs.size();
      go += (int)c->groups.size();
    }
    // fix the group seg0 offsets (each chain's groups index its own segs)
    {
      int gi = g0;
      for (size_t c = 0; c < chains.size(); ++c)
        for (size_t k = 0; k < chains[c]->groups.size(); ++k, ++gi)
          groups[gi].seg0 = chains[c]->groups[k].seg0 + sbase[c];
    }
    size_t maxlen = 0;
    for (const Plan* c : chains) maxlen = std::max(maxlen, c->ops.size());
    const size_t zl = std::min(maxlen, max_levels);
    for (size_t l = 0; l < zl; ++l) {
      const int ph = n_phases++;
      for (size_t c = 0; c < chains.size(); ++c) {
        if (l >= chains[c]->ops.size()) continue;
        PlanOp op = chains[c]->ops[l];
        op.group0 += gbase[c];
        op.phase = ph;
        ops.push_back(op);
      }
    }
    // levels beyond max_levels: one phase per level and chain pair (a, b) of
    // `pairs`, i.e. chains that write the same output never share a phase
    for (size_t c = 0; c < chains.size(); ++c)
      for (size_t l = zl; l < chains[c]->ops.size(); ++l) {
        PlanOp op = chains[c]->ops[l];
        op.group0 += gbase[c];
        op.phase = -1;
        ops.push_back(op);
      }
  }
  // Appends chains placed by phase: op l of chain c joins the (start[c] + l)-th
  // new phase.  The caller guarantees that the ops sharing a phase are
  // independent (each reads only what earlier phases or plan ops wrote).
  void zip_at(const std::vector<const Plan*>& chains, const std::vector<int>& start) {
    const int s0 = (int)segs.size();
    std::vector<int> sbase, gbase;
    int so = s0, go = (int)groups.size();
    for (const Plan* c : chains) {
      sbase.push_back(so);
      gbase.push_back(go);
      for (auto x : c->segs) segs.push_back(x);
      for (auto G : c->groups) { G.seg0 += so; groups.push_back(G); }
      so += (int)c->segs.size();
      go += (int)c->groups.size();
    }
    int nl = 0;
    for (size_t c = 0; c < chains.size(); ++c) nl = std::max(nl, start[c] + (int)chains[c]->ops.size());
    for (int l = 0; l < nl; ++l) {
      int ph = -1;
      for (size_t c = 0; c < chains.size(); ++c) {
        const int k = l - start[c];
        if (k < 0 || k >= (int)chains[c]->ops.size()) continue;
        if (ph < 0) ph = n_phases++;
        PlanOp op = chains[c]->ops[k];
        op.group0 += gbase[c];
        op.phase = ph;
        ops.push_back(op);
      }
    }
  }
  // Copy of ops [from, to) with the argument tables they use.
  Plan slice(size_t from, size_t to) const {
    Plan r;
    to = std::min(to, ops.size());
    for (size_t i = from; i < to; ++i) {
      PlanOp op = ops[i];
      op.phase = -1;
      if (op.kind == PlanOp::GEMM) {
        const int g0 = (int)r.groups.size();
        for (int k = 0; k < op.g.n_groups; ++k) {
          GemmGroup G = groups[op.group0 + k];
          const int s0 = (int)r.segs.size();
          for (int j = 0; j < G.nseg; ++j) r.segs.push_back(segs[G.seg0 + j]);
          G.seg0 = s0;
          r.groups.push_back(G);
        }
        op.group0 = g0;
      }
      r.ops.push_back(op);
    }
    return r;
  }
  // Like zip, but chain i of `a` and chain i of `b` (different outputs) share
  // one phase per level; used for the conflicting last levels.
  void zip_pairs(const std::vector<const Plan*>& a, const std::vector<const Plan*>& b) {
    const size_t n = std::max(a.size(), b.size());
    for (size_t i = 0; i < n; ++i) {
      std::vector<const Plan*> c;
      if (i < a.size()) c.push_back(a[i]);
      if (i < b.size()) c.push_back(b[i]);
      zip(c);
    }
  }
  void finalize() {
    release();
    bool open = false;
    for (auto& op : ops) {
      if (op.kind == PlanOp::FORK && open) throw CudaError{cudaErrorInvalidValue, "plan: nested background chain"};
      if (op.kind == PlanOp::FORK) open = true;
      if (op.kind == PlanOp::JOIN) open = false;
    }
    if (open) throw CudaError{cudaErrorInvalidValue, "plan: background chain without join"};
    for (auto& b : bgs) {
      b->skip = skip;
      b->finalize();
    }
    for (auto& op : ops) {
      if ((op.kind == PlanOp::GEMV || op.kind == PlanOp::GEMV32) && op.phase < 0 && (op.z || op.zs))
        throw CudaError{cudaErrorInvalidValue, "plan: a GEMV with z or zs must be part of a zipped chain"};
      if (op.face() && op.phase < 0)
        throw CudaError{cudaErrorInvalidValue, "plan: face-set ops must be part of a zipped chain"};
    }
    phase_units.assign(n_phases, {});
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
    // merged launch tables for phased ops
    std::vector<char> blob;
    auto put = [&](const void* p, size_t n) {
      size_t off = (blob.size() + 255) / 256 * 256;
      blob.resize(off + n);
      std::memcpy(blob.data() + off, p, n);
      return off;
    };
    for (int ph = 0; ph < n_phases; ++ph) {
      for (int f32 = 0; f32 < 2; ++f32) {
        for (int tile = 0; tile < 3; ++tile) {
          std::vector<MOp> mops;
          i64 total = 0;
          for (auto& op : ops) {
            if (op.phase != ph || op.kind != PlanOp::GEMM || op.g.f32 != f32 || op.g.tile != tile) continue;
            const int bm = tile == 2 ? 16 : (tile == 1 ? 32 : 64);
            MOp m{};
            m.g = op.g;
            m.tiles_x = (op.g.n + 63) / 64;
            m.tiles_y = (op.g.m + bm - 1) / bm;
            m.tile_begin = total;
            total += (i64)m.tiles_x * m.tiles_y * op.g.batch * op.g.n_groups;
            mops.push_back(m);
          }
          if (mops.empty()) continue;
          LaunchUnit u{0, f32, tile == 2 ? 16 : (tile == 1 ? 32 : 64), (int)mops.size(), total, 0};
          u.offset = put(mops.data(), mops.size() * sizeof(MOp));
          phase_units[ph].push_back(u);
        }
        std::vector<MGemv> gops;
        i64 rows = 0;
        int maxn = 0;
        for (auto& op : ops) {
          const bool is32 = op.kind == PlanOp::GEMV32;
          if (op.phase != ph || !(op.kind == PlanOp::GEMV || is32) || (int)is32 != f32) continue;
          MGemv m{};
          m.A = op.A; m.x = op.x; m.z = op.z ? op.z : op.y; m.y = op.y; m.zs = op.zs;
          m.lda = op.lda; m.row_begin = rows; m.m = op.m; m.n = op.n; m.tri = op.tri;
          m.alpha = op.alpha; m.beta = op.beta; m.skip = skip;
          rows += op.m;
          maxn = std::max(maxn, op.n);
          gops.push_back(m);
        }
        if (!gops.empty()) {
          LaunchUnit u{1, f32, mgemv_split(rows, maxn), (int)gops.size(), rows, 0};  // bm: warps per row
          u.offset = put(gops.data(), gops.size() * sizeof(MGemv));
          phase_units[ph].push_back(u);
        }
        // face-set ops: one table per kind
        {
          std::vector<ContrOp> co;
          std::vector<BilOp> bo;
          std::vector<ExpAddOp> eo;
          i64 ic = 0, ib = 0, ie = 0;
          for (auto& op : ops) {
            if (op.phase != ph || !op.face() || op.fc_f32 != f32) continue;
            if (op.kind == PlanOp::CONTR) {
              ContrOp o = op.fco;
              o.items = contr_items(o.pre, o.post);
              o.item_begin = ic;
              o.skip = skip;
              ic += o.items;
              co.push_back(o);
            } else if (op.kind == PlanOp::BILIN) {
              BilOp o = op.fbo;
              o.items = (i64)std::max(o.batch, 1) * ((o.R + FACE_RB - 1) / FACE_RB);
              o.item_begin = ib;
              o.skip = skip;
              ib += o.items;
              bo.push_back(o);
            } else {
              ExpAddOp o = op.feo;
              o.items = (o.n + FACE_EXP_ELEMS - 1) / FACE_EXP_ELEMS;
              o.item_begin = ie;
              o.skip = skip;
              ie += o.items;
              eo.push_back(o);
            }
          }
          if (!co.empty()) {
            LaunchUnit u{2, f32, 0, (int)co.size(), ic, 0};
            u.offset = put(co.data(), co.size() * sizeof(ContrOp));
            phase_units[ph].push_back(u);
          }
          if (!bo.empty()) {
            LaunchUnit u{3, f32, 0, (int)bo.size(), ib, 0};
            u.offset = put(bo.data(), bo.size() * sizeof(BilOp));
            i64 sm = 0;
            for (auto& o : bo) sm = std::max(sm, bilin_smem_elems(o.C, o.K1, o.K2, o.nA, o.nX, o.nB, o.nt));
            u.smem = (int)(sm * (f32 ? 4 : 8));
            if (u.smem > FACE_SMEM_MAX) throw CudaError{cudaErrorInvalidValue, "plan: bilinear form too large"};
            phase_units[ph].push_back(u);
          }
          if (!eo.empty()) {
            LaunchUnit u{4, f32, 0, (int)eo.size(), ie, 0};
            u.offset = put(eo.data(), eo.size() * sizeof(ExpAddOp));
            phase_units[ph].push_back(u);
          }
        }
      }
    }
    if (!blob.empty()) {
      GPFVM_CUDA(cudaMalloc(&d_tables, blob.size()));
      GPFVM_CUDA(cudaMemcpy(d_tables, blob.data(), blob.size(), cudaMemcpyHostToDevice));
    }
  }
  void run_op(const PlanOp& op, cudaStream_t st) const {
    if (op.kind == PlanOp::GEMM) launch_gemm64(op.g, st);
    else if (op.kind == PlanOp::GEMV)
      launch_gemv64(op.m, op.n, op.A, op.lda, op.x, op.y, op.alpha, op.beta, op.tri, st, skip);
    else if (op.kind == PlanOp::GEMV32)
      launch_gemv32(op.m, op.n, (const float*)op.A, op.lda, (const float*)op.x, (float*)op.y, (float)op.alpha,
                    (float)op.beta, op.tri, st, skip);
    else if (op.kind == PlanOp::TC)
      launch_tc_modes(op.tc_ops, op.tc_nops, op.tc_tiles, op.tc_maxn, op.tc_status, st, op.tc_split);
    else if (op.kind == PlanOp::COPY) {
      if (op.cp_bytes > 0) GPFVM_CUDA(cudaMemcpyAsync(op.cp_dst, op.cp_src, op.cp_bytes, cudaMemcpyDeviceToDevice, st));
    } else if (op.kind == PlanOp::FORK) {
      if (!fan) {
        bgs[op.bg]->run(st);  // no side stream: in place
      } else {
        GPFVM_CUDA(cudaEventRecord(fan->bg_fork, st));
        GPFVM_CUDA(cudaStreamWaitEvent(fan->bgs, fan->bg_fork, 0));
        bgs[op.bg]->run(fan->bgs);
        GPFVM_CUDA(cudaEventRecord(fan->bg_join, fan->bgs));
      }
    } else if (op.kind == PlanOp::JOIN) {
      if (fan) GPFVM_CUDA(cudaStreamWaitEvent(st, fan->bg_join, 0));
    } else op.fn(st);
  }
  void run_unit(const LaunchUnit& u, cudaStream_t st) const {
    if (u.kind == 0) launch_multi_gemm((const MOp*)(d_tables + u.offset), u.nops, u.total, u.f32, u.bm, st);
    else if (u.kind == 1) launch_multi_gemv((const MGemv*)(d_tables + u.offset), u.nops, u.total, u.f32, u.bm, st);
    else launch_face(u.kind - 2, d_tables + u.offset, u.nops, u.total, u.f32, u.smem, st);
  }
  // Ops of one phase are consecutive; its merged launch units and FUNC ops
  // are mutually independent.  Without a fan they run in order on st.
  void run(cudaStream_t st) const {
    if (prog && persist_enabled() && persist_run(prog, st)) return;
    size_t i = 0;
    while (i < ops.size()) {
      const PlanOp& op = ops[i];
      if (op.phase < 0) {
        run_op(op, st);
        ++i;
        continue;
      }
      const int ph = op.phase;
      size_t j = i;
      while (j < ops.size() && ops[j].phase == ph) ++j;
      int lanes = (int)phase_units[ph].size();
      for (size_t t = i; t < j; ++t) lanes += ops[t].func_like();
      if (!fan || lanes <= 1) {
        for (const LaunchUnit& u : phase_units[ph]) run_unit(u, st);
        for (size_t t = i; t < j; ++t)
          if (ops[t].func_like()) run_op(ops[t], st);
      } else {
        GPFVM_CUDA(cudaEventRecord(fan->fork, st));
        bool used[Fan::NAUX] = {};
        int lane = 0;
        auto lane_stream = [&](int l) {
          if (l == 0) return st;
          const int a = (l - 1) % Fan::NAUX;
          if (!used[a]) {
            GPFVM_CUDA(cudaStreamWaitEvent(fan->aux[a], fan->fork, 0));
            used[a] = true;
          }
          return fan->aux[a];
        };
        for (const LaunchUnit& u : phase_units[ph]) run_unit(u, lane_stream(lane++));
        for (size_t t = i; t < j; ++t)
          if (ops[t].func_like()) run_op(ops[t], lane_stream(lane++));
        for (int a = 0; a < Fan::NAUX; ++a)
          if (used[a]) {
            GPFVM_CUDA(cudaEventRecord(fan->join[a], fan->aux[a]));
            GPFVM_CUDA(cudaStreamWaitEvent(st, fan->join[a], 0));
          }
      }
      i = j;
    }
  }
  int launches() const { return (int)ops.size(); }
};

// Builds the recursive Cholesky + inverse of an n x n SPD matrix A (lower
// triangle read, lda) into L and Linv (lower, row-major, lda); scratch must
// hold n*n/4 + 64 doubles.  status receives DEV_NOT_SPD on a pivot <= 0.
// Dense FP64 GEMMs of the factorisation by digit products on the tensor cores
// (oz_gemm) when given: exponent scratch for m and n rows of ceil(k / 128)
// windows each (rows x windows <= cap) and the status word of bounded waits.
struct OzChol {
  int* Aexp;
  int* Bexp;
  i64 cap;
  int* status;
};
void plan_chol_inverse(Plan& plan, double* A, double* L, double* Linv, int n, i64 lda,
                       double* scratch, int* status, const OzChol* oz = nullptr);
// One dense FP64 GEMM (one group, one segment; a_cs == 1): by digit products
// when `oz` is given and it is large, else the FP64 FMA kernel.
void plan_dense_gemm(Plan& plan, const GemmDesc& g, const GemmGroup& G, const GemmSeg& S, const OzChol* oz);
int dense_tile(int m, int n);

}  // namespace gpfvm
