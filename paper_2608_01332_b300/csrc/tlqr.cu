// libtlqr: C ABI and runtime of the rake-compress solver (Alg. 1) on sm_103a.
//
// The runtime owns the device copy of the plan and the workspace of one
// factorisation, and drives the per-round kernel sequence of kernels.cuh:
//   factor: condense -> for each round {rake, absorb, compress}
//           -> for each round backwards {expand} -> local factor
//           -> for each round {compose transition matrices}
//   solve:  affine init -> for each round {affine rake, absorb, compress}
//           -> backwards {affine expand} -> local solve
//           -> for each round {state compress} -> backwards {state expand}
//           -> recover
// In MIXED precision the factor and solve kernels run in FP32 and tlqr_solve
// adds FP64 iterative refinement (FP64 residual eq. (kkt) -> FP32 correction
// solve through the stored factors -> FP64 update).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/tlqr.h"
#include "fixed.cuh"
#include "kernels.cuh"
#include "plan.hpp"
#include "residual.cuh"
#include "residual_nodes.cuh"

using namespace tlqr;

namespace {

constexpr int kMaxWarpsPerBlock = 8;
constexpr int kTailOps = 128;        // per-phase operation count below which rounds join the tail kernel
// FP64 re-solve slots per factorisation (3 n^2 doubles each)
constexpr int kRedoCap = 4096;
constexpr int kTailThreads = fx::kTailBlock;
constexpr int kPanel = 8;            // right-hand sides per panel of tlqr_solve_rhs_panel
constexpr int kAsyncOps = 1024;     // default: rounds with at most this many operations run level-asynchronously
constexpr int kSpinLimit = 1 << 22;  // polls of one dependency wait (with backoff: about a second) before TIMEOUT
constexpr size_t kSmemBudget = 200 * 1024;

inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Shared memory of one warp for each kernel, in elements of T (+ ints).
struct WarpBytes {
  size_t condense, tau, compress, local_factor, compose_T, aff_init, vec1, local_solve, recover;
};

WarpBytes warp_bytes(int n, int m, size_t ts) {
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  WarpBytes w;
  w.condense = align16(ts * (mm + 4 * nm)) + align16(8 * mm);                 // + FP64 Cholesky scratch
  w.tau = align16(ts * 5 * nn + 4 * n);
  w.compress = align16(ts * 7 * nn + 4 * n);
  w.local_factor = align16(ts * (5 * nn + 3 * nm + mm) + 4 * n) + align16(ts * mm) + align16(8 * mm);
  w.compose_T = align16(ts * 2 * nn);
  w.aff_init = align16(ts * (2 * nn + 2 * nm + 2 * n + m));
  w.vec1 = align16(ts * (nn + n));
  w.local_solve = align16(ts * (nn + nm + mm + 4 * n + m));
  w.recover = align16(ts * (nn + nm + 2 * n + std::max(n, m)));
  return w;
}

// Raise (never lower) a kernel's dynamic shared-memory limit; done outside
// stream capture so that captured launches find it already set.
template <typename Kernel>
cudaError_t ensure_smem(Kernel kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<const void*, size_t> have;
  if (bytes <= 48 * 1024) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = have[(const void*)kernel];
  if (cur >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

inline int warps_per_block(size_t wbytes) {
  if (wbytes == 0) return kMaxWarpsPerBlock;
  return (int)std::max<size_t>(1, std::min<size_t>(kMaxWarpsPerBlock, kSmemBudget / wbytes));
}

// What one host-side pass over the plan launched: per-kind launch and unit
// counts, and CUDA-event pairs around the launches of the kinds in `mask`.
// When `capture` is set the events are recorded as external event nodes of a
// CUDA graph (they then fire on every replay).
struct EvPair { int kind; cudaEvent_t a, b; int64_t units = 0; };
struct Recorder {
  uint32_t mask = 0;
  bool capture = false;
  bool pdl = false;                    // launch with programmatic dependent launch (see pdl_entry)
  int64_t launches[TLQR_K_COUNT] = {}, units[TLQR_K_COUNT] = {};
  std::vector<EvPair> recs;
  std::vector<cudaEvent_t>* pool = nullptr;
  cudaEvent_t event() {
    if (pool && !pool->empty()) { cudaEvent_t e = pool->back(); pool->pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void record(cudaEvent_t e, cudaStream_t st) {
    if (capture) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
  }
};

// Per-factor accumulated profile.
struct Profiler {
  uint32_t mask = 0;
  int64_t launches[TLQR_K_COUNT] = {}, units[TLQR_K_COUNT] = {}, timed[TLQR_K_COUNT] = {};
  double ms[TLQR_K_COUNT] = {};
  std::vector<EvPair> pending;
  std::vector<char> pending_owned;
  std::vector<cudaEvent_t> pool;
  bool event_error = false;
  struct Launch { int kind; int64_t units; double ms; };
  std::vector<Launch> log;             // harvested timed launches, in launch order
  void add(const Recorder& r, bool owned) {
    for (int k = 0; k < TLQR_K_COUNT; ++k) { launches[k] += r.launches[k]; units[k] += r.units[k]; }
    for (const EvPair& p : r.recs) { pending.push_back(p); pending_owned.push_back(owned); }
  }
  // Read the events of completed launches (synchronises on them).
  void harvest() {
    for (size_t t = 0; t < pending.size(); ++t) {
      const EvPair& p = pending[t];
      float v = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&v, p.a, p.b) == cudaSuccess) {
        ms[p.kind] += v;
        timed[p.kind]++;
        if (log.size() < (1u << 20)) log.push_back(Launch{p.kind, p.units, (double)v});
      } else {
        event_error = true;
        cudaGetLastError();
      }
      if (pending_owned[t]) { pool.push_back(p.a); pool.push_back(p.b); }
    }
    pending.clear();
    pending_owned.clear();
  }
  ~Profiler() {
    for (size_t t = 0; t < pending.size(); ++t)
      if (pending_owned[t]) { cudaEventDestroy(pending[t].a); cudaEventDestroy(pending[t].b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// kernel<<<grid, block, smem, st>>>(args...), with programmatic stream
// serialisation when pdl is set: the kernel may be scheduled while its
// predecessor drains and waits for it on the device (pdl_entry), which hides
// the launch gap between the short kernels of a pass.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args... args) {
  if (!pdl) {
    kernel<<<grid, block, smem, st>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Launch `count` warps, each with `wbytes` of dynamic shared memory.
template <typename Kernel, typename... Args>
cudaError_t launch_warps(Recorder* rc, int kind, Kernel kernel, int count, size_t wbytes, cudaStream_t st,
                         Args... args) {
  if (count <= 0) return cudaSuccess;
  const int wpb = warps_per_block(wbytes);
  const size_t smem = wbytes * wpb;
  if (!(rc && rc->capture)) {
    cudaError_t e = ensure_smem(kernel, smem);
    if (e != cudaSuccess) return e;
  }
  const int blocks = (count + wpb - 1) / wpb;
  const bool timed = rc && (rc->mask >> kind) & 1u;
  EvPair ev{kind, nullptr, nullptr, count};
  if (timed) { ev.a = rc->event(); ev.b = rc->event(); rc->record(ev.a, st); }
  cudaError_t e = launch_k(rc && rc->pdl && !timed, kernel, blocks, 32 * wpb, smem, st, args...);
  if (timed) { rc->record(ev.b, st); rc->recs.push_back(ev); }
  if (rc) { rc->launches[kind]++; rc->units[kind] += count; }
  return e;
}

// An instantiated CUDA graph of one launch sequence, valid for one key (the
// pointers and flags it was captured with).
struct GraphCache {
  std::vector<uintptr_t> key;
  cudaGraphExec_t exec = nullptr;
  Recorder rec;                      // counts per replay and the graph's own events
  void clear() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    for (const EvPair& p : rec.recs) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    rec = Recorder{};
    key.clear();
  }
};

template <typename T>
T* dalloc(size_t count, cudaError_t* err) {
  if (count == 0) count = 1;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess && *err == cudaSuccess) *err = e;
  return (T*)p;
}

// Operation list of the level-asynchronous factorisation tail (fx::kf_async):
// the rakes, absorptions and compressions of rounds [r0, R) and then the
// expansions of those compressions in reverse round order, each with the
// operations whose outputs it reads:
//   rake of leaf j            <- last writer of U_j, last writer of edge slot j
//   absorption into i         <- all rakes of its segment (a counter), last writer of U_i
//   compression of j (i, k)   <- last writers of U_j, edge slot j, edge slot k
//   expansion of j            <- the compression of j (its tape), producer of P_k
//                                (the expansion of k, else the last writer of U_k)
// Writers before round r0 ran in earlier launches and are not waited for.
// Operations are sorted by dependency level (eq. earliest-level) and every run
// of one (level, kind) is padded to whole warps of `ops_per_warp` operations,
// so that a warp's operations share one code path and never depend on each
// other.
struct AsyncPlan {
  int r0 = 0, n_ops = 0, n_flags = 0, levels = 0;
  std::vector<int32_t> op, dep_flag, dep_target, signal;
};

AsyncPlan build_async(const tlqr_plan_t* P, int r0, int ops_per_warp) {
  AsyncPlan A;
  const int R = (int)P->rounds.size();
  A.r0 = r0;
  if (r0 >= R) return A;
  struct Op { int kind, idx, level; int dep[3]; int sig; };
  std::vector<Op> ops;
  const int N = P->N;
  std::vector<int> lastU(N, -1), lastE(N, -1), lastP(N, -1);
  const int seg0 = P->rounds[r0].seg_begin, seg1 = P->rounds[R - 1].seg_end;
  const int nseg = seg1 - seg0;
  std::vector<int> seg_level(nseg, 0), seg_size(nseg, 0);
  std::vector<int> comp_op(P->comp_j.size(), -1);
  auto level_of = [&](const Op& o) {
    int l = 0;
    for (int d : o.dep) {
      if (d >= 0) l = std::max(l, ops[d].level);
      else if (d <= -2) l = std::max(l, seg_level[-2 - d]);
    }
    return l + 1;
  };
  for (int r = r0; r < R; ++r) {
    const tlqr_round& rd = P->rounds[r];
    for (int s = rd.seg_begin; s < rd.seg_end; ++s) {
      for (int rr = P->seg_start[s]; rr < P->seg_start[s + 1]; ++rr) {
        const int j = P->rake_leaf[rr];
        Op o{fx::AK_RAKE, rr, 0, {lastU[j], lastE[j], -1}, s - seg0};
        o.level = level_of(o);
        seg_level[s - seg0] = std::max(seg_level[s - seg0], o.level);
        seg_size[s - seg0]++;
        ops.push_back(o);
      }
    }
    for (int s = rd.seg_begin; s < rd.seg_end; ++s) {
      const int i = P->seg_parent[s];
      Op o{fx::AK_ABSORB, s, 0, {-2 - (s - seg0), lastU[i], -1}, -1};
      o.level = level_of(o);
      lastU[i] = (int)ops.size();
      ops.push_back(o);
    }
    for (int c = rd.comp_begin; c < rd.comp_end; ++c) {
      const int j = P->comp_j[c], k = P->comp_k[c];
      Op o{fx::AK_COMPRESS, c, 0, {lastU[j], lastE[j], lastE[k]}, -1};
      o.level = level_of(o);
      comp_op[c] = (int)ops.size();
      lastE[k] = lastE[j] = (int)ops.size();
      ops.push_back(o);
    }
  }
  for (int r = R - 1; r >= r0; --r) {
    const tlqr_round& rd = P->rounds[r];
    for (int c = rd.comp_begin; c < rd.comp_end; ++c) {
      const int j = P->comp_j[c], k = P->comp_k[c];
      Op o{fx::AK_EXPAND, c, 0, {comp_op[c], lastP[k] >= 0 ? lastP[k] : lastU[k], -1}, -1};
      o.level = level_of(o);
      lastP[j] = (int)ops.size();
      ops.push_back(o);
    }
  }
  std::vector<int> order(ops.size());
  for (size_t t = 0; t < ops.size(); ++t) order[t] = (int)t;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return ops[a].level != ops[b].level ? ops[a].level < ops[b].level : ops[a].kind < ops[b].kind;
  });
  std::vector<int> pos_of(ops.size(), -1);
  std::vector<int> slot_op;                                  // op id per position, -1 = padding
  for (size_t t = 0; t < order.size(); ++t) {
    const Op& o = ops[order[t]];
    if (t > 0) {
      const Op& prev = ops[order[t - 1]];
      if (prev.level != o.level || prev.kind != o.kind)
        while (slot_op.size() % ops_per_warp) slot_op.push_back(-1);
    }
    pos_of[order[t]] = (int)slot_op.size();
    slot_op.push_back(order[t]);
    A.levels = std::max(A.levels, o.level);
  }
  while (slot_op.size() % ops_per_warp) slot_op.push_back(-1);
  A.n_ops = (int)slot_op.size();
  A.n_flags = A.n_ops + nseg;
  A.op.assign(A.n_ops, 0);
  A.dep_flag.assign(3 * (size_t)A.n_ops, -1);
  A.dep_target.assign(3 * (size_t)A.n_ops, 0);
  A.signal.assign(A.n_ops, -1);
  int last_kind = 0;
  for (int p = 0; p < A.n_ops; ++p) {
    const int id = slot_op[p];
    if (id < 0) {                                            // padding: the kind of its run
      A.op[p] = (last_kind << 28) | fx::kAsyncPad;
      continue;
    }
    const Op& o = ops[id];
    last_kind = o.kind;
    A.op[p] = (o.kind << 28) | o.idx;
    for (int d = 0; d < 3; ++d) {
      if (o.dep[d] >= 0) {
        A.dep_flag[3 * (size_t)p + d] = pos_of[o.dep[d]];
        A.dep_target[3 * (size_t)p + d] = 1;
      } else if (o.dep[d] <= -2) {
        A.dep_flag[3 * (size_t)p + d] = A.n_ops + (-2 - o.dep[d]);
        A.dep_target[3 * (size_t)p + d] = seg_size[-2 - o.dep[d]];
      }
    }
    if (o.sig >= 0) A.signal[p] = A.n_ops + o.sig;
  }
  return A;
}

// Operation list of the level-asynchronous state pass (fx::kf_async_vec, state
// kinds): the offset compositions b_k <- Tr_j b_j + b_k of every compression in
// forward round order, then per round in reverse order the state expansions
// x_j = T_j x_i + b_j of the compressed centres and of the raked leaves.
//   composition of j (into k)   <- last writers of b_j and b_k
//   expansion of j (from i)     <- last writer of b_j, the expansion that wrote x_i
// (b comes from the local solve and x of a root from the root solve, both in
// earlier launches).  Sorted and padded as build_async.
AsyncPlan build_async_state(const tlqr_plan_t* P, int ops_per_warp) {
  AsyncPlan A;
  const int R = (int)P->rounds.size();
  A.r0 = 0;
  if (R == 0) return A;
  struct Op { int kind, idx, level; int dep[2]; };
  std::vector<Op> ops;
  const int N = P->N;
  std::vector<int> lastB(N, -1), lastX(N, -1);
  auto level_of = [&](const Op& o) {
    int l = 0;
    for (int d : o.dep) if (d >= 0) l = std::max(l, ops[d].level);
    return l + 1;
  };
  for (int r = 0; r < R; ++r) {
    const tlqr_round& rd = P->rounds[r];
    for (int c = rd.comp_begin; c < rd.comp_end; ++c) {
      const int j = P->comp_j[c], k = P->comp_k[c];
      Op o{fx::SK_COMPOSE, c, 0, {lastB[j], lastB[k]}};
      o.level = level_of(o);
      lastB[k] = (int)ops.size();
      ops.push_back(o);
    }
  }
  for (int r = R - 1; r >= 0; --r) {
    const tlqr_round& rd = P->rounds[r];
    for (int c = rd.comp_begin; c < rd.comp_end; ++c) {
      const int j = P->comp_j[c], i = P->comp_i[c];
      Op o{fx::SK_EXPAND_C, c, 0, {lastB[j], lastX[i]}};
      o.level = level_of(o);
      lastX[j] = (int)ops.size();
      ops.push_back(o);
    }
    for (int t = rd.rake_begin; t < rd.rake_end; ++t) {
      const int j = P->rake_leaf[t], i = P->rake_parent[t];
      Op o{fx::SK_EXPAND_R, t, 0, {lastB[j], lastX[i]}};
      o.level = level_of(o);
      lastX[j] = (int)ops.size();
      ops.push_back(o);
    }
  }
  std::vector<int> order(ops.size());
  for (size_t t = 0; t < ops.size(); ++t) order[t] = (int)t;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return ops[a].level != ops[b].level ? ops[a].level < ops[b].level : ops[a].kind < ops[b].kind;
  });
  std::vector<int> pos_of(ops.size(), -1), slot_op;
  for (size_t t = 0; t < order.size(); ++t) {
    const Op& o = ops[order[t]];
    if (t > 0) {
      const Op& prev = ops[order[t - 1]];
      if (prev.level != o.level || prev.kind != o.kind)
        while (slot_op.size() % ops_per_warp) slot_op.push_back(-1);
    }
    pos_of[order[t]] = (int)slot_op.size();
    slot_op.push_back(order[t]);
    A.levels = std::max(A.levels, o.level);
  }
  while (slot_op.size() % ops_per_warp) slot_op.push_back(-1);
  A.n_ops = (int)slot_op.size();
  A.n_flags = A.n_ops;
  A.op.assign(A.n_ops, 0);
  A.dep_flag.assign(3 * (size_t)A.n_ops, -1);
  A.dep_target.assign(3 * (size_t)A.n_ops, 0);
  A.signal.assign(A.n_ops, -1);
  int last_kind = 0;
  for (int p = 0; p < A.n_ops; ++p) {
    const int id = slot_op[p];
    if (id < 0) { A.op[p] = (last_kind << 28) | fx::kAsyncPad; continue; }
    const Op& o = ops[id];
    last_kind = o.kind;
    A.op[p] = (o.kind << 28) | o.idx;
    for (int d = 0; d < 2; ++d)
      if (o.dep[d] >= 0) {
        A.dep_flag[3 * (size_t)p + d] = pos_of[o.dep[d]];
        A.dep_target[3 * (size_t)p + d] = 1;
      }
  }
  return A;
}

// Solve-pass vectors of a panel of right-hand sides ([nrhs][..] each).
struct PanelBufs {
  void *h = nullptr, *z = nullptr, *s = nullptr, *cv = nullptr, *bv = nullptr, *kv = nullptr, *xs = nullptr;
};

// One level-asynchronous operation list on the device.
struct DevAsync {
  AsyncPlan plan;                  // host copy; plan.n_ops == 0: not used
  int *op = nullptr, *dep_flag = nullptr, *dep_target = nullptr, *signal = nullptr;
  int* flags = nullptr;            // [n_flags] flags, then the work counter and the abort word
  int blocks = 0;                  // persistent grid
};

struct DevPlan {
  int *rake_leaf = nullptr, *rake_parent = nullptr, *seg_parent = nullptr, *seg_start = nullptr;
  int *comp_j = nullptr, *comp_i = nullptr, *comp_k = nullptr;
  int *parent = nullptr, *child_start = nullptr, *child_list = nullptr;
  int* tree = nullptr;           // forest only: tree ordinal of each node
};

}  // namespace

struct tlqr_factor_t {
  const tlqr_plan_t* plan = nullptr;
  tlqr_options opt{};
  int device = 0;
  size_t ts = 8;                 // bytes per factor element
  DevPlan dp;
  std::vector<void*> allocs;
  // factor workspace (typed by precision)
  void *U = nullptr, *Ea = nullptr, *Ec = nullptr, *Ep = nullptr, *contrib = nullptr;
  void *K = nullptr, *Tm = nullptr, *Tr = nullptr, *W = nullptr, *Finv = nullptr, *LG = nullptr;
  void *h = nullptr, *z = nullptr, *s = nullptr, *cv = nullptr, *bv = nullptr, *kv = nullptr, *xs = nullptr;
  unsigned char* dflag = nullptr;
  int* status = nullptr;
  // FP64 residual buffers and staging for host-memory calls
  double *res_x = nullptr, *res_u = nullptr, *res_c = nullptr;
  // MIXED: (hi, lo) FP32 splits of x, u, y for the float-float residual
  float *xh = nullptr, *xl = nullptr, *uh = nullptr, *ul = nullptr, *yh = nullptr, *yl = nullptr;
  // MIXED with compile-time (n, m): the node-organised residual's child messages
  float *rwh = nullptr, *rwl = nullptr, *rwk = nullptr;
  unsigned long long* maxes = nullptr;
  unsigned long long* h_maxes = nullptr;   // pinned mirror
  double* d_gate = nullptr;                 // speculative refinement: [0] eta of the first residual
  double* h_gate = nullptr;                 // pinned mirror
  bool speculate = false;                   // the last mixed solve needed a refinement step
  int* h_status = nullptr;                  // pinned mirror
  double* stage = nullptr;                  // FP64 staging (host-memory calls), lazily allocated
  double* upd = nullptr;                    // diagonal increments of tlqr_update_solve (when the staged P is too small)
  double* redo_scratch = nullptr;           // FP64 re-solve slots (see fixed.cuh, kSolveRatio)
  int redo_cap = 0;
  size_t redo_slot = 0;
  size_t arena_bytes = 0;                   // the one device allocation holding plan arrays + workspace
  size_t stage_elems = 0;
  // problem pointers of the last factorisation (device), for refinement/residual
  tlqr_problem dprob{};
  bool factored = false;
  tlqr_info info{};
  Profiler prof;
  // CUDA graphs of the launch sequences (factor, up to four solves, residual)
  GraphCache g_factor, g_solve[4], g_resid[2];
  int solve_lru = 0;
  bool graphs_broken = false;      // a capture failed once: launch directly from then on
  // own non-blocking work stream (capturable), fenced to the caller's stream
  cudaStream_t work = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int fixed_n = 0;                 // n of the fixed-dimension kernels in use (0 = run-time n)
  int fixed_m = 0;                 // m of the fixed (n, m) kernels in use (0 = run-time m)
  fx::RoundDesc* d_rounds = nullptr;  // device copy of the plan's rounds
  int sms = 0;                     // streaming multiprocessors of the factor's device
  int tail_r0 = 0;                 // first round handled by the single-block tail kernels
  // level-asynchronous launches (compile-time-n kernels only): the factorisation
  // tail, and the affine and state passes of every right-hand side
  DevAsync fa, aa, sa;
  // panel solves: vectors for up to kPanel right-hand sides (one lazy allocation)
  PanelBufs panel;
  void* panel_mem = nullptr;

  template <typename T>
  Ws<T> ws(const tlqr_problem& p) const {
    Ws<T> w{};
    const tlqr_plan_t* P = plan;
    w.N = P->N; w.n = opt.n; w.m = opt.m;
    w.has_M = opt.has_M; w.has_delta = opt.has_delta;
    w.Q = p.Q; w.M = p.M; w.R = p.R; w.A = p.A; w.B = p.B; w.Delta = p.Delta;
    w.q = p.q; w.r = p.r; w.c = p.c;
    w.rake_leaf = dp.rake_leaf; w.rake_parent = dp.rake_parent; w.seg_parent = dp.seg_parent;
    w.seg_start = dp.seg_start; w.comp_j = dp.comp_j; w.comp_i = dp.comp_i; w.comp_k = dp.comp_k;
    w.parent = dp.parent; w.child_start = dp.child_start; w.child_list = dp.child_list;
    w.U = (T*)U; w.Ea = (T*)Ea; w.Ec = (T*)Ec; w.Ep = (T*)Ep; w.contrib = (T*)contrib;
    w.K = (T*)K; w.Tm = (T*)Tm; w.Tr = (T*)Tr; w.W = (T*)W; w.Finv = (T*)Finv; w.LG = (T*)LG;
    w.dflag = dflag;
    w.h = (T*)h; w.z = (T*)z; w.s = (T*)s; w.cv = (T*)cv; w.bv = (T*)bv; w.kv = (T*)kv; w.xs = (T*)xs;
    w.status = status;
    w.redo_count = redo_scratch ? status + 1 : nullptr;
    w.redo_cap = redo_cap;
    w.redo_scratch = redo_scratch;
    w.redo_slot = redo_slot;
    w.nrhs = 1;
    w.sv = (size_t)P->N * opt.n;
    w.sm = (size_t)P->N * opt.m;
    w.scv = std::max<size_t>(1, P->rake_leaf.size()) * opt.n;
    return w;
  }
  ~tlqr_factor_t() {
    if (work) cudaStreamSynchronize(work);
    g_factor.clear();
    for (auto& g : g_solve) g.clear();
    for (auto& g : g_resid) g.clear();
    for (void* p : allocs) cudaFree(p);
    if (panel_mem) cudaFree(panel_mem);
    if (h_maxes) cudaFreeHost(h_maxes);
    if (h_gate) cudaFreeHost(h_gate);
    if (h_status) cudaFreeHost(h_status);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (work) cudaStreamDestroy(work);
  }
};

namespace {
// All work of a public call runs on the factor's own stream, ordered after
// the caller's stream on entry; on exit the caller's stream waits for it.
struct StreamScope {
  tlqr_factor_t* f;
  cudaStream_t user;
  cudaStream_t st;
  StreamScope(tlqr_factor_t* f_, void* stream) : f(f_), user((cudaStream_t)stream), st(f_->work) {
    cudaEventRecord(f->ev_in, user);
    cudaStreamWaitEvent(st, f->ev_in, 0);
  }
  ~StreamScope() {
    cudaEventRecord(f->ev_out, st);
    cudaStreamWaitEvent(user, f->ev_out, 0);
  }
};
}  // namespace

namespace {

int map_status(int st) {
  switch (st) {
    case ST_OK: return TLQR_OK;
    case ST_NOT_PD: return TLQR_ERR_NOT_PD;
    case ST_SINGULAR: return TLQR_ERR_SINGULAR;
    case ST_NONFINITE: return TLQR_ERR_NONFINITE;
    case ST_TIMEOUT: return TLQR_ERR_TIMEOUT;
    default: return TLQR_ERR_CUDA;
  }
}

// Device memory of a factor object: the plan's arrays and the whole workspace
// are carved from one allocation (one cudaMalloc and one cudaFree per factor,
// so that creating and destroying factors does not fragment memory or
// serialise the device more than once).  A pass with base == nullptr only
// sizes the layout.
struct Carve {
  unsigned char* base = nullptr;
  size_t off = 0;
  void* take(size_t bytes) {
    const size_t o = (off + 255) & ~size_t(255);
    off = o + std::max<size_t>(bytes, 1);
    return base ? base + o : nullptr;
  }
  template <typename T>
  T* take(size_t elems, size_t es) { return reinterpret_cast<T*>(take(elems * es)); }
};

std::vector<int32_t> round_table(const tlqr_plan_t* P) {
  std::vector<int32_t> rd;
  for (const tlqr_round& r : P->rounds)
    rd.insert(rd.end(), {r.rake_begin, r.rake_end, r.seg_begin, r.seg_end, r.comp_begin, r.comp_end});
  return rd;
}

// Assign (or size) every device pointer of f.
void carve_factor(tlqr_factor_t* f, Carve& c) {
  const tlqr_plan_t* P = f->plan;
  auto ints = [&](const std::vector<int32_t>& v) { return c.take<int>(v.size(), sizeof(int)); };
  f->dp.rake_leaf = ints(P->rake_leaf);
  f->dp.rake_parent = ints(P->rake_parent);
  f->dp.seg_parent = ints(P->seg_parent);
  f->dp.seg_start = ints(P->seg_start);
  f->dp.comp_j = ints(P->comp_j);
  f->dp.comp_i = ints(P->comp_i);
  f->dp.comp_k = ints(P->comp_k);
  f->dp.parent = ints(P->parent);
  f->dp.child_start = ints(P->child_start);
  f->dp.child_list = ints(P->child_list);
  f->dp.tree = P->n_trees > 1 ? ints(P->tree_of) : nullptr;
  f->d_rounds = reinterpret_cast<fx::RoundDesc*>(c.take<int>(6 * P->rounds.size(), sizeof(int)));
  for (DevAsync* d : {&f->fa, &f->aa, &f->sa}) {
    if (d->plan.n_ops == 0) continue;
    d->op = ints(d->plan.op);
    d->dep_flag = ints(d->plan.dep_flag);
    d->dep_target = ints(d->plan.dep_target);
    d->signal = ints(d->plan.signal);
    d->flags = c.take<int>((size_t)d->plan.n_flags + 2, sizeof(int));
  }
  const size_t N = P->N, n = f->opt.n, m = f->opt.m, nn = n * n, nm = n * m, mm = m * m;
  const size_t nrake = std::max<size_t>(1, P->rake_leaf.size());
  const size_t ts = f->ts;
  f->U = c.take(N * nn * ts); f->Ea = c.take(N * nn * ts); f->Ec = c.take(N * nn * ts); f->Ep = c.take(N * nn * ts);
  f->contrib = c.take(nrake * nn * ts);
  f->K = c.take(N * nm * ts); f->Tm = c.take(N * nn * ts); f->Tr = c.take(N * nn * ts);
  f->LG = c.take(N * mm * ts);
  f->W = f->Finv = nullptr;
  if (f->opt.has_delta) { f->W = c.take(N * nn * ts); f->Finv = c.take(N * nn * ts); }
  f->h = c.take(N * n * ts); f->z = c.take(N * n * ts); f->s = c.take(N * n * ts); f->cv = c.take(nrake * n * ts);
  f->bv = c.take(N * n * ts); f->kv = c.take(N * m * ts); f->xs = c.take(N * n * ts);
  f->dflag = c.take<unsigned char>(N, 1);
  f->status = c.take<int>(2, sizeof(int));          // [0] status word, [1] FP64 re-solve tickets
  f->redo_scratch = nullptr;
  f->redo_cap = 0;
  f->redo_slot = 0;
  if (f->ts == 4 && f->fixed_n > 0 && f->opt.fp64_resolve >= 0) {
    f->redo_cap = kRedoCap;
    f->redo_slot = 3 * nn;                              // S (n x n) and a right-hand side of up to 2n columns
    f->redo_scratch = c.take<double>((size_t)f->redo_cap * f->redo_slot, 8);
  }
  f->res_x = c.take<double>(N * n, 8); f->res_u = c.take<double>(N * m, 8); f->res_c = c.take<double>(N * n, 8);
  f->maxes = c.take<unsigned long long>(4 * (size_t)P->n_trees, 8);
  f->d_gate = c.take<double>(2, 8);
  f->xh = f->xl = f->uh = f->ul = f->yh = f->yl = nullptr;
  f->rwh = f->rwl = f->rwk = nullptr;
  if (f->opt.precision == TLQR_PREC_MIXED) {
    f->xh = c.take<float>(N * n, 4); f->xl = c.take<float>(N * n, 4);
    f->uh = c.take<float>(N * m, 4); f->ul = c.take<float>(N * m, 4);
    f->yh = c.take<float>(N * n, 4); f->yl = c.take<float>(N * n, 4);
    f->rwh = c.take<float>(N * n, 4); f->rwl = c.take<float>(N * n, 4); f->rwk = c.take<float>(N * n, 4);
  }
}

// Copy the plan's arrays into their carved slots and pick the tail rounds.
int upload_plan(tlqr_factor_t* f) {
  const tlqr_plan_t* P = f->plan;
  cudaError_t err = cudaSuccess;
  auto up = [&](const std::vector<int32_t>& v, int* dst) {
    if (err == cudaSuccess && !v.empty() && dst)
      err = cudaMemcpy(dst, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice);
  };
  up(P->rake_leaf, f->dp.rake_leaf);
  up(P->rake_parent, f->dp.rake_parent);
  up(P->seg_parent, f->dp.seg_parent);
  up(P->seg_start, f->dp.seg_start);
  up(P->comp_j, f->dp.comp_j);
  up(P->comp_i, f->dp.comp_i);
  up(P->comp_k, f->dp.comp_k);
  up(P->parent, f->dp.parent);
  up(P->child_start, f->dp.child_start);
  up(P->child_list, f->dp.child_list);
  if (P->n_trees > 1) up(P->tree_of, f->dp.tree);
  up(round_table(P), reinterpret_cast<int*>(f->d_rounds));
  for (DevAsync* d : {&f->fa, &f->aa, &f->sa}) {
    if (d->plan.n_ops == 0) continue;
    up(d->plan.op, d->op);
    up(d->plan.dep_flag, d->dep_flag);
    up(d->plan.dep_target, d->dep_target);
    up(d->plan.signal, d->signal);
  }
  // tail: the longest suffix of rounds whose phases each hold at most tail_ops operations
  const int R = (int)P->rounds.size();
  const int tail_ops = f->opt.tail_ops > 0 ? f->opt.tail_ops : f->opt.tail_ops < 0 ? 0 : kTailOps;
  f->tail_r0 = R;
  while (tail_ops > 0 && f->tail_r0 > 0) {
    const tlqr_round& r = P->rounds[f->tail_r0 - 1];
    const int mx = std::max({r.rake_end - r.rake_begin, r.seg_end - r.seg_begin, r.comp_end - r.comp_begin});
    if (mx > tail_ops) break;
    --f->tail_r0;
  }
  if (err != cudaSuccess) return TLQR_ERR_CUDA;
  return TLQR_OK;
}

// Launch `count` operations of a fixed-dimension kernel: groups of G lanes,
// 128-thread blocks, `gbytes` of shared memory per group.
template <typename Kernel, typename... Args>
cudaError_t launch_groups(Recorder* rc, int kind, Kernel kernel, int count, int G, size_t gbytes, cudaStream_t st,
                          Args... args) {
  if (count <= 0) return cudaSuccess;
  constexpr int threads = 128;
  const int gpb = threads / G;
  const size_t smem = gbytes * gpb;
  if (!(rc && rc->capture)) {
    cudaError_t e = ensure_smem(kernel, smem);
    if (e != cudaSuccess) return e;
  }
  const int blocks = (count + gpb - 1) / gpb;
  const bool timed = rc && (rc->mask >> kind) & 1u;
  EvPair ev{kind, nullptr, nullptr, count};
  if (timed) { ev.a = rc->event(); ev.b = rc->event(); rc->record(ev.a, st); }
  cudaError_t e = launch_k(rc && rc->pdl && !timed, kernel, blocks, threads, smem, st, args...);
  if (timed) { rc->record(ev.b, st); rc->recs.push_back(ev); }
  if (rc) { rc->launches[kind]++; rc->units[kind] += count; }
  return e;
}

// One block of kTailThreads threads runs the tail rounds of a pass.
template <typename Kernel, typename... Args>
cudaError_t launch_tail(Recorder* rc, int kind, Kernel kernel, cudaStream_t st, Args... args) {
  const bool timed = rc && (rc->mask >> kind) & 1u;
  EvPair ev{kind, nullptr, nullptr, 1};
  if (timed) { ev.a = rc->event(); ev.b = rc->event(); rc->record(ev.a, st); }
  cudaError_t e = launch_k(rc && rc->pdl && !timed, kernel, 1, kTailThreads, 0, st, args...);
  if (timed) { rc->record(ev.b, st); rc->recs.push_back(ev); }
  if (rc) { rc->launches[kind]++; rc->units[kind] += 1; }
  return e;
}

cudaError_t launch_split(Recorder* rc, const SplitList& L, int sms, cudaStream_t st) {
  const int blocks = sms * 4, threads = 256;
  k_split_ff<<<blocks, threads, 0, st>>>(L);
  cudaError_t e = cudaGetLastError();
  if (rc) { rc->launches[TLQR_K_RESIDUAL]++; }
  return e;
}

// One persistent launch of a level-asynchronous operation list: reset its
// flags, counter and abort word, then run `kernel` (kf_async for the
// factorisation tail, kf_async_vec for a right-hand-side pass).
template <typename T, int N, typename Kernel>
cudaError_t launch_async(tlqr_factor_t* f, Recorder* rc, int kind, Kernel kernel, const DevAsync& d, size_t smem,
                         const Ws<T>& w, cudaStream_t st) {
  const AsyncPlan& A = d.plan;
  cudaError_t e = cudaMemsetAsync(d.flags, 0, ((size_t)A.n_flags + 2) * sizeof(int), st);
  if (e) return e;
  fx::AsyncArgs a{};
  a.op = d.op; a.dep_flag = d.dep_flag; a.dep_target = d.dep_target; a.signal = d.signal;
  a.flags = d.flags; a.counter = d.flags + A.n_flags; a.abort = d.flags + A.n_flags + 1;
  a.n_ops = A.n_ops;
  a.spin_limit = f->opt.spin_limit > 0 ? f->opt.spin_limit : kSpinLimit;
  a.withhold = ((f->opt.test_withhold & 1) && &d == &f->fa) ? 0 : -1;
  constexpr int gpb = 128 / fx::D<T, N>::G;
  if (!(rc && rc->capture) && smem > 0 && (e = ensure_smem(kernel, smem))) return e;
  const int blocks = std::max(1, std::min((A.n_ops + gpb - 1) / gpb, d.blocks));
  const bool timed = rc && (rc->mask >> kind) & 1u;
  EvPair ev{kind, nullptr, nullptr, A.n_ops};
  if (timed) { ev.a = rc->event(); ev.b = rc->event(); rc->record(ev.a, st); }
  e = launch_k(rc && rc->pdl && !timed, kernel, blocks, 128, smem, st, w, a);
  if (timed) { rc->record(ev.b, st); rc->recs.push_back(ev); }
  if (rc) { rc->launches[kind]++; rc->units[kind] += A.n_ops; }
  return e;
}

// Factorisation sequence (Alg. 1 steps 2-3).  NF = compile-time n of the
// fixed-dimension kernels, 0 = the run-time-n kernels.
template <typename T, int NF, int MF>
cudaError_t run_factor(tlqr_factor_t* f, Recorder* rc, const tlqr_problem& p, cudaStream_t st) {
  const tlqr_plan_t* P = f->plan;
  const Ws<T> w = f->ws<T>(p);
  const WarpBytes wb = warp_bytes(f->opt.n, f->opt.m, sizeof(T));
  constexpr int NX = NF > 0 ? NF : 4;          // placeholder dimension when NF == 0 (never launched)
  constexpr int MX = MF > 0 ? MF : 2;
  constexpr int G = fx::D<T, NX>::G;
  cudaError_t e;
  if ((e = cudaMemsetAsync(f->status, 0, 2 * sizeof(int), st))) return e;
  if constexpr (MF > 0) {
    if ((e = launch_groups(rc, TLQR_K_CONDENSE, fx::kf_condense<T, NX, MX>, P->N, G, fx::CondSmem<T, NX, MX>::bytes,
                           st, w, P->N))) return e;
  } else if ((e = launch_warps(rc, TLQR_K_CONDENSE, k_condense<T>, P->N, wb.condense, st, w, (int)wb.condense))) {
    return e;
  }
  const int R = (int)P->rounds.size();
  // rounds [RA, R) and their expansions run in the level-asynchronous kernel
  const int RA = (NF > 0 && f->fa.plan.n_ops > 0) ? f->fa.plan.r0 : R;
  for (int ri = 0; ri < RA; ++ri) {
    const tlqr_round& rd = P->rounds[ri];
    const int nr = rd.rake_end - rd.rake_begin, ns = rd.seg_end - rd.seg_begin, nc = rd.comp_end - rd.comp_begin;
    if constexpr (NF > 0) {
      if ((e = launch_groups(rc, TLQR_K_RAKE, fx::kf_rake<T, NX>, nr, G, fx::TauSmem<T, NX>::bytes, st, w,
                             rd.rake_begin, nr))) return e;
    } else if ((e = launch_warps(rc, TLQR_K_RAKE, k_rake<T>, nr, wb.tau, st, w, rd.rake_begin, nr, (int)wb.tau))) {
      return e;
    }
    if ((e = launch_warps(rc, TLQR_K_ABSORB, k_absorb<T>, ns, 0, st, w, rd.seg_begin, ns))) return e;
    if constexpr (NF > 0) {
      if ((e = launch_groups(rc, TLQR_K_COMPRESS, fx::kf_compress<T, NX>, nc, G, fx::CompSmem<T, NX>::bytes, st, w,
                             rd.comp_begin, nc))) return e;
    } else if ((e = launch_warps(rc, TLQR_K_COMPRESS, k_compress<T>, nc, wb.compress, st, w, rd.comp_begin, nc,
                                 (int)wb.compress))) {
      return e;
    }
  }
  if constexpr (NF > 0) {
    if (RA < R && (e = launch_async<T, NX>(f, rc, TLQR_K_FACTOR_TAIL, fx::kf_async<T, NX>, f->fa,
                                            (size_t)fx::AsyncSmem<T, NX>::bytes * (128 / G), w, st)))
      return e;
  }
  for (int ri = RA - 1; ri >= 0; --ri) {
    const tlqr_round* it = &P->rounds[ri];
    const int nc = it->comp_end - it->comp_begin;
    if constexpr (NF > 0) {
      if ((e = launch_groups(rc, TLQR_K_EXPAND, fx::kf_expand<T, NX>, nc, G, fx::TauSmem<T, NX>::bytes, st, w,
                             it->comp_begin, nc))) return e;
    } else if ((e = launch_warps(rc, TLQR_K_EXPAND, k_expand<T>, nc, wb.tau, st, w, it->comp_begin, nc, (int)wb.tau))) {
      return e;
    }
  }
  if constexpr (MF > 0) {
    if ((e = launch_groups(rc, TLQR_K_LOCAL_FACTOR, fx::kf_local_factor<T, NX, MX>, P->N, G,
                           fx::LfSmem<T, NX, MX>::bytes, st, w, P->N))) return e;
  } else if ((e = launch_warps(rc, TLQR_K_LOCAL_FACTOR, k_local_factor<T>, P->N, wb.local_factor, st, w,
                               (int)wb.local_factor))) {
    return e;
  }
  for (int ri = 0; ri < R; ++ri) {
    const tlqr_round& rd = P->rounds[ri];
    const int nc = rd.comp_end - rd.comp_begin;
    if constexpr (NF > 0) {
      if ((e = launch_groups(rc, TLQR_K_COMPOSE_T, fx::kf_compose_T<T, NX>, nc, G, fx::ComposeSmem<T, NX>::bytes, st,
                             w, rd.comp_begin, nc))) return e;
    } else if ((e = launch_warps(rc, TLQR_K_COMPOSE_T, k_compose_T<T>, nc, wb.compose_T, st, w, rd.comp_begin, nc,
                                 (int)wb.compose_T))) {
      return e;
    }
  }
  return cudaSuccess;
}

// Right-hand-side sequence (Alg. 1 steps 4-6).
template <typename T, int NF, int MF>
cudaError_t run_solve(tlqr_factor_t* f, Recorder* rc, const double* q, const double* r, const double* c,
                      double* x, double* u, double* y, int accumulate, cudaStream_t st, int nrhs = 1,
                      const PanelBufs* pb = nullptr) {
  const tlqr_plan_t* P = f->plan;
  tlqr_problem p = f->dprob;
  p.q = q; p.r = r; p.c = c;
  Ws<T> w = f->ws<T>(p);
  if (pb) {                                   // a panel: nrhs right-hand sides, [nrhs][..] vectors
    w.nrhs = nrhs;
    w.h = (T*)pb->h; w.z = (T*)pb->z; w.s = (T*)pb->s; w.cv = (T*)pb->cv;
    w.bv = (T*)pb->bv; w.kv = (T*)pb->kv; w.xs = (T*)pb->xs;
  }
  const WarpBytes wb = warp_bytes(f->opt.n, f->opt.m, sizeof(T));
  constexpr int NX = NF > 0 ? NF : 4;
  constexpr int MX = MF > 0 ? MF : 2;
  constexpr int G = fx::D<T, NX>::G;
  cudaError_t e;
  if constexpr (MF > 0) {
    if ((e = launch_groups(rc, TLQR_K_AFF_INIT, fx::kf_aff_init<T, NX, MX>, P->N, G, fx::AiSmem<T, NX, MX>::bytes, st, w, P->N))) return e;
  } else if ((e = launch_warps(rc, TLQR_K_AFF_INIT, k_aff_init<T>, P->N, wb.aff_init, st, w, (int)wb.aff_init))) {
    return e;
  }
  auto local_solve = [&]() -> cudaError_t {
    if constexpr (MF > 0)
      return launch_groups(rc, TLQR_K_LOCAL_SOLVE, fx::kf_local_solve<T, NX, MX>, P->N, G,
                           fx::LsSmem<T, NX, MX>::bytes, st, w, P->N);
    return launch_warps(rc, TLQR_K_LOCAL_SOLVE, k_local_solve<T>, P->N, wb.local_solve, st, w, (int)wb.local_solve);
  };
  auto recover = [&]() -> cudaError_t {
    if constexpr (MF > 0)
      return launch_groups(rc, TLQR_K_RECOVER, fx::kf_recover<T, NX, MX>, P->N, G, 0, st, w, x, u, y, accumulate,
                           P->N);
    return launch_warps(rc, TLQR_K_RECOVER, k_recover<T>, P->N, wb.recover, st, w, x, u, y, accumulate,
                        (int)wb.recover);
  };
  if constexpr (NF > 0) {
    if (f->aa.plan.n_ops > 0) {
      // every round of the affine pass in one level-asynchronous launch, the local
      // solves, every round of the state pass in a second one, the recovery
      if ((e = launch_async<T, NX>(f, rc, TLQR_K_AFF_TAIL, fx::kf_async_vec<T, NX>, f->aa, 0, w, st))) return e;
      if ((e = local_solve())) return e;
      if ((e = launch_async<T, NX>(f, rc, TLQR_K_STATE_TAIL, fx::kf_async_vec<T, NX>, f->sa, 0, w, st))) return e;
      return recover();
    }
  }
  const int R = (int)P->rounds.size();
  const int r_tail = NF > 0 ? f->tail_r0 : R;     // rounds [r_tail, R) run in the tail kernel
  for (int ri = 0; ri < r_tail; ++ri) {
    const tlqr_round& rd = P->rounds[ri];
    const int nr = rd.rake_end - rd.rake_begin, ns = rd.seg_end - rd.seg_begin, nc = rd.comp_end - rd.comp_begin;
    if constexpr (NF > 0) {
      if ((e = launch_groups(rc, TLQR_K_AFF_RAKE, fx::kf_aff_rake<T, NX>, nr, G, 0, st, w, rd.rake_begin, nr))) return e;
    } else if ((e = launch_warps(rc, TLQR_K_AFF_RAKE, k_aff_rake<T>, nr, wb.vec1, st, w, rd.rake_begin, nr,
                                 (int)wb.vec1))) {
      return e;
    }
    if constexpr (NF > 0) {
      if ((e = launch_groups(rc, TLQR_K_AFF_ABSORB, fx::kf_aff_absorb<T, NX>, ns, G, 0, st, w, rd.seg_begin, ns)))
        return e;
    } else if ((e = launch_warps(rc, TLQR_K_AFF_ABSORB, k_aff_absorb<T>, ns, 0, st, w, rd.seg_begin, ns))) {
      return e;
    }
    if constexpr (NF > 0) {
      if ((e = launch_groups(rc, TLQR_K_AFF_COMPRESS, fx::kf_aff_compress<T, NX>, nc, G, 0, st, w, rd.comp_begin,
                             nc))) return e;
    } else if ((e = launch_warps(rc, TLQR_K_AFF_COMPRESS, k_aff_compress<T>, nc, wb.vec1, st, w, rd.comp_begin, nc,
                                 (int)wb.vec1))) {
      return e;
    }
  }
  if constexpr (NF > 0) {
    if (r_tail < R && (e = launch_tail(rc, TLQR_K_AFF_TAIL, fx::kf_aff_tail<T, NX>, st, w, f->d_rounds, r_tail, R)))
      return e;
  }
  for (int ri = r_tail - 1; ri >= 0; --ri) {
    const tlqr_round* it = &P->rounds[ri];
    const int nc = it->comp_end - it->comp_begin;
    if constexpr (NF > 0) {
      if ((e = launch_groups(rc, TLQR_K_AFF_EXPAND, fx::kf_aff_expand<T, NX>, nc, G, 0, st, w, it->comp_begin,
                             nc))) return e;
    } else if ((e = launch_warps(rc, TLQR_K_AFF_EXPAND, k_aff_expand<T>, nc, wb.vec1, st, w, it->comp_begin, nc,
                                 (int)wb.vec1))) {
      return e;
    }
  }
  if ((e = local_solve())) return e;
  for (int ri = 0; ri < r_tail; ++ri) {
    const tlqr_round& rd = P->rounds[ri];
    const int nc = rd.comp_end - rd.comp_begin;
    if constexpr (NF > 0) {
      if ((e = launch_groups(rc, TLQR_K_STATE_COMPRESS, fx::kf_state_compress<T, NX>, nc, G, 0, st, w,
                             rd.comp_begin, nc))) return e;
    } else if ((e = launch_warps(rc, TLQR_K_STATE_COMPRESS, k_state_compress<T>, nc, wb.vec1, st, w, rd.comp_begin,
                                 nc, (int)wb.vec1))) {
      return e;
    }
  }
  if constexpr (NF > 0) {
    if (r_tail < R &&
        (e = launch_tail(rc, TLQR_K_STATE_TAIL, fx::kf_state_tail<T, NX>, st, w, f->d_rounds, r_tail, R)))
      return e;
  }
  for (int ri = r_tail - 1; ri >= 0; --ri) {
    const tlqr_round* it = &P->rounds[ri];
    const int nc = it->comp_end - it->comp_begin, nr = it->rake_end - it->rake_begin;
    const int *cj = f->dp.comp_j, *ci = f->dp.comp_i, *rl = f->dp.rake_leaf, *rp = f->dp.rake_parent;
    if constexpr (NF > 0) {
      if ((e = launch_groups(rc, TLQR_K_STATE_EXPAND, fx::kf_state_expand<T, NX>, nc, G, 0, st, w, cj, ci,
                             it->comp_begin, nc))) return e;
      if ((e = launch_groups(rc, TLQR_K_STATE_EXPAND, fx::kf_state_expand<T, NX>, nr, G, 0, st, w, rl, rp,
                             it->rake_begin, nr))) return e;
    } else {
      if ((e = launch_warps(rc, TLQR_K_STATE_EXPAND, k_state_expand<T>, nc, wb.vec1, st, w, cj, ci, it->comp_begin,
                            nc, (int)wb.vec1))) return e;
      if ((e = launch_warps(rc, TLQR_K_STATE_EXPAND, k_state_expand<T>, nr, wb.vec1, st, w, rl, rp, it->rake_begin,
                            nr, (int)wb.vec1))) return e;
    }
  }
  return recover();
}

// FP64 keeps the run-time-n kernels at n = 32 (a row of 32 doubles per lane
// does not fit the register file), so those are not instantiated.
template <typename T>
constexpr bool fixed_for(int n) { return !(sizeof(T) == 8 && n == 32); }

// Dimension dispatch.  fixed_n: compile-time n of the n x n kernels (0 = run time);
// fixed_m: compile-time m of the (n, m) kernels for that n (0 = run time).
#define TLQR_FIXED_CASES(X)                                                     \
  X(4, 0) X(4, 2) X(6, 0) X(6, 2) X(8, 0) X(8, 2) X(12, 0) X(12, 4) X(16, 0) X(16, 4) X(32, 0) X(32, 8)
// the (n, m) pairs of the list above
#define TLQR_FIXED_PAIRS(X) X(4, 2) X(6, 2) X(8, 2) X(12, 4) X(16, 4) X(32, 8)

template <typename T>
cudaError_t dispatch_factor(tlqr_factor_t* f, Recorder* rc, const tlqr_problem& p, cudaStream_t st) {
#define X(n_, m_)                                                   \
  if constexpr (fixed_for<T>(n_))                                   \
    if (f->fixed_n == n_ && f->fixed_m == m_) return run_factor<T, n_, m_>(f, rc, p, st);
  TLQR_FIXED_CASES(X)
#undef X
  return run_factor<T, 0, 0>(f, rc, p, st);
}
template <typename T>
cudaError_t dispatch_solve(tlqr_factor_t* f, Recorder* rc, const double* q, const double* r, const double* c,
                           double* x, double* u, double* y, int accumulate, cudaStream_t st, int nrhs = 1,
                           const PanelBufs* pb = nullptr) {
#define X(n_, m_)                                                   \
  if constexpr (fixed_for<T>(n_))                                   \
    if (f->fixed_n == n_ && f->fixed_m == m_)                       \
      return run_solve<T, n_, m_>(f, rc, q, r, c, x, u, y, accumulate, st, nrhs, pb);
  TLQR_FIXED_CASES(X)
#undef X
  return run_solve<T, 0, 0>(f, rc, q, r, c, x, u, y, accumulate, st, nrhs, pb);
}

bool has_fixed_kernels(int n) { return n == 4 || n == 6 || n == 8 || n == 12 || n == 16 || n == 32; }
bool has_fixed_pair(int n, int m) {
  return (m == 2 && (n == 4 || n == 6 || n == 8)) || (m == 4 && (n == 12 || n == 16)) || (m == 8 && n == 32);
}

// Resident blocks per SM of a kernel at a launch shape (cached; the first query
// for a shape happens when the factor is configured, outside stream capture).
template <typename Kernel>
int resident_blocks(Kernel kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, size_t>, int> have;
  std::lock_guard<std::mutex> lock(mu);
  auto it = have.find({(const void*)kernel, smem});
  if (it != have.end()) return it->second;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    b = 1;
  }
  b = std::max(1, b);
  have[{(const void*)kernel, smem}] = b;
  return b;
}

// Node-organised float-float residual for compile-time (n, m): edge pass then
// node pass with bulk-copy staging (see residual_nodes.cuh).  Grids are one
// wave: every resident block slot of every SM, each warp walking a contiguous
// node range.  Returns cudaErrorNotSupported when (n, m) has no such kernels.
template <int N, int M>
cudaError_t launch_res_nodes(const ResidualArgs& a, const FFArgs& fa, const rn::NodeArgs& na, int sms,
                             cudaStream_t st, bool capturing) {
  constexpr int OPS = rn::RG<N>::OPS, threads = 128, gpb = (threads / 32) * OPS;
  const size_t se = (size_t)rn::EdgeBuf<N, M>::group_bytes(a.Delta != nullptr, a.M != nullptr) * gpb;
  const size_t sn = (size_t)rn::NodeBuf<N>::group_bytes * gpb;
  const bool forest = a.tree != nullptr;
  auto ek = forest ? rn::k_res_edge<N, M, true> : rn::k_res_edge<N, M, false>;
  auto nk = forest ? rn::k_res_node<N, true> : rn::k_res_node<N, false>;
  if (!capturing) {
    cudaError_t e = ensure_smem(ek, se);
    if (!e) e = ensure_smem(nk, sn);
    if (e) return e;
  }
  const long long need = ((long long)a.N + gpb - 1) / gpb;
  const int be = (int)std::max<long long>(1, std::min<long long>(need, (long long)sms * resident_blocks(ek, threads, se)));
  const int bn = (int)std::max<long long>(1, std::min<long long>(need, (long long)sms * resident_blocks(nk, threads, sn)));
  ek<<<be, threads, se, st>>>(a, fa, na);
  nk<<<bn, threads, sn, st>>>(a, fa, na);
  return cudaGetLastError();
}

cudaError_t configure_res_nodes(int n, int m) {
#define X(n_, m_)                                                                              \
  if (n == n_ && m == m_) {                                                                    \
    constexpr int gpb = 4 * rn::RG<n_>::OPS;                                                   \
    const size_t sn = (size_t)rn::NodeBuf<n_>::group_bytes * gpb;                                 \
    cudaError_t e = ensure_smem(rn::k_res_node<n_, true>, sn);                                    \
    if (!e) e = ensure_smem(rn::k_res_node<n_, false>, sn);                                       \
    resident_blocks(rn::k_res_node<n_, true>, 128, sn);                                           \
    resident_blocks(rn::k_res_node<n_, false>, 128, sn);                                          \
    for (int hd = 0; hd < 2 && !e; ++hd)                                                       \
      for (int hm = 0; hm < 2 && !e; ++hm) {                                                   \
        const size_t se = (size_t)rn::EdgeBuf<n_, m_>::group_bytes(hd, hm) * gpb;                 \
        e = ensure_smem(rn::k_res_edge<n_, m_, true>, se);                                        \
        if (!e) e = ensure_smem(rn::k_res_edge<n_, m_, false>, se);                               \
        resident_blocks(rn::k_res_edge<n_, m_, true>, 128, se);                                   \
        resident_blocks(rn::k_res_edge<n_, m_, false>, 128, se);                                  \
      }                                                                                        \
    return e;                                                                                  \
  }
  TLQR_FIXED_PAIRS(X)
#undef X
  return cudaSuccess;
}

cudaError_t dispatch_res_nodes(int n, int m, const ResidualArgs& a, const FFArgs& fa, const rn::NodeArgs& na,
                               int sms, cudaStream_t st, bool capturing) {
#define X(n_, m_) \
  if (n == n_ && m == m_) return launch_res_nodes<n_, m_>(a, fa, na, sms, st, capturing);
  TLQR_FIXED_PAIRS(X)
#undef X
  return cudaErrorNotSupported;
}

// Which float-float residual runs (options.residual): 1 = the row-per-thread
// kernels, 2 = the node-organised bulk-copy kernels, 0 = the library's choice
// per n (kResNodeDefault).  The node kernels need compile-time (n, m) and
// 16-byte aligned matrix arrays; otherwise the row kernels run.
// Measured on B300 (refinement residual per step, row kernels vs node kernels
// with bulk-copied blocks and vectors): n = 12 (long trunk, 65,536 nodes) 0.24
// vs 0.32 ms; n = 16 (1,024 trees, 2.9 M nodes) 23.7 vs 14.5 ms; n = 32
// (2^20 nodes) 23.1 vs 21.1 ms.
bool res_node_default(int n) { return n == 16 || n == 32; }

// polls of one mbarrier wait of the node residual before it gives up (each
// poll may suspend the thread for a while, so this is ~a second or more)
constexpr int kBarSpin = 1 << 20;
bool use_node_residual(const tlqr_factor_t* f, const tlqr_problem& p, const double* x, const double* u,
                       const double* y) {
  if (f->fixed_m == 0 || f->ts != 4) return false;
  const int kind = f->opt.residual;
  if (kind == 1 || (kind == 0 && !res_node_default(f->fixed_n))) return false;
  auto al = [](const void* q) { return q == nullptr || ((uintptr_t)q & 15u) == 0; };
  return al(p.Q) && al(p.A) && al(p.B) && al(p.R) && (!f->opt.has_M || al(p.M)) &&
         (!f->opt.has_delta || al(p.Delta)) && al(p.q) && al(p.r) && al(p.c) && al(x) && al(u) && al(y);
}

// ff = 1: float-float kernel on the FP32 pipe (refinement); ff = 0: plain FP64 kernel.
cudaError_t run_residual(tlqr_factor_t* f, Recorder* rc, const tlqr_problem& p, const double* x,
                         const double* u, const double* y, int with_knorm, cudaStream_t st, int ff = 0,
                         const unsigned char* dflag = nullptr) {
  ResidualArgs a{};
  const tlqr_plan_t* P = f->plan;
  a.N = P->N; a.n = f->opt.n; a.m = f->opt.m; a.with_knorm = with_knorm;
  a.parent = f->dp.parent; a.child_start = f->dp.child_start; a.child_list = f->dp.child_list;
  a.Q = p.Q; a.q = p.q; a.M = f->opt.has_M ? p.M : nullptr; a.R = p.R; a.r = p.r; a.A = p.A;
  a.B = p.B; a.c = p.c; a.Delta = f->opt.has_delta ? p.Delta : nullptr;
  a.x = x; a.u = u; a.y = y;
  a.dflag = a.Delta ? dflag : nullptr;
  a.res_x = f->res_x; a.res_u = f->res_u; a.res_c = f->res_c;
  a.maxes = f->maxes;
  a.T = P->n_trees;
  a.tree = a.T > 1 ? f->dp.tree : nullptr;
  // slot-major [4][T]: the ||K|| slot (last) is kept from an earlier call unless with_knorm
  cudaError_t e = cudaMemsetAsync(f->maxes, 0, (with_knorm ? 4 : 3) * (size_t)a.T * sizeof(unsigned long long), st);
  if (e) return e;
  FFArgs fa{};
  // the node kernels split x, u, y themselves and form all four maxima
  const bool by_node = ff && use_node_residual(f, p, x, u, y);
  if (ff && !by_node) {
    // split x, u, y once per call; for one tree ||z|| and ||b|| maxima come
    // from the same pass (a forest forms them per tree in the residual kernel)
    const size_t N = P->N, n = f->opt.n, m = f->opt.m;
    const int zs = a.tree ? -1 : 1, bs = a.tree ? -1 : 2;
    SplitList L{};
    auto add = [&](const double* src, float* hi, float* lo, size_t len, int slot) {
      L.src[L.count] = src; L.hi[L.count] = hi; L.lo[L.count] = lo; L.len[L.count] = len; L.slot[L.count] = slot;
      ++L.count;
    };
    add(x, f->xh, f->xl, N * n, zs);
    add(u, f->uh, f->ul, N * m, zs);
    add(y, f->yh, f->yl, N * n, zs);
    if (bs >= 0) {
      add(p.q, nullptr, nullptr, N * n, bs);
      add(p.r, nullptr, nullptr, N * m, bs);
      add(p.c, nullptr, nullptr, N * n, bs);
    }
    L.maxes = f->maxes;
    if ((e = launch_split(rc, L, f->sms, st))) return e;
    fa = FFArgs{f->xh, f->xl, f->uh, f->ul, f->yh, f->yl};
  }
  const size_t rows = (size_t)P->N * (2 * f->opt.n + f->opt.m);
  const int threads = 256;
  // grid-stride over the rows with at most 32 blocks per SM (measured faster
  // than fewer blocks holding equal row counts, despite the uneven last rows)
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((rows + threads - 1) / threads, (size_t)f->sms * 32));
  const bool timed = rc && (rc->mask >> TLQR_K_RESIDUAL) & 1u;
  EvPair ev{TLQR_K_RESIDUAL, nullptr, nullptr, P->N};
  if (timed) { ev.a = rc->event(); ev.b = rc->event(); rc->record(ev.a, st); }
  if (by_node) {
    const rn::NodeArgs na{f->rwh,
                          f->rwl,
                          f->rwk,
                          f->opt.has_delta ? dflag : nullptr,
                          f->status,
                          f->opt.spin_limit > 0 ? f->opt.spin_limit : kBarSpin,
                          (f->opt.test_withhold & 2) ? 1 : 0};
    if ((e = dispatch_res_nodes(f->fixed_n, f->fixed_m, a, fa, na, f->sms, st, rc && rc->capture))) return e;
  } else if (a.tree) {
    if (ff) k_residual_ff_trees<<<blocks, threads, 0, st>>>(a, fa);
    else k_residual_trees<<<blocks, threads, 0, st>>>(a);
  } else {
    if (ff) k_residual_ff<<<blocks, threads, 0, st>>>(a, fa);
    else k_residual<<<blocks, threads, 0, st>>>(a);
  }
  if ((e = cudaGetLastError())) return e;
  if (timed) { rc->record(ev.b, st); rc->recs.push_back(ev); }
  if (rc) { rc->launches[TLQR_K_RESIDUAL]++; rc->units[TLQR_K_RESIDUAL] += P->N; }
  if ((e = cudaMemcpyAsync(f->h_maxes, f->maxes, 4 * (size_t)a.T * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, st)))
    return e;
  return cudaMemcpyAsync(f->h_status, f->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
}

// Run one launch sequence, through a cached CUDA graph when graphs are on.
template <typename Body>
cudaError_t run_seq(tlqr_factor_t* f, GraphCache* g, std::vector<uintptr_t> key, cudaStream_t st, Body body) {
  key.push_back(f->prof.mask);
  if (!f->opt.use_graphs || f->graphs_broken || !g) {
    Recorder r;
    r.pdl = f->opt.pdl >= 0;
    r.mask = f->prof.mask;
    r.pool = &f->prof.pool;
    cudaError_t e = body(&r);
    f->prof.add(r, true);
    return e;
  }
  if (!g->exec || g->key != key) {
    g->clear();
    Recorder r;
    r.pdl = f->opt.pdl >= 0;
    r.mask = f->prof.mask;
    r.capture = true;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    cudaError_t eb = e ? e : body(&r);
    cudaGraph_t graph = nullptr;
    if (!e) e = cudaStreamEndCapture(st, &graph);
    if (!e && !eb) e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e || eb) {
      // capture not possible here: fall back to direct launches for good
      for (const EvPair& p : r.recs) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
      if (g->exec) cudaGraphExecDestroy(g->exec);
      g->exec = nullptr;
      cudaGetLastError();
      f->graphs_broken = true;
      return run_seq(f, nullptr, key, st, body);
    }
    g->key = key;
    g->rec = r;
  }
  cudaError_t e = cudaGraphLaunch(g->exec, st);
  f->prof.add(g->rec, false);
  return e;
}

uintptr_t up(const void* p) { return (uintptr_t)p; }

std::vector<uintptr_t> problem_key(const tlqr_problem& p) {
  return {up(p.Q), up(p.q), up(p.M), up(p.R), up(p.r), up(p.A), up(p.B), up(p.c), up(p.Delta)};
}

GraphCache* solve_cache(tlqr_factor_t* f, const std::vector<uintptr_t>& key) {
  std::vector<uintptr_t> k = key;
  k.push_back(f->prof.mask);
  for (auto& g : f->g_solve)
    if (g.exec && g.key == k) return &g;
  GraphCache* g = &f->g_solve[f->solve_lru];
  f->solve_lru = (f->solve_lru + 1) % 4;
  return g;
}

// ||K z - b|| and eta of tree t from the slot-major maxima [4][T].
void tree_stats(const tlqr_factor_t* f, int t, double* abs_res, double* eta) {
  const int T = f->plan->n_trees;
  double v[4];
  for (int q = 0; q < 4; ++q) std::memcpy(&v[q], &f->h_maxes[(size_t)q * T + t], sizeof(double));
  *abs_res = v[0];
  const double den = v[3] * v[1] + v[2];
  *eta = den > 0 ? v[0] / den : v[0];
  if (!std::isfinite(v[0])) *eta = INFINITY;
}

// Whole problem: the largest residual, and the largest eta over the trees
// (for one tree, the plain eta).
void residual_stats(const tlqr_factor_t* f, double* abs_res, double* eta) {
  *abs_res = 0.0;
  *eta = 0.0;
  for (int t = 0; t < f->plan->n_trees; ++t) {
    double a, e;
    tree_stats(f, t, &a, &e);
    if (!(a <= *abs_res)) *abs_res = a;
    if (!(e <= *eta)) *eta = e;
  }
}

size_t problem_elems(int N, int n, int m) {
  const size_t nn = (size_t)n * n, nm = (size_t)n * m;
  // Q q M R r A B c Delta  +  x u y P K
  return (size_t)N * (nn + n + nm + (size_t)m * m + m + nn + nm + n + nn) + (size_t)N * (n + m + n + nn + nm);
}

int ensure_stage(tlqr_factor_t* f) {
  if (f->stage) return TLQR_OK;
  const size_t e = problem_elems(f->plan->N, f->opt.n, f->opt.m);
  cudaError_t err = cudaSuccess;
  f->stage = dalloc<double>(e, &err);
  if (err != cudaSuccess) return TLQR_ERR_OOM;
  f->allocs.push_back(f->stage);
  f->stage_elems = e;
  return TLQR_OK;
}

// Device staging layout for host-memory calls.
struct Stage {
  double *Q, *q, *M, *R, *r, *A, *B, *c, *Delta, *x, *u, *y, *P, *K;
};
Stage stage_layout(tlqr_factor_t* f) {
  const size_t N = f->plan->N, n = f->opt.n, m = f->opt.m;
  Stage s;
  double* p = f->stage;
  s.Q = p; p += N * n * n;
  s.q = p; p += N * n;
  s.M = p; p += N * n * m;
  s.R = p; p += N * m * m;
  s.r = p; p += N * m;
  s.A = p; p += N * n * n;
  s.B = p; p += N * n * m;
  s.c = p; p += N * n;
  s.Delta = p; p += N * n * n;
  s.x = p; p += N * n;
  s.u = p; p += N * m;
  s.y = p; p += N * n;
  s.P = p; p += N * n * n;
  s.K = p;
  return s;
}

cudaError_t h2d(double* dst, const double* src, size_t count, cudaStream_t st) {
  if (!src || !count) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyHostToDevice, st);
}
cudaError_t d2h(double* dst, const double* src, size_t count, cudaStream_t st) {
  if (!dst || !count) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDeviceToHost, st);
}

// Copy a host-memory problem into staging and return the device view.
int stage_problem(tlqr_factor_t* f, const tlqr_problem* in, tlqr_problem* out, bool matrices, bool rhs,
                  cudaStream_t st) {
  int rc = ensure_stage(f);
  if (rc) return rc;
  Stage s = stage_layout(f);
  const size_t N = f->plan->N, n = f->opt.n, m = f->opt.m;
  *out = *in;
  out->mem = TLQR_MEM_DEVICE;
  cudaError_t e = cudaSuccess;
  if (matrices) {
    if (!e) e = h2d(s.Q, in->Q, N * n * n, st);
    if (!e && f->opt.has_M) e = h2d(s.M, in->M, N * n * m, st);
    if (!e) e = h2d(s.R, in->R, N * m * m, st);
    if (!e) e = h2d(s.A, in->A, N * n * n, st);
    if (!e) e = h2d(s.B, in->B, N * n * m, st);
    if (!e && f->opt.has_delta) e = h2d(s.Delta, in->Delta, N * n * n, st);
    out->Q = s.Q; out->M = f->opt.has_M ? s.M : nullptr; out->R = s.R; out->A = s.A; out->B = s.B;
    out->Delta = f->opt.has_delta ? s.Delta : nullptr;
  }
  if (rhs) {
    if (!e) e = h2d(s.q, in->q, N * n, st);
    if (!e) e = h2d(s.r, in->r, N * m, st);
    if (!e) e = h2d(s.c, in->c, N * n, st);
    out->q = s.q; out->r = s.r; out->c = s.c;
  }
  return e ? TLQR_ERR_CUDA : TLQR_OK;
}

int check_problem(const tlqr_factor_t* f, const tlqr_problem* p, bool rhs) {
  if (!p) return TLQR_ERR_ARG;
  if (p->mem != TLQR_MEM_DEVICE && p->mem != TLQR_MEM_HOST) return TLQR_ERR_ARG;
  if (!p->Q || !p->R || !p->A || !p->B) return TLQR_ERR_ARG;
  if ((f->opt.has_M != 0) != (p->M != nullptr)) return TLQR_ERR_ARG;
  if ((f->opt.has_delta != 0) != (p->Delta != nullptr)) return TLQR_ERR_ARG;
  if (rhs && (!p->q || !p->r || !p->c)) return TLQR_ERR_ARG;
  return TLQR_OK;
}

// Read the device status word (synchronises the stream).
int read_status(tlqr_factor_t* f, cudaStream_t st) {
  if (cudaMemcpyAsync(f->h_status, f->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) return TLQR_ERR_CUDA;
  if (cudaStreamSynchronize(st)) return TLQR_ERR_CUDA;
  f->info.fp64_resolves = std::min(f->h_status[1], f->redo_cap);
  return map_status(*f->h_status);
}

// Set the dynamic shared-memory limits of every kernel this factor launches
// (outside any stream capture).
template <typename T>
cudaError_t configure_kernels(int n, int m) {
  const WarpBytes wb = warp_bytes(n, m, sizeof(T));
  auto sz = [](size_t w) { return w * warps_per_block(w); };
  cudaError_t e = cudaSuccess;
  if (!e) e = ensure_smem(k_condense<T>, sz(wb.condense));
  if (!e) e = ensure_smem(k_rake<T>, sz(wb.tau));
  if (!e) e = ensure_smem(k_expand<T>, sz(wb.tau));
  if (!e) e = ensure_smem(k_compress<T>, sz(wb.compress));
  if (!e) e = ensure_smem(k_local_factor<T>, sz(wb.local_factor));
  if (!e) e = ensure_smem(k_compose_T<T>, sz(wb.compose_T));
  if (!e) e = ensure_smem(k_aff_init<T>, sz(wb.aff_init));
  if (!e) e = ensure_smem(k_aff_rake<T>, sz(wb.vec1));
  if (!e) e = ensure_smem(k_aff_compress<T>, sz(wb.vec1));
  if (!e) e = ensure_smem(k_aff_expand<T>, sz(wb.vec1));
  if (!e) e = ensure_smem(k_local_solve<T>, sz(wb.local_solve));
  if (!e) e = ensure_smem(k_state_compress<T>, sz(wb.vec1));
  if (!e) e = ensure_smem(k_state_expand<T>, sz(wb.vec1));
  if (!e) e = ensure_smem(k_recover<T>, sz(wb.recover));
  return e;
}

template <typename T, int N>
cudaError_t configure_fixed() {
  constexpr int gpb = 128 / fx::D<T, N>::G;
  cudaError_t e = ensure_smem(fx::kf_rake<T, N>, (size_t)fx::TauSmem<T, N>::bytes * gpb);
  if (!e) e = ensure_smem(fx::kf_expand<T, N>, (size_t)fx::TauSmem<T, N>::bytes * gpb);
  if (!e) e = ensure_smem(fx::kf_compress<T, N>, (size_t)fx::CompSmem<T, N>::bytes * gpb);
  if (!e) e = ensure_smem(fx::kf_compose_T<T, N>, (size_t)fx::ComposeSmem<T, N>::bytes * gpb);
  if (!e) e = ensure_smem(fx::kf_async<T, N>, (size_t)fx::AsyncSmem<T, N>::bytes * gpb);
  return e;
}

// Resident 128-thread blocks of kf_async per SM (its persistent grid is this
// times the SM count; correctness does not depend on it).
template <typename T, int N>
int async_occupancy() {
  constexpr int gpb = 128 / fx::D<T, N>::G;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fx::kf_async<T, N>, 128,
                                                    (size_t)fx::AsyncSmem<T, N>::bytes * gpb) != cudaSuccess) {
    cudaGetLastError();
    b = 1;
  }
  return std::max(1, b);
}
template <typename T, int N>
int async_vec_occupancy() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fx::kf_async_vec<T, N>, 128, 0) != cudaSuccess) {
    cudaGetLastError();
    b = 1;
  }
  return std::max(1, b);
}
// vec = false: kf_async; true: kf_async_vec
template <typename T>
int async_occupancy_n(int n, bool vec) {
  switch (n) {
    case 4: return vec ? async_vec_occupancy<T, 4>() : async_occupancy<T, 4>();
    case 6: return vec ? async_vec_occupancy<T, 6>() : async_occupancy<T, 6>();
    case 8: return vec ? async_vec_occupancy<T, 8>() : async_occupancy<T, 8>();
    case 12: return vec ? async_vec_occupancy<T, 12>() : async_occupancy<T, 12>();
    case 16: return vec ? async_vec_occupancy<T, 16>() : async_occupancy<T, 16>();
    case 32:
      if constexpr (fixed_for<T>(32)) return vec ? async_vec_occupancy<T, 32>() : async_occupancy<T, 32>();
      return 1;
    default: return 1;
  }
}
template <typename T, int N, int M>
cudaError_t configure_fixed_nm() {
  constexpr int gpb = 128 / fx::D<T, N>::G;
  cudaError_t e = ensure_smem(fx::kf_condense<T, N, M>, (size_t)fx::CondSmem<T, N, M>::bytes * gpb);
  if (!e) e = ensure_smem(fx::kf_local_factor<T, N, M>, (size_t)fx::LfSmem<T, N, M>::bytes * gpb);
  if (!e) e = ensure_smem(fx::kf_aff_init<T, N, M>, (size_t)fx::AiSmem<T, N, M>::bytes * gpb);
  if (!e) e = ensure_smem(fx::kf_local_solve<T, N, M>, (size_t)fx::LsSmem<T, N, M>::bytes * gpb);
  return e;
}
template <typename T>
cudaError_t configure_fixed_pair(int n, int m) {
#define X(n_, m_) \
  if constexpr (m_ > 0 && fixed_for<T>(n_)) { if (n == n_ && m == m_) return configure_fixed_nm<T, n_, m_>(); }
  TLQR_FIXED_CASES(X)
#undef X
  return cudaSuccess;
}
template <typename T>
cudaError_t configure_fixed_n(int n) {
  switch (n) {
    case 4: return configure_fixed<T, 4>();
    case 6: return configure_fixed<T, 6>();
    case 8: return configure_fixed<T, 8>();
    case 12: return configure_fixed<T, 12>();
    case 16: return configure_fixed<T, 16>();
    case 32:
      if constexpr (fixed_for<T>(32)) return configure_fixed<T, 32>();
      return cudaSuccess;
    default: return cudaSuccess;
  }
}

// Host-side kernel selection of a factor object (no CUDA calls): the
// compile-time-(n, m) kernels where they exist, and the rounds handed to the
// level-asynchronous kernel -- every round from the first one after which each
// round holds at most async_ops operations (default kAsyncOps).  Returns
// nonzero when the host ran out of memory.
int select_kernels(tlqr_factor_t* f) {
  const tlqr_options& o = f->opt;
  const int n = o.n, m = o.m;
  f->fixed_n = (has_fixed_kernels(n) && !o.generic_kernels) ? n : 0;
  // FP64: groups of 8 / 16 lanes for n = 6 / 12 leave lanes idle, which costs FP64 issue slots;
  // the run-time-n kernels keep all 32 lanes busy and are faster there.
  if (f->ts == 8 && (n == 6 || n == 12 || n == 32)) f->fixed_n = 0;
  f->fixed_m = (f->fixed_n && has_fixed_pair(n, m)) ? m : 0;
  f->fa = DevAsync{};
  f->aa = DevAsync{};
  f->sa = DevAsync{};
  f->fa.plan.r0 = (int)f->plan->rounds.size();
  const int G = n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32;
  try {
    if (f->fixed_n > 0 && o.async_ops >= 0) {
      const int thr = o.async_ops > 0 ? o.async_ops : kAsyncOps;
      int r0 = (int)f->plan->rounds.size();
      while (r0 > 0) {
        const tlqr_round& r = f->plan->rounds[r0 - 1];
        if ((r.rake_end - r.rake_begin) + (r.comp_end - r.comp_begin) > thr) break;
        --r0;
      }
      f->fa.plan = build_async(f->plan, r0, 32 / G);
    }
    // right-hand-side passes: the affine pass has the dependency structure of the
    // whole factorisation (every round), the state pass its own list
    if (f->fixed_n > 0 && o.async_solve > 0 && !f->plan->rounds.empty()) {
      f->aa.plan = build_async(f->plan, 0, 32 / G);
      f->sa.plan = build_async_state(f->plan, 32 / G);
    }
  } catch (const std::bad_alloc&) {
    return 1;
  }
  return 0;
}

// Enqueue the factorisation; with `sync` also wait and report its status.
int factor_impl(tlqr_factor_t* f, const tlqr_problem* dp, cudaStream_t st, bool sync) {
  f->dprob = *dp;
  f->factored = false;
  tlqr_problem key = *dp;
  key.q = key.r = key.c = nullptr;
  cudaError_t e = run_seq(f, &f->g_factor, problem_key(key), st, [&](Recorder* rc) {
    return f->ts == 8 ? dispatch_factor<double>(f, rc, *dp, st) : dispatch_factor<float>(f, rc, *dp, st);
  });
  if (e) return TLQR_ERR_CUDA;
  f->factored = true;
  if (!sync) return TLQR_OK;
  const int rc = read_status(f, st);
  f->prof.harvest();
  if (rc != TLQR_OK) f->factored = false;
  return rc;
}

cudaError_t solve_impl(tlqr_factor_t* f, const double* q, const double* r, const double* c, double* x,
                       double* u, double* y, int accumulate, cudaStream_t st) {
  std::vector<uintptr_t> key = problem_key(f->dprob);
  for (const void* p : {(const void*)q, (const void*)r, (const void*)c, (const void*)x, (const void*)u, (const void*)y})
    key.push_back(up(p));
  key.push_back((uintptr_t)accumulate);
  return run_seq(f, solve_cache(f, key), key, st, [&](Recorder* rc) {
    return f->ts == 8 ? dispatch_solve<double>(f, rc, q, r, c, x, u, y, accumulate, st)
                      : dispatch_solve<float>(f, rc, q, r, c, x, u, y, accumulate, st);
  });
}

// dflag: the factor's per-node "Delta_i is nonzero" flags when p holds the
// matrices the factor was formed from (the node kernels then copy no zero
// Delta block); null otherwise.
cudaError_t residual_impl(tlqr_factor_t* f, const tlqr_problem& p, const double* x, const double* u,
                          const double* y, int with_knorm, cudaStream_t st, const unsigned char* dflag = nullptr) {
  std::vector<uintptr_t> key = problem_key(p);
  for (const void* v : {(const void*)x, (const void*)u, (const void*)y, (const void*)dflag}) key.push_back(up(v));
  key.push_back((uintptr_t)with_knorm);
  return run_seq(f, &f->g_resid[with_knorm ? 1 : 0], key, st,
                 [&](Recorder* rc) { return run_residual(f, rc, p, x, u, y, with_knorm, st, 1, dflag); });
}

}  // namespace

// ====================================================================== C ABI

extern "C" const char* tlqr_status_string(int code) {
  switch (code) {
    case TLQR_OK: return "ok";
    case TLQR_ERR_ARG: return "invalid argument";
    case TLQR_ERR_TOPOLOGY: return "parent array is not a rooted tree";
    case TLQR_ERR_NOT_PD: return "Cholesky of R or G failed (not positive definite)";
    case TLQR_ERR_SINGULAR: return "singular or nonfinite pivot in I + C P or I + Delta P";
    case TLQR_ERR_NONFINITE: return "non-finite value";
    case TLQR_ERR_OOM: return "out of memory";
    case TLQR_ERR_TIMEOUT: return "bounded device wait timed out";
    case TLQR_ERR_NO_CONVERGENCE: return "iterative refinement did not converge";
    case TLQR_ERR_CUDA: return "CUDA runtime error";
    case TLQR_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

extern "C" int tlqr_factor_create(const tlqr_plan_t* plan, const tlqr_options* opts, tlqr_factor_t** out) {
  if (!plan || !opts || !out) return TLQR_ERR_ARG;
  *out = nullptr;
  const int n = opts->n, m = opts->m;
  if (n < 1 || m < 1 || n > TLQR_MAX_DIM || m > TLQR_MAX_DIM) return TLQR_ERR_ARG;
  if (opts->precision != TLQR_PREC_FP64 && opts->precision != TLQR_PREC_MIXED) return TLQR_ERR_ARG;
  if (opts->residual < 0 || opts->residual > 2) return TLQR_ERR_ARG;
  tlqr_factor_t* f = new (std::nothrow) tlqr_factor_t;
  if (!f) return TLQR_ERR_OOM;
  f->plan = plan;
  f->opt = *opts;
  if (f->opt.max_refine <= 0) f->opt.max_refine = 10;
  if (!(f->opt.refine_tol > 0)) f->opt.refine_tol = 1e-8;
  f->ts = opts->precision == TLQR_PREC_FP64 ? 8 : 4;
  if (cudaGetDevice(&f->device) ||
      cudaDeviceGetAttribute(&f->sms, cudaDevAttrMultiProcessorCount, f->device) || f->sms < 1) {
    delete f;
    return TLQR_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&f->work, cudaStreamNonBlocking) ||
      cudaEventCreateWithFlags(&f->ev_in, cudaEventDisableTiming) ||
      cudaEventCreateWithFlags(&f->ev_out, cudaEventDisableTiming)) {
    delete f;
    return TLQR_ERR_CUDA;
  }
  // per-warp shared memory must fit one warp per block
  const WarpBytes wb = warp_bytes(n, m, f->ts);
  const size_t worst = std::max({wb.compress, wb.local_factor, wb.tau, wb.condense});
  if (worst > kSmemBudget) { delete f; return TLQR_ERR_ARG; }
  if (select_kernels(f)) { delete f; return TLQR_ERR_OOM; }
  if ((f->ts == 8 ? configure_kernels<double>(n, m) : configure_kernels<float>(n, m)) != cudaSuccess ||
      (f->ts == 8 ? configure_fixed_n<double>(f->fixed_n) : configure_fixed_n<float>(f->fixed_n)) != cudaSuccess ||
      (f->ts == 8 ? configure_fixed_pair<double>(f->fixed_n, f->fixed_m)
                  : configure_fixed_pair<float>(f->fixed_n, f->fixed_m)) != cudaSuccess ||
      (f->ts == 4 && f->fixed_m > 0 && configure_res_nodes(f->fixed_n, f->fixed_m) != cudaSuccess)) {
    delete f;
    return TLQR_ERR_CUDA;
  }
  if (f->fa.plan.n_ops > 0)
    f->fa.blocks = f->sms * (f->ts == 8 ? async_occupancy_n<double>(n, false) : async_occupancy_n<float>(n, false));
  if (f->aa.plan.n_ops > 0) {
    f->aa.blocks = f->sa.blocks =
        f->sms * (f->ts == 8 ? async_occupancy_n<double>(n, true) : async_occupancy_n<float>(n, true));
  }
  Carve sizing;
  carve_factor(f, sizing);
  void* arena = nullptr;
  cudaError_t err = cudaMalloc(&arena, sizing.off);
  if (err != cudaSuccess) {
    cudaGetLastError();
    delete f;
    return err == cudaErrorMemoryAllocation ? TLQR_ERR_OOM : TLQR_ERR_CUDA;
  }
  f->allocs.push_back(arena);
  f->arena_bytes = sizing.off;
  Carve c;
  c.base = static_cast<unsigned char*>(arena);
  carve_factor(f, c);
  int rc = upload_plan(f);
  if (rc) { delete f; return rc; }
  const size_t N = plan->N, T = (size_t)plan->n_trees;
  if (err == cudaSuccess) err = cudaMallocHost((void**)&f->h_maxes, 4 * T * sizeof(unsigned long long));
  if (err == cudaSuccess) err = cudaMallocHost((void**)&f->h_gate, 2 * sizeof(double));
  if (err == cudaSuccess) err = cudaMallocHost((void**)&f->h_status, 2 * sizeof(int));
  if (err == cudaSuccess) f->h_status[0] = f->h_status[1] = 0;
  if (err == cudaSuccess && f->dflag) err = cudaMemset(f->dflag, 0, N);
  if (err != cudaSuccess) {
    delete f;
    return err == cudaErrorMemoryAllocation ? TLQR_ERR_OOM : TLQR_ERR_CUDA;
  }
  *out = f;
  return TLQR_OK;
}

extern "C" int tlqr_factor_workspace_bytes(const tlqr_plan_t* plan, const tlqr_options* opts, size_t* bytes) {
  if (!plan || !opts || !bytes) return TLQR_ERR_ARG;
  if (opts->n < 1 || opts->m < 1 || opts->n > TLQR_MAX_DIM || opts->m > TLQR_MAX_DIM) return TLQR_ERR_ARG;
  if (opts->precision != TLQR_PREC_FP64 && opts->precision != TLQR_PREC_MIXED) return TLQR_ERR_ARG;
  tlqr_factor_t tmp;                       // host-side shell: no CUDA resources
  tmp.plan = plan;
  tmp.opt = *opts;
  tmp.ts = opts->precision == TLQR_PREC_FP64 ? 8 : 4;
  if (select_kernels(&tmp)) return TLQR_ERR_OOM;
  Carve c;
  carve_factor(&tmp, c);
  *bytes = c.off;
  return TLQR_OK;
}

extern "C" int tlqr_async_schedule(const tlqr_plan_t* plan, int32_t n, int32_t which, int32_t async_ops,
                                   int32_t* counts, int32_t* kind, int32_t* node, int32_t* round, int32_t* dep_flag,
                                   int32_t* dep_target, int32_t* signal) {
  if (!plan || !counts || n < 1 || n > TLQR_MAX_DIM || which < 0 || which > 2) return TLQR_ERR_ARG;
  const int R = (int)plan->rounds.size();
  int r0 = which == 0 ? R : 0;
  if (which == 0 && async_ops >= 0) {
    const int thr = async_ops > 0 ? async_ops : kAsyncOps;
    while (r0 > 0) {
      const tlqr_round& r = plan->rounds[r0 - 1];
      if ((r.rake_end - r.rake_begin) + (r.comp_end - r.comp_begin) > thr) break;
      --r0;
    }
  }
  const int G = n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32;
  AsyncPlan A;
  try {
    A = which == 2 ? build_async_state(plan, 32 / G) : build_async(plan, r0, 32 / G);
  } catch (const std::bad_alloc&) {
    return TLQR_ERR_OOM;
  }
  counts[0] = A.r0; counts[1] = A.n_ops; counts[2] = A.n_flags; counts[3] = A.levels;
  if (!kind) return TLQR_OK;
  std::vector<int> seg_round(plan->seg_parent.size(), 0);
  for (int r = 0; r < R; ++r)
    for (int s2 = plan->rounds[r].seg_begin; s2 < plan->rounds[r].seg_end; ++s2) seg_round[s2] = r + 1;
  for (int p = 0; p < A.n_ops; ++p) {
    const int k = A.op[p] >> 28, idx = A.op[p] & fx::kAsyncPad;
    kind[p] = k;
    int v = -1, rr = 0;
    if (idx != fx::kAsyncPad) {
      if (k == fx::AK_RAKE || k == fx::SK_EXPAND_R) { v = plan->rake_leaf[idx]; rr = plan->round_of_node[v]; }
      else if (k == fx::AK_ABSORB) { v = plan->seg_parent[idx]; rr = seg_round[idx]; }
      else { v = plan->comp_j[idx]; rr = plan->round_of_node[v]; }
    }
    if (node) node[p] = v;
    if (round) round[p] = rr;
    for (int d = 0; d < 3; ++d) {
      if (dep_flag) dep_flag[3 * p + d] = A.dep_flag[3 * (size_t)p + d];
      if (dep_target) dep_target[3 * p + d] = A.dep_target[3 * (size_t)p + d];
    }
    if (signal) signal[p] = A.signal[p];
  }
  return TLQR_OK;
}

extern "C" int tlqr_factor_options(const tlqr_factor_t* f, tlqr_options* out) {
  if (!f || !out) return TLQR_ERR_ARG;
  *out = f->opt;
  return TLQR_OK;
}

extern "C" int tlqr_factor_dims(const tlqr_factor_t* f, int32_t* dims) {
  if (!f || !dims) return TLQR_ERR_ARG;
  dims[0] = f->plan->N;
  dims[1] = f->opt.n;
  dims[2] = f->opt.m;
  return TLQR_OK;
}

extern "C" int tlqr_factor_bytes(const tlqr_factor_t* f, size_t* bytes) {
  if (!f || !bytes) return TLQR_ERR_ARG;
  *bytes = f->arena_bytes + f->stage_elems * sizeof(double);
  return TLQR_OK;
}

extern "C" void tlqr_factor_destroy(tlqr_factor_t* f) { delete f; }

extern "C" int tlqr_factor(tlqr_factor_t* f, const tlqr_problem* prob, void* stream) {
  if (!f) return TLQR_ERR_ARG;
  int rc = check_problem(f, prob, false);
  if (rc) return rc;
  StreamScope scope(f, stream);
  cudaStream_t st = scope.st;
  tlqr_problem dp = *prob;
  if (prob->mem == TLQR_MEM_HOST) {
    if ((rc = stage_problem(f, prob, &dp, true, false, st))) return rc;
  }
  return factor_impl(f, &dp, st, true);
}

extern "C" int tlqr_solve_rhs(tlqr_factor_t* f, int32_t mem, const double* q, const double* r,
                              const double* c, double* x, double* u, double* y, void* stream) {
  if (!f || !q || !r || !c || !x || !u || !y) return TLQR_ERR_ARG;
  if (mem != TLQR_MEM_DEVICE && mem != TLQR_MEM_HOST) return TLQR_ERR_ARG;
  if (!f->factored) return TLQR_ERR_STATE;
  StreamScope scope(f, stream);
  cudaStream_t st = scope.st;
  const size_t N = f->plan->N, n = f->opt.n, m = f->opt.m;
  if (mem == TLQR_MEM_DEVICE) {
    if (solve_impl(f, q, r, c, x, u, y, 0, st)) return TLQR_ERR_CUDA;
    return TLQR_OK;
  }
  int rc = ensure_stage(f);
  if (rc) return rc;
  Stage s = stage_layout(f);
  cudaError_t e = h2d(s.q, q, N * n, st);
  if (!e) e = h2d(s.r, r, N * m, st);
  if (!e) e = h2d(s.c, c, N * n, st);
  if (!e) e = solve_impl(f, s.q, s.r, s.c, s.x, s.u, s.y, 0, st);
  if (!e) e = d2h(x, s.x, N * n, st);
  if (!e) e = d2h(u, s.u, N * m, st);
  if (!e) e = d2h(y, s.y, N * n, st);
  if (!e) e = cudaStreamSynchronize(st);
  f->prof.harvest();
  return e ? TLQR_ERR_CUDA : TLQR_OK;
}

extern "C" int tlqr_solve_rhs_panel(tlqr_factor_t* f, int32_t nrhs, const double* q, const double* r,
                                    const double* c, double* x, double* u, double* y, void* stream) {
  if (!f || nrhs < 1 || !q || !r || !c || !x || !u || !y) return TLQR_ERR_ARG;
  if (!f->factored) return TLQR_ERR_STATE;
  StreamScope scope(f, stream);
  cudaStream_t st = scope.st;
  const size_t N = f->plan->N, n = f->opt.n, m = f->opt.m;
  const size_t sv = N * n, sm = N * m;
  // the panel kernels: compile-time (n, m)
  const bool panel = f->fixed_m > 0;
  if (!panel) {
    for (int k = 0; k < nrhs; ++k)
      if (solve_impl(f, q + k * sv, r + k * sm, c + k * sv, x + k * sv, u + k * sm, y + k * sv, 0, st))
        return TLQR_ERR_CUDA;
  } else {
    if (!f->panel_mem) {
      const size_t ts = f->ts, nrake = std::max<size_t>(1, f->plan->rake_leaf.size());
      Carve c0;
      const size_t sizes[7] = {sv, sv, sv, nrake * n, sv, sm, sv};
      for (size_t b : sizes) c0.take(b * kPanel * ts);
      void* mem = nullptr;
      if (cudaMalloc(&mem, c0.off)) { cudaGetLastError(); return TLQR_ERR_OOM; }
      f->panel_mem = mem;
      Carve c1;
      c1.base = static_cast<unsigned char*>(mem);
      void** slots[7] = {&f->panel.h, &f->panel.z, &f->panel.s, &f->panel.cv, &f->panel.bv, &f->panel.kv,
                         &f->panel.xs};
      for (int t = 0; t < 7; ++t) *slots[t] = c1.take(sizes[t] * kPanel * ts);
    }
    for (int k0 = 0; k0 < nrhs; k0 += kPanel) {
      const int kc = std::min(kPanel, nrhs - k0);
      Recorder rcd;
      rcd.mask = f->prof.mask;
      rcd.pool = &f->prof.pool;
      cudaError_t e = f->ts == 8
          ? dispatch_solve<double>(f, &rcd, q + k0 * sv, r + k0 * sm, c + k0 * sv, x + k0 * sv, u + k0 * sm,
                                   y + k0 * sv, 0, st, kc, &f->panel)
          : dispatch_solve<float>(f, &rcd, q + k0 * sv, r + k0 * sm, c + k0 * sv, x + k0 * sv, u + k0 * sm,
                                  y + k0 * sv, 0, st, kc, &f->panel);
      f->prof.add(rcd, true);
      if (e) return TLQR_ERR_CUDA;
    }
  }
  int rc = read_status(f, st);
  f->prof.harvest();
  return rc;
}

namespace {
int get_PK_impl(tlqr_factor_t* f, int32_t mem, double* P, double* K, cudaStream_t st) {
  const size_t N = f->plan->N, n = f->opt.n, m = f->opt.m;
  double *dP = P, *dK = K;
  if (mem == TLQR_MEM_HOST) {
    int rc = ensure_stage(f);
    if (rc) return rc;
    Stage s = stage_layout(f);
    dP = P ? s.P : nullptr;
    dK = K ? s.K : nullptr;
  }
  const int blocks = 4 * f->sms;
  if (f->ts == 8)
    k_export_PK<double><<<blocks, 256, 0, st>>>((int)N, (int)n, (int)m, (const int*)f->dp.parent, (const double*)f->U,
                                                (const double*)f->K, dP, dK);
  else
    k_export_PK<float><<<blocks, 256, 0, st>>>((int)N, (int)n, (int)m, (const int*)f->dp.parent, (const float*)f->U,
                                               (const float*)f->K, dP, dK);
  if (cudaGetLastError()) return TLQR_ERR_CUDA;
  f->prof.launches[TLQR_K_EXPORT]++;
  f->prof.units[TLQR_K_EXPORT] += (int64_t)N;
  if (mem == TLQR_MEM_HOST) {
    cudaError_t e = d2h(P, dP, N * n * n, st);
    if (!e) e = d2h(K, dK, N * m * n, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return TLQR_ERR_CUDA;
  }
  return TLQR_OK;
}
}  // namespace

extern "C" int tlqr_get_PK(tlqr_factor_t* f, int32_t mem, double* P, double* K, void* stream) {
  if (!f) return TLQR_ERR_ARG;
  if (!f->factored) return TLQR_ERR_STATE;
  StreamScope scope(f, stream);
  return get_PK_impl(f, mem, P, K, scope.st);
}

namespace {
// Speculative refinement gate: the largest per-tree eta of the residual just
// evaluated (slot-major maxima [4][T], the reduction of tree_stats) goes to
// gate[0]; when it already meets the tolerance the residual vectors are
// zeroed, so that the correction solve enqueued behind this kernel adds
// exactly zero.  Every block forms eta itself (T words), so no grid sync.
__global__ void k_refine_gate(const unsigned long long* maxes, int T, double tol, double* gate, double* rx,
                              size_t nx, double* ru, size_t nu, double* rc, size_t nc) {
  __shared__ double s_eta;
  if (threadIdx.x == 0) {
    double e = 0.0;
    for (int t = 0; t < T; ++t) {
      const double v0 = __longlong_as_double((long long)maxes[t]);
      const double v1 = __longlong_as_double((long long)maxes[(size_t)T + t]);
      const double v2 = __longlong_as_double((long long)maxes[2 * (size_t)T + t]);
      const double v3 = __longlong_as_double((long long)maxes[3 * (size_t)T + t]);
      const double den = v3 * v1 + v2;
      double et = den > 0 ? v0 / den : v0;
      if (!isfinite(v0)) et = INFINITY;
      if (!(et <= e)) e = et;
    }
    s_eta = e;
    if (blockIdx.x == 0) gate[0] = e;
  }
  __syncthreads();
  if (!(s_eta <= tol)) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nx; t += stride) { rx[t] = 0.0; rc[t] = 0.0; }
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nu; t += stride) ru[t] = 0.0;
}

// FP64 iterative refinement through the FP32 factors: the FP64 residual of
// eq. (kkt) for the problem dp (matrices and right-hand side) is re-solved
// and added to (x, u, y) until the largest per-tree eta <= refine_tol.
// When the previous solve on this factor needed a step, the first step is
// enqueued speculatively (residual, gate, correction, residual) and the host
// waits once; the gate turns the correction into an exact no-op when the first
// residual already met the tolerance, so the result equals the checked loop.
int refine(tlqr_factor_t* f, const tlqr_problem& dp, double* x, double* u, double* y, cudaStream_t st) {
  int steps = 0, rc = 0;
  double absr = 0, eta = INFINITY;
  bool first = true;
  if (f->speculate && f->opt.max_refine >= 1) {
    const size_t N = f->plan->N, n = f->opt.n, m = f->opt.m;
    if (residual_impl(f, dp, x, u, y, 1, st, f->dflag)) return TLQR_ERR_CUDA;
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>((N * n + 255) / 256, (size_t)f->sms * 4));
    k_refine_gate<<<blocks, 256, 0, st>>>(f->maxes, f->plan->n_trees, f->opt.refine_tol, f->d_gate, f->res_x,
                                          N * n, f->res_u, N * m, f->res_c, N * n);
    if (cudaGetLastError()) return TLQR_ERR_CUDA;
    if (cudaMemcpyAsync(f->h_gate, f->d_gate, sizeof(double), cudaMemcpyDeviceToHost, st)) return TLQR_ERR_CUDA;
    if (solve_impl(f, f->res_x, f->res_u, f->res_c, x, u, y, 1, st)) return TLQR_ERR_CUDA;
    if (residual_impl(f, dp, x, u, y, 0, st, f->dflag)) return TLQR_ERR_CUDA;
    if (cudaStreamSynchronize(st)) return TLQR_ERR_CUDA;
    f->prof.harvest();
    if ((rc = map_status(*f->h_status))) { f->factored = false; return rc; }
    residual_stats(f, &absr, &eta);
    steps = f->h_gate[0] <= f->opt.refine_tol ? 0 : 1;
    first = false;
  }
  for (;;) {
    if (first) {
      // residual graph: FP64 residual, ||.|| maxima and the status word to the host
      if (residual_impl(f, dp, x, u, y, 1, st, f->dflag)) return TLQR_ERR_CUDA;
      if (cudaStreamSynchronize(st)) return TLQR_ERR_CUDA;
      f->prof.harvest();
      if ((rc = map_status(*f->h_status))) { f->factored = false; return rc; }
      residual_stats(f, &absr, &eta);
      first = false;
    }
    if (eta <= f->opt.refine_tol || steps >= f->opt.max_refine || !std::isfinite(eta)) break;
    if (solve_impl(f, f->res_x, f->res_u, f->res_c, x, u, y, 1, st)) return TLQR_ERR_CUDA;
    ++steps;
    if (residual_impl(f, dp, x, u, y, 0, st, f->dflag)) return TLQR_ERR_CUDA;
    if (cudaStreamSynchronize(st)) return TLQR_ERR_CUDA;
    f->prof.harvest();
    if ((rc = map_status(*f->h_status))) { f->factored = false; return rc; }
    residual_stats(f, &absr, &eta);
  }
  f->speculate = steps >= 1;
  f->info.refine_steps = steps;
  f->info.eta = eta;
  f->info.abs_residual = absr;
  f->info.fp64_resolves = std::min(f->h_status[1], f->redo_cap);
  if (!std::isfinite(eta)) return TLQR_ERR_NONFINITE;
  if (eta > f->opt.refine_tol) return TLQR_ERR_NO_CONVERGENCE;
  return TLQR_OK;
}
}  // namespace

extern "C" int tlqr_solve_adjoint(tlqr_factor_t* f, int32_t mem, const double* xbar, const double* ubar,
                                  const double* ybar, double* qbar, double* rbar, double* cbar, void* stream) {
  if (!f || !xbar || !ubar || !ybar || !qbar || !rbar || !cbar) return TLQR_ERR_ARG;
  if (mem != TLQR_MEM_DEVICE && mem != TLQR_MEM_HOST) return TLQR_ERR_ARG;
  if (!f->factored) return TLQR_ERR_STATE;
  StreamScope scope(f, stream);
  cudaStream_t st = scope.st;
  const size_t N = f->plan->N, n = f->opt.n, m = f->opt.m;
  const double *q = xbar, *r = ubar, *c = ybar;
  double *x = qbar, *u = rbar, *y = cbar;
  int rc = 0;
  if (mem == TLQR_MEM_HOST) {
    if ((rc = ensure_stage(f))) return rc;
    Stage s = stage_layout(f);
    cudaError_t e = h2d(s.q, xbar, N * n, st);
    if (!e) e = h2d(s.r, ubar, N * m, st);
    if (!e) e = h2d(s.c, ybar, N * n, st);
    if (e) return TLQR_ERR_CUDA;
    q = s.q; r = s.r; c = s.c; x = s.x; u = s.u; y = s.y;
  }
  f->info = tlqr_info{};
  // the KKT matrix of eq. (kkt) is symmetric: the cotangent is the right-hand side
  if (solve_impl(f, q, r, c, x, u, y, 0, st)) return TLQR_ERR_CUDA;
  if (f->opt.precision == TLQR_PREC_MIXED) {
    tlqr_problem dp = f->dprob;
    dp.q = q; dp.r = r; dp.c = c;
    if ((rc = refine(f, dp, x, u, y, st))) return rc;
  }
  if (mem == TLQR_MEM_HOST) {
    cudaError_t e = d2h(qbar, x, N * n, st);
    if (!e) e = d2h(rbar, u, N * m, st);
    if (!e) e = d2h(cbar, y, N * n, st);
    if (e) return TLQR_ERR_CUDA;
  }
  rc = read_status(f, st);
  f->prof.harvest();
  return rc;
}

namespace {
// Factor, solve and (MIXED) refine the device problem dp, writing sol.
int solve_device_problem(tlqr_factor_t* f, const tlqr_problem& dp, tlqr_solution* sol, cudaStream_t st) {
  const size_t N = f->plan->N, n = f->opt.n, m = f->opt.m;
  int rc = 0;
  double *x = sol->x, *u = sol->u, *y = sol->y;
  if (sol->mem == TLQR_MEM_HOST) {
    if ((rc = ensure_stage(f))) return rc;
    Stage s = stage_layout(f);
    x = s.x; u = s.u; y = s.y;
  }
  if ((rc = factor_impl(f, &dp, st, false))) return rc;
  f->info = tlqr_info{};
  if (solve_impl(f, dp.q, dp.r, dp.c, x, u, y, 0, st)) return TLQR_ERR_CUDA;
  if (f->opt.precision == TLQR_PREC_MIXED && (rc = refine(f, dp, x, u, y, st))) return rc;
  if (sol->P || sol->K) {
    if ((rc = get_PK_impl(f, sol->mem, sol->P, sol->K, st))) return rc;
  }
  if (sol->mem == TLQR_MEM_HOST) {
    cudaError_t e = d2h(sol->x, x, N * n, st);
    if (!e) e = d2h(sol->u, u, N * m, st);
    if (!e) e = d2h(sol->y, y, N * n, st);
    if (e) return TLQR_ERR_CUDA;
  }
  // one status read for factor, solve and recovery (synchronises the stream);
  // in MIXED precision the refinement has read it after the last kernel
  // already unless P, K or host copies followed
  if (f->opt.precision != TLQR_PREC_MIXED || sol->P || sol->K || sol->mem == TLQR_MEM_HOST) {
    rc = read_status(f, st);
    f->prof.harvest();
    if (rc) { f->factored = false; return rc; }
  }
  return TLQR_OK;
}

// Q_i += diag(dq_i), R_i += diag(dr_i) in place (either increment may be null).
__global__ void k_add_diagonals(int N, int n, int m, double* Q, const double* dq, double* R, const double* dr) {
  const size_t total = (size_t)N * (n + m);
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    if (t < (size_t)N * n) {
      if (!dq) continue;
      const size_t i = t / n, r = t - i * n;
      Q[i * n * n + r * (n + 1)] += dq[t];
    } else {
      if (!dr) continue;
      const size_t tu = t - (size_t)N * n, i = tu / m, r = tu - i * m;
      R[i * m * m + r * (m + 1)] += dr[tu];
    }
  }
}
}  // namespace

extern "C" int tlqr_solve(tlqr_factor_t* f, const tlqr_problem* prob, tlqr_solution* sol, void* stream) {
  if (!f || !sol || !sol->x || !sol->u || !sol->y) return TLQR_ERR_ARG;
  if (sol->mem != TLQR_MEM_DEVICE && sol->mem != TLQR_MEM_HOST) return TLQR_ERR_ARG;
  int rc = check_problem(f, prob, true);
  if (rc) return rc;
  StreamScope scope(f, stream);
  cudaStream_t st = scope.st;
  tlqr_problem dp = *prob;
  if (prob->mem == TLQR_MEM_HOST) {
    if ((rc = stage_problem(f, prob, &dp, true, true, st))) return rc;
  }
  return solve_device_problem(f, dp, sol, st);
}

extern "C" int tlqr_update_solve(tlqr_factor_t* f, int32_t mem, const double* dq, const double* dr, const double* q,
                                 const double* r, const double* c, tlqr_solution* sol, void* stream) {
  if (!f || !sol || !sol->x || !sol->u || !sol->y) return TLQR_ERR_ARG;
  if (mem != TLQR_MEM_DEVICE && mem != TLQR_MEM_HOST) return TLQR_ERR_ARG;
  if (sol->mem != TLQR_MEM_DEVICE && sol->mem != TLQR_MEM_HOST) return TLQR_ERR_ARG;
  if (!f->dprob.Q || !f->dprob.R || !f->dprob.q) return TLQR_ERR_STATE;   // nothing resident yet
  StreamScope scope(f, stream);
  cudaStream_t st = scope.st;
  const size_t N = f->plan->N, n = f->opt.n, m = f->opt.m;
  tlqr_problem dp = f->dprob;
  const double *ddq = dq, *ddr = dr;
  int rc = 0;
  if (mem == TLQR_MEM_HOST) {
    // the right-hand side goes to the staging area; the increments to a scratch
    // of N (n + m) doubles (the staged P block, unused until P is exported)
    if ((rc = ensure_stage(f))) return rc;
    Stage s = stage_layout(f);
    cudaError_t e = cudaSuccess;
    if (q) { e = h2d(s.q, q, N * n, st); dp.q = s.q; }
    if (!e && r) { e = h2d(s.r, r, N * m, st); dp.r = s.r; }
    if (!e && c) { e = h2d(s.c, c, N * n, st); dp.c = s.c; }
    double* inc = N * n * n >= N * (n + m) ? s.P : nullptr;
    if (!inc && (dq || dr)) {
      if (!f->upd) {
        f->upd = dalloc<double>(N * (n + m), &e);
        if (e) return TLQR_ERR_OOM;
        f->allocs.push_back(f->upd);
      }
      inc = f->upd;
    }
    if (!e && dq) { e = h2d(inc, dq, N * n, st); ddq = inc; }
    if (!e && dr) { e = h2d(inc + N * n, dr, N * m, st); ddr = inc + N * n; }
    if (e) return TLQR_ERR_CUDA;
  } else {
    if (q) dp.q = q;
    if (r) dp.r = r;
    if (c) dp.c = c;
  }
  if (ddq || ddr) {
    const size_t total = N * (n + m);
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, (size_t)f->sms * 8));
    k_add_diagonals<<<blocks, 256, 0, st>>>((int)N, (int)n, (int)m, const_cast<double*>(dp.Q), ddq,
                                            const_cast<double*>(dp.R), ddr);
    if (cudaGetLastError()) return TLQR_ERR_CUDA;
  }
  return solve_device_problem(f, dp, sol, st);
}

extern "C" int tlqr_kkt_residual(tlqr_factor_t* f, const tlqr_problem* prob, int32_t mem, const double* x,
                                 const double* u, const double* y, double* stats, void* stream) {
  if (!f || !x || !u || !y || !stats) return TLQR_ERR_ARG;
  int rc = check_problem(f, prob, true);
  if (rc) return rc;
  StreamScope scope(f, stream);
  cudaStream_t st = scope.st;
  const size_t N = f->plan->N, n = f->opt.n, m = f->opt.m;
  tlqr_problem dp = *prob;
  if (prob->mem == TLQR_MEM_HOST) {
    if ((rc = stage_problem(f, prob, &dp, true, true, st))) return rc;
  }
  const double *dx = x, *du = u, *dy = y;
  if (mem == TLQR_MEM_HOST) {
    if ((rc = ensure_stage(f))) return rc;
    Stage s = stage_layout(f);
    if (h2d(s.x, x, N * n, st) || h2d(s.u, u, N * m, st) || h2d(s.y, y, N * n, st)) return TLQR_ERR_CUDA;
    dx = s.x; du = s.u; dy = s.y;
  }
  if (run_residual(f, nullptr, dp, dx, du, dy, 1, st) || cudaStreamSynchronize(st)) return TLQR_ERR_CUDA;
  residual_stats(f, &stats[0], &stats[1]);
  return TLQR_OK;
}

extern "C" int tlqr_tree_residuals(const tlqr_factor_t* f, double* abs_res, double* eta, int32_t max_trees) {
  if (!f || max_trees < 0) return TLQR_ERR_ARG;
  const int T = std::min<int>(f->plan->n_trees, max_trees);
  for (int t = 0; t < T; ++t) {
    double a, e;
    tree_stats(f, t, &a, &e);
    if (abs_res) abs_res[t] = a;
    if (eta) eta[t] = e;
  }
  return TLQR_OK;
}

extern "C" int tlqr_last_info(const tlqr_factor_t* f, tlqr_info* out) {
  if (!f || !out) return TLQR_ERR_ARG;
  *out = f->info;
  return TLQR_OK;
}

// ------------------------------------------------------- batched primitives

namespace {

// FP64 <-> working precision on the device (a plain copy when both are FP64).
template <typename D, typename S>
__global__ void k_convert(D* dst, const S* src, size_t count) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (D)src[e];
}
template <typename D, typename S>
cudaError_t convert(D* dst, const S* src, size_t count, int sms, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int blocks = (int)std::min<size_t>((count + 255) / 256, (size_t)sms * 8);
  k_convert<D, S><<<blocks, 256, 0, st>>>(dst, src, count);
  return cudaGetLastError();
}

enum { B_TAU = 0, B_COMPOSE, B_CONDENSE, B_EXPAND, B_LOCAL_FACTOR, B_COMPOSE_T };

// Launch one batched primitive with the compile-time-(n, m) group kernels the
// solver itself runs for this n (NF > 0; at n = 32 in FP32 with the
// tensor-core block products), or the run-time-n warp kernels (NF == 0).
template <typename T, int NF, int MF>
cudaError_t batched_launch(int kind, const Ws<T>& w, int count, int n, int m, cudaStream_t st) {
  const WarpBytes wb = warp_bytes(n, m, sizeof(T));
  constexpr int NX = NF > 0 ? NF : 4;
  constexpr int MX = MF > 0 ? MF : 2;
  constexpr int G = fx::D<T, NX>::G;
  switch (kind) {
    case B_TAU:
      if constexpr (NF > 0) return launch_groups(nullptr, TLQR_K_RAKE, fx::kf_rake<T, NX>, count, G, fx::TauSmem<T, NX>::bytes, st, w, 0, count);
      return launch_warps(nullptr, TLQR_K_RAKE, k_rake<T>, count, wb.tau, st, w, 0, count, (int)wb.tau);
    case B_EXPAND:
      if constexpr (NF > 0) return launch_groups(nullptr, TLQR_K_EXPAND, fx::kf_expand<T, NX>, count, G, fx::TauSmem<T, NX>::bytes, st, w, 0, count);
      return launch_warps(nullptr, TLQR_K_EXPAND, k_expand<T>, count, wb.tau, st, w, 0, count, (int)wb.tau);
    case B_COMPOSE:
      if constexpr (NF > 0) return launch_groups(nullptr, TLQR_K_COMPRESS, fx::kf_compress<T, NX>, count, G, fx::CompSmem<T, NX>::bytes, st, w, 0, count);
      return launch_warps(nullptr, TLQR_K_COMPRESS, k_compress<T>, count, wb.compress, st, w, 0, count, (int)wb.compress);
    case B_COMPOSE_T:
      if constexpr (NF > 0) return launch_groups(nullptr, TLQR_K_COMPOSE_T, fx::kf_compose_T<T, NX>, count, G, fx::ComposeSmem<T, NX>::bytes, st, w, 0, count);
      return launch_warps(nullptr, TLQR_K_COMPOSE_T, k_compose_T<T>, count, wb.compose_T, st, w, 0, count, (int)wb.compose_T);
    case B_CONDENSE:
      if constexpr (MF > 0) return launch_groups(nullptr, TLQR_K_CONDENSE, fx::kf_condense<T, NX, MX>, count, G, fx::CondSmem<T, NX, MX>::bytes, st, w, count);
      return launch_warps(nullptr, TLQR_K_CONDENSE, k_condense<T>, count, wb.condense, st, w, (int)wb.condense);
    case B_LOCAL_FACTOR:
      if constexpr (MF > 0) return launch_groups(nullptr, TLQR_K_LOCAL_FACTOR, fx::kf_local_factor<T, NX, MX>, count, G, fx::LfSmem<T, NX, MX>::bytes, st, w, count);
      return launch_warps(nullptr, TLQR_K_LOCAL_FACTOR, k_local_factor<T>, count, wb.local_factor, st, w, (int)wb.local_factor);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t batched_dispatch(int kind, const Ws<T>& w, int count, int n, int m, int generic, cudaStream_t st) {
  const bool nm_kind = kind == B_CONDENSE || kind == B_LOCAL_FACTOR;
  if (!generic) {
#define X(n_, m_)                                                                       \
    if constexpr (fixed_for<T>(n_))                                                     \
      if (n == n_ && (m_ == 0 ? !nm_kind || !has_fixed_pair(n, m) : (nm_kind && m == m_))) \
        return batched_launch<T, n_, m_>(kind, w, count, n, m, st);
    TLQR_FIXED_CASES(X)
#undef X
  }
  return batched_launch<T, 0, 0>(kind, w, count, n, m, st);
}

// Batched primitives: count independent problems in contiguous FP64 device
// arrays.  Slots 0..count-1 of the workspace hold the "left" operands (the
// edge into a compressed centre, the tape, the node whose factor is built),
// slots count..2count-1 the "right" ones; index arrays map operation t to
// slots t and count + t.  Inputs are converted to T and results back to FP64
// by device kernels on `stream`.
template <typename T>
int batched_ops(int kind, int count, int n, int m, const double* const* in, double* const* out, int generic,
                cudaStream_t st) {
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  const size_t S = 2 * (size_t)count;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) || sms < 1)
    return TLQR_ERR_CUDA;
  std::vector<void*> mine;
  cudaError_t err = cudaSuccess;
  auto take = [&](size_t elems, size_t es) -> void* {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(1, elems) * es);
    if (e != cudaSuccess) { if (err == cudaSuccess) err = e; return nullptr; }
    mine.push_back(p);
    return p;
  };
  Ws<T> w{};
  w.N = count; w.n = n; w.m = m;
  T *U = (T*)take(S * nn, sizeof(T)), *Ea = (T*)take(S * nn, sizeof(T)), *Ec = (T*)take(S * nn, sizeof(T)),
    *Ep = (T*)take(S * nn, sizeof(T)), *contrib = (T*)take(count * nn, sizeof(T));
  T *K = (T*)take(count * nm, sizeof(T)), *Tm = (T*)take(S * nn, sizeof(T)), *Tr = (T*)take(count * nn, sizeof(T)),
    *W = (T*)take(count * nn, sizeof(T)), *Finv = (T*)take(count * nn, sizeof(T)),
    *LG = (T*)take(count * mm, sizeof(T));
  int* idx = (int*)take(S, sizeof(int));
  int* status = (int*)take(2, sizeof(int));            // status word, FP64 re-solve tickets
  double* zeros = (double*)take(count * nn, sizeof(double));
  unsigned char* flags = (unsigned char*)take(count, 1);
  // FP32 compile-time-n kernels: one FP64 re-solve slot per operation (the solver's rule)
  double* redo = (sizeof(T) == 4 && !generic) ? (double*)take((size_t)count * 3 * nn, sizeof(double)) : nullptr;
  if (err) { for (void* p : mine) cudaFree(p); return TLQR_ERR_OOM; }
  if (redo) {
    w.redo_count = status + 1;
    w.redo_cap = count;
    w.redo_scratch = redo;
    w.redo_slot = 3 * nn;
  }
  std::vector<int> hidx(S);
  for (size_t t = 0; t < S; ++t) hidx[t] = (int)t;
  cudaError_t e = cudaMemcpyAsync(idx, hidx.data(), S * sizeof(int), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemsetAsync(status, 0, 2 * sizeof(int), st);
  w.U = U; w.Ea = Ea; w.Ec = Ec; w.Ep = Ep; w.contrib = contrib; w.status = status;
  w.K = K; w.Tm = Tm; w.Tr = Tr; w.W = W; w.Finv = Finv; w.LG = LG;
  auto in_ = [&](T* dst, const double* src, size_t elems) { if (!e) e = convert(dst, src, elems, sms, st); };
  auto out_ = [&](double* dst, const T* src, size_t elems) { if (!e) e = convert(dst, src, elems, sms, st); };
  const size_t L = (size_t)count * nn;
  switch (kind) {
    case B_TAU:                 // in = A, C, P, U; out = P + A^T U (I + C U)^{-1} A
      in_(Ea, in[0], L); in_(Ec, in[1], L); in_(Ep, in[2], L); in_(U, in[3], L);
      w.rake_leaf = idx;
      if (!e) e = batched_dispatch<T>(kind, w, count, n, m, generic, st);
      out_(out[0], contrib, L);
      break;
    case B_EXPAND:              // in = Ar, Cr, Pt (tape into slot t), Pk (slot count + t); out = P_j (slot t)
      in_(Ea, in[0], L); in_(Ec, in[1], L); in_(Ep, in[2], L); in_(U + L, in[3], L);
      w.comp_j = idx; w.comp_k = idx + count;
      if (!e) e = batched_dispatch<T>(kind, w, count, n, m, generic, st);
      out_(out[0], U, L);
      break;
    case B_COMPOSE:             // in = Al Cl Pl (slot t) Ar Cr Pr (slot count + t) U (slot t)
      in_(Ea, in[0], L); in_(Ec, in[1], L); in_(Ep, in[2], L);
      in_(Ea + L, in[3], L); in_(Ec + L, in[4], L); in_(Ep + L, in[5], L); in_(U, in[6], L);
      w.comp_j = idx; w.comp_k = idx + count;
      if (!e) e = batched_dispatch<T>(kind, w, count, n, m, generic, st);
      out_(out[0], Ea + L, L); out_(out[1], Ec + L, L); out_(out[2], Ep + L, L); out_(out[3], Ep, L);
      break;
    case B_COMPOSE_T:           // in = T_k (slot count + t), T_j (slot t); out = T_k T_j
      in_(Tm + L, in[0], L); in_(Tm, in[1], L);
      w.comp_j = idx; w.comp_k = idx + count;
      if (!e) e = batched_dispatch<T>(kind, w, count, n, m, generic, st);
      out_(out[0], Tm + L, L);
      break;
    case B_CONDENSE:            // in = A B R M Delta (FP64, read directly); U <- Q = 0
      w.A = in[0]; w.B = in[1]; w.R = in[2]; w.M = in[3]; w.Delta = in[4];
      w.has_M = in[3] != nullptr; w.has_delta = in[4] != nullptr;
      w.Q = zeros;
      if (!e) e = cudaMemsetAsync(zeros, 0, L * sizeof(double), st);
      w.dflag = flags;
      if (!e) e = batched_dispatch<T>(kind, w, count, n, m, generic, st);
      out_(out[0], Ea, L); out_(out[1], Ec, L); out_(out[2], Ep, L);
      break;
    case B_LOCAL_FACTOR:        // in = P, A B R M Delta; out = K [m x n], T = F^{-1} A_cl
      in_(U, in[0], L);
      w.A = in[1]; w.B = in[2]; w.R = in[3]; w.M = in[4]; w.Delta = in[5];
      w.has_M = in[4] != nullptr; w.has_delta = in[5] != nullptr;
      w.dflag = flags;
      if (!e) e = cudaMemsetAsync(flags, w.has_delta ? 1 : 0, count, st);
      if (!e) e = batched_dispatch<T>(kind, w, count, n, m, generic, st);
      out_(out[0], K, (size_t)count * nm); out_(out[1], Tm, L);
      break;
    default:
      e = cudaErrorInvalidValue;
  }
  int hs = 0;
  if (!e) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  for (void* p : mine) cudaFree(p);
  if (e) return TLQR_ERR_CUDA;
  return map_status(hs);
}

int batched(int kind, int count, int n, int m, const double* const* in, double* const* out, int32_t precision,
            void* stream) {
  const int generic = (precision >> 8) & 1;
  const int prec = precision & 0xff;
  if (prec != TLQR_PREC_FP64 && prec != TLQR_PREC_MIXED) return TLQR_ERR_ARG;
  return prec == TLQR_PREC_FP64 ? batched_ops<double>(kind, count, n, m, in, out, generic, (cudaStream_t)stream)
                                : batched_ops<float>(kind, count, n, m, in, out, generic, (cudaStream_t)stream);
}

}  // namespace

extern "C" int tlqr_batched_tau(int32_t count, int32_t n, const double* A, const double* C,
                                const double* P, const double* U, double* out, int32_t precision,
                                void* stream) {
  if (count < 1 || n < 1 || n > TLQR_MAX_DIM || !A || !C || !P || !U || !out) return TLQR_ERR_ARG;
  const double* in[4] = {A, C, P, U};
  double* o[1] = {out};
  return batched(B_TAU, count, n, 1, in, o, precision, stream);
}

extern "C" int tlqr_batched_compose(int32_t count, int32_t n, const double* Al, const double* Cl,
                                    const double* Pl, const double* Ar, const double* Cr, const double* Pr,
                                    const double* U, double* An, double* Cn, double* Pn, double* Pt,
                                    int32_t precision, void* stream) {
  if (count < 1 || n < 1 || n > TLQR_MAX_DIM || !Al || !Cl || !Pl || !Ar || !Cr || !Pr || !U || !An || !Cn ||
      !Pn || !Pt)
    return TLQR_ERR_ARG;
  const double* in[7] = {Al, Cl, Pl, Ar, Cr, Pr, U};
  double* o[4] = {An, Cn, Pn, Pt};
  return batched(B_COMPOSE, count, n, 1, in, o, precision, stream);
}

extern "C" int tlqr_batched_condense(int32_t count, int32_t n, int32_t m, const double* A, const double* B,
                                     const double* R, const double* M, const double* Delta, double* Abar,
                                     double* Cbar, double* Pbar, int32_t precision, void* stream) {
  if (count < 1 || n < 1 || m < 1 || n > TLQR_MAX_DIM || m > TLQR_MAX_DIM || !A || !B || !R || !Abar ||
      !Cbar || !Pbar)
    return TLQR_ERR_ARG;
  const double* in[5] = {A, B, R, M, Delta};
  double* o[3] = {Abar, Cbar, Pbar};
  return batched(B_CONDENSE, count, n, m, in, o, precision, stream);
}

extern "C" int tlqr_batched_expand(int32_t count, int32_t n, const double* Ar, const double* Cr,
                                   const double* Pt, const double* Pk, double* Pj, int32_t precision,
                                   void* stream) {
  if (count < 1 || n < 1 || n > TLQR_MAX_DIM || !Ar || !Cr || !Pt || !Pk || !Pj) return TLQR_ERR_ARG;
  const double* in[4] = {Ar, Cr, Pt, Pk};
  double* o[1] = {Pj};
  return batched(B_EXPAND, count, n, 1, in, o, precision, stream);
}

extern "C" int tlqr_batched_local_factor(int32_t count, int32_t n, int32_t m, const double* P, const double* A,
                                         const double* B, const double* R, const double* M, const double* Delta,
                                         double* K, double* T, int32_t precision, void* stream) {
  if (count < 1 || n < 1 || m < 1 || n > TLQR_MAX_DIM || m > TLQR_MAX_DIM || !P || !A || !B || !R || !K || !T)
    return TLQR_ERR_ARG;
  const double* in[6] = {P, A, B, R, M, Delta};
  double* o[2] = {K, T};
  return batched(B_LOCAL_FACTOR, count, n, m, in, o, precision, stream);
}

extern "C" int tlqr_batched_compose_T(int32_t count, int32_t n, const double* Tk, const double* Tj, double* out,
                                      int32_t precision, void* stream) {
  if (count < 1 || n < 1 || n > TLQR_MAX_DIM || !Tk || !Tj || !out) return TLQR_ERR_ARG;
  const double* in[2] = {Tk, Tj};
  double* o[1] = {out};
  return batched(B_COMPOSE_T, count, n, 1, in, o, precision, stream);
}

extern "C" int tlqr_profile_mask(tlqr_factor_t* f, uint32_t mask) {
  if (!f) return TLQR_ERR_ARG;
  f->prof.mask = mask;
  return TLQR_OK;
}

extern "C" int tlqr_profile_read(tlqr_factor_t* f, tlqr_kernel_profile* out) {
  if (!f || !out) return TLQR_ERR_ARG;
  f->prof.harvest();
  for (int k = 0; k < TLQR_K_COUNT; ++k) {
    out[k] = tlqr_kernel_profile{f->prof.launches[k], f->prof.units[k], f->prof.timed[k], f->prof.ms[k]};
    f->prof.launches[k] = f->prof.units[k] = f->prof.timed[k] = 0;
    f->prof.ms[k] = 0.0;
  }
  const bool bad = f->prof.event_error;
  f->prof.event_error = false;
  f->prof.log.clear();
  return bad ? TLQR_ERR_CUDA : TLQR_OK;
}

extern "C" int tlqr_profile_launches(tlqr_factor_t* f, int32_t* kind, int64_t* units, double* ms, int32_t max,
                                     int32_t* count) {
  if (!f || !count || max < 0) return TLQR_ERR_ARG;
  f->prof.harvest();
  const int32_t n = (int32_t)f->prof.log.size();
  *count = n;
  for (int32_t t = 0; t < n && t < max; ++t) {
    if (kind) kind[t] = f->prof.log[t].kind;
    if (units) units[t] = f->prof.log[t].units;
    if (ms) ms[t] = f->prof.log[t].ms;
  }
  return TLQR_OK;
}
