// Autotuner (tlqr_autotune): picks the execution shape of the factorisation
// and of the right-hand-side passes for one plan and problem by timing them on
// the device that runs them.  Candidates: the round from which the
// factorisation runs level-asynchronously (async_ops), and the right-hand-side
// passes either level-asynchronous (async_solve = 1) or round by round with a
// single-block tail of tail_ops operations (or none).  Each candidate is a factor object
// of its own; one full tlqr_solve (factor, solve, refinement) warms it up and
// the median of `trials` timed solves (CUDA events on `stream`) scores it.
// In mixed precision the refinement's residual kernels (row per thread, or
// node-organised with bulk-copy staging) are then tried on the fastest shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/tlqr.h"

extern "C" int tlqr_autotune(const tlqr_plan_t* plan, const tlqr_options* base, const tlqr_problem* prob,
                             int32_t trials, tlqr_options* best, tlqr_autotune_entry* table, int32_t max_entries,
                             int32_t* n_entries, void* stream) {
  if (!plan || !base || !prob || !best || trials < 1) return TLQR_ERR_ARG;
  if (prob->mem != TLQR_MEM_DEVICE) return TLQR_ERR_ARG;
  tlqr_plan_stats_t ps{};
  int rc = tlqr_plan_stats(plan, &ps);
  if (rc) return rc;
  const size_t N = (size_t)ps.N, n = (size_t)base->n, m = (size_t)base->m;
  struct Cand { int32_t async_ops, async_solve, tail_ops, residual; };
  std::vector<Cand> cands;
  for (int32_t a : {-1, 256, 1024, 4096}) {
    cands.push_back({a, 1, 0, base->residual});
    for (int32_t t : {-1, 64, 128, 512}) cands.push_back({a, -1, t, base->residual});
  }
  const size_t n_shapes = cands.size();
  const bool tune_residual = base->precision == TLQR_PREC_MIXED && base->residual == 0;
  cudaStream_t st = (cudaStream_t)stream;
  double *x = nullptr, *u = nullptr, *y = nullptr;
  if (cudaMalloc((void**)&x, N * n * sizeof(double)) || cudaMalloc((void**)&u, N * m * sizeof(double)) ||
      cudaMalloc((void**)&y, N * n * sizeof(double))) {
    cudaGetLastError();
    cudaFree(x); cudaFree(u); cudaFree(y);
    return TLQR_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  tlqr_solution sol{};
  sol.mem = TLQR_MEM_DEVICE;
  sol.x = x; sol.u = u; sol.y = y;
  double best_ms = 0;
  int count = 0;
  *best = *base;
  for (size_t ci = 0;; ++ci) {
    if (ci == n_shapes && tune_residual && best_ms > 0) {
      // second stage: the residual kernels on the fastest shape
      for (int32_t r : {1, 2}) cands.push_back({best->async_ops, best->async_solve, best->tail_ops, r});
    }
    if (ci >= cands.size()) break;
    const Cand c = cands[ci];
    tlqr_options o = *base;
    o.async_ops = c.async_ops;
    o.async_solve = c.async_solve;
    o.tail_ops = c.tail_ops;
    o.residual = c.residual;
    tlqr_factor_t* f = nullptr;
    double ms = -1.0;
    int status = tlqr_factor_create(plan, &o, &f);
    if (!status) status = tlqr_solve(f, prob, &sol, stream);            // warm-up, graph capture
    if (!status) {
      std::vector<float> t;
      for (int k = 0; k < trials && !status; ++k) {
        cudaEventRecord(e0, st);
        status = tlqr_solve(f, prob, &sol, stream);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float v = 0.f;
        cudaEventElapsedTime(&v, e0, e1);
        t.push_back(v);
      }
      if (!status) {
        std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
        ms = t[t.size() / 2];
      }
    }
    if (f) tlqr_factor_destroy(f);
    if (table && count < max_entries) {
      table[count].async_ops = c.async_ops;
      table[count].async_solve = c.async_solve;
      table[count].tail_ops = c.tail_ops;
      table[count].residual = c.residual;
      table[count].status = status;
      table[count].ms = ms;
    }
    ++count;
    if (!status && ms >= 0 && (best_ms == 0 || ms < best_ms)) {
      best_ms = ms;
      *best = o;
    }
    if (status && status != TLQR_ERR_NO_CONVERGENCE && status != TLQR_ERR_OOM) { rc = status; break; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x); cudaFree(u); cudaFree(y);
  if (n_entries) *n_entries = std::min(count, max_entries);
  if (rc) return rc;
  return best_ms > 0 ? TLQR_OK : TLQR_ERR_NO_CONVERGENCE;
}
