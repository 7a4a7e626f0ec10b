// Primal-dual interior-point driver for box-constrained tree LQR
// (tlqr_ipm_box): the call pattern of an interior-point method that uses the
// tree solver for its Newton systems (Sec. IX-B, XI-B).  The problem of
// eq. (1)-(2) gets bounds u_lo <= u_e <= u_hi on every control component
// (infinite = absent).  With slacks s_lo = u - u_lo, s_hi = u_hi - u and
// multipliers l_lo, l_hi > 0, the Newton point for barrier parameter mu is the
// solution of the tree KKT system with
//     R~ = R + diag(S),  r~ = r - S u - mu / s_lo + mu / s_hi,
//     S = l_lo / s_lo + l_hi / s_hi,
// so every iteration is one tlqr_solve on the same plan and factor object
// (its captured launch graphs are reused: the buffers do not move).  The
// multiplier steps follow from linearising l s = mu; the step length keeps
// slacks and multipliers positive (fraction to the boundary tau); then
// mu <- sigma * mean(l s).  At convergence the multipliers are recovered from
// the control rows of the KKT system.  Everything per component runs in device kernels;
// the host reads two numbers per iteration (step length and gap).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/tlqr.h"
#include "plan.hpp"

namespace {

struct Ipm {
  int N, n, m;
  const unsigned char* edge;       // [N] 1 for a nonroot node (its edge carries a control)
  const double *R, *r, *lo, *hi;
  double *Rt, *rt;                 // Newton system data
  double *x, *u, *y;               // current iterate (caller's output buffers)
  double *xp, *up, *yp;            // Newton point
  double *l_lo, *l_hi, *du, *dl_lo, *dl_hi;
  unsigned long long* alpha_bits;  // step length (bits of a positive double, atomicMin)
  double* gap;                     // sum of l s over the bounded components
  double* gap_part;                // [gridDim.x] per-block partial sums (fixed order: deterministic)
  unsigned long long* smax_bits;   // largest barrier term l / s after the step (atomicMax of bits)
  const int* parent;               // [N] the plan's parent array
};

// Block sum of one double per thread in a fixed order (shuffles, then warp
// partials by thread 0); returns the total in thread 0.
__device__ double block_sum(double v) {
  __shared__ double part[32];
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) t += part[w];
  return t;
}

__device__ __forceinline__ bool bounded(double b) { return isfinite(b); }

// Interior start: box midpoint (one unit inside a one-sided bound), l = mu0 / s.
__global__ void k_ipm_init(Ipm a, double mu0) {
  const size_t total = (size_t)a.N * a.m;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / a.m);
    const double lo = a.lo[t], hi = a.hi[t];
    const bool on = a.edge[j], hl = on && bounded(lo), hh = on && bounded(hi);
    const double u = !on ? 0.0 : (hl && hh) ? 0.5 * (lo + hi) : hl ? lo + 1.0 : hh ? hi - 1.0 : 0.0;
    a.u[t] = u;
    a.l_lo[t] = hl ? mu0 / (u - lo) : 0.0;
    a.l_hi[t] = hh ? mu0 / (hi - u) : 0.0;
  }
  const size_t nx = (size_t)a.N * a.n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nx; t += (size_t)gridDim.x * blockDim.x) {
    a.x[t] = 0.0;
    a.y[t] = 0.0;
  }
}

// R~, r~ of the Newton system; also resets the step length and the gap.
__global__ void k_ipm_form(Ipm a, double mu) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.alpha_bits = (unsigned long long)__double_as_longlong(1.0);
  const int m = a.m;
  const size_t total = (size_t)a.N * m;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / m), c = (int)(t - (size_t)j * m);
    const double lo = a.lo[t], hi = a.hi[t], u = a.u[t];
    const bool on = a.edge[j], hl = on && bounded(lo), hh = on && bounded(hi);
    const double s_lo = hl ? u - lo : 1.0, s_hi = hh ? hi - u : 1.0;
    const double S = (hl ? a.l_lo[t] / s_lo : 0.0) + (hh ? a.l_hi[t] / s_hi : 0.0);
    const double* Rrow = a.R + (size_t)j * m * m + (size_t)c * m;
    double* Rtrow = a.Rt + (size_t)j * m * m + (size_t)c * m;
    for (int b = 0; b < m; ++b) Rtrow[b] = Rrow[b] + (b == c ? S : 0.0);
    a.rt[t] = a.r[t] - S * u - (hl ? mu / s_lo : 0.0) + (hh ? mu / s_hi : 0.0);
  }
}

// Step directions of u and the multipliers, and the largest step that keeps
// every slack and multiplier positive (times tau).
__global__ void k_ipm_step(Ipm a, double mu, double tau) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.smax_bits = 0ull;
  double amin = 1.0;
  const size_t total = (size_t)a.N * a.m;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / a.m);
    const double lo = a.lo[t], hi = a.hi[t], u = a.u[t];
    const bool on = a.edge[j], hl = on && bounded(lo), hh = on && bounded(hi);
    const double du = on ? a.up[t] - u : 0.0;
    double dll = 0.0, dlh = 0.0;
    if (hl) {
      const double s = u - lo, l = a.l_lo[t];
      dll = mu / s - l - (l / s) * du;
      if (du < 0) amin = fmin(amin, -tau * s / du);
      if (dll < 0) amin = fmin(amin, -tau * l / dll);
    }
    if (hh) {
      const double s = hi - u, l = a.l_hi[t];
      dlh = mu / s - l + (l / s) * du;
      if (du > 0) amin = fmin(amin, tau * s / du);
      if (dlh < 0) amin = fmin(amin, -tau * l / dlh);
    }
    a.du[t] = du;
    a.dl_lo[t] = dll;
    a.dl_hi[t] = dlh;
  }
  for (int off = 16; off; off >>= 1) amin = fmin(amin, __shfl_xor_sync(0xffffffffu, amin, off));
  if ((threadIdx.x & 31) == 0 && amin < 1.0)
    atomicMin(a.alpha_bits, (unsigned long long)__double_as_longlong(fmax(amin, 0.0)));
}

// Take the step and sum the new complementarity gap.
__global__ void k_ipm_update(Ipm a) {
  const double alpha = __longlong_as_double((long long)*a.alpha_bits);
  double g = 0.0, smax = 0.0;
  const size_t total = (size_t)a.N * a.m;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / a.m);
    const double lo = a.lo[t], hi = a.hi[t];
    const bool on = a.edge[j], hl = on && bounded(lo), hh = on && bounded(hi);
    const double u = on ? a.u[t] + alpha * a.du[t] : 0.0;
    a.u[t] = u;
    if (hl) {
      a.l_lo[t] += alpha * a.dl_lo[t];
      g += a.l_lo[t] * (u - lo);
      smax = fmax(smax, a.l_lo[t] / (u - lo));
    }
    if (hh) {
      a.l_hi[t] += alpha * a.dl_hi[t];
      g += a.l_hi[t] * (hi - u);
      smax = fmax(smax, a.l_hi[t] / (hi - u));
    }
  }
  for (int off = 16; off; off >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, off));
  if ((threadIdx.x & 31) == 0 && smax > 0.0)
    atomicMax(a.smax_bits, (unsigned long long)__double_as_longlong(isnan(smax) ? INFINITY : smax));
  const size_t nx = (size_t)a.N * a.n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nx; t += (size_t)gridDim.x * blockDim.x) {
    a.x[t] += alpha * (a.xp[t] - a.x[t]);
    a.y[t] += alpha * (a.yp[t] - a.y[t]);
  }
  const double b = block_sum(g);
  if (threadIdx.x == 0) a.gap_part[blockIdx.x] = b;
}

// Dual recovery at convergence: each control row of eq. (kkt) with the bound
// multipliers, g - l_lo + l_hi = 0 with g = R u + r + M^T x_parent + B^T y, fixes
// l_lo - l_hi = g; split by sign (l_lo = max(g, 0), l_hi = max(-g, 0) where the
// bound exists).  The updated multipliers of the last Newton step carry the
// rounding of the barrier terms l / s ~ 1 / tol on the active rows; these
// satisfy stationarity to ordinary rounding, and l s stays at the scale of the
// final gap (g vanishes on inactive rows, s on active ones).
__global__ void k_ipm_duals(Ipm a, const double* M, const double* B) {
  const int n = a.n, m = a.m;
  const size_t total = (size_t)a.N * m;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / m), c = (int)(t - (size_t)j * m);
    if (!a.edge[j]) continue;
    const int i = a.parent[j];
    double g = a.r[t];
    for (int b = 0; b < m; ++b) g += a.R[(size_t)j * m * m + (size_t)c * m + b] * a.u[(size_t)j * m + b];
    for (int q = 0; q < n; ++q) {
      g += B[(size_t)j * n * m + (size_t)q * m + c] * a.y[(size_t)j * n + q];
      if (M) g += M[(size_t)j * n * m + (size_t)q * m + c] * a.x[(size_t)i * n + q];
    }
    const bool hl = bounded(a.lo[t]), hh = bounded(a.hi[t]);
    if (hl) a.l_lo[t] = g > 0 ? g : 0.0;
    if (hh) a.l_hi[t] = g < 0 ? -g : 0.0;
  }
}

// The gap: the block partials summed in block order by one thread.
__global__ void k_ipm_gap(Ipm a, int parts) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double g = 0.0;
    for (int t = 0; t < parts; ++t) g += a.gap_part[t];
    *a.gap = g;
  }
}

// An FP64 factor object can stand in for a MIXED one.
bool o64_possible(const tlqr_factor_t* f) {
  tlqr_options o{};
  return tlqr_factor_options(f, &o) == TLQR_OK && o.precision == TLQR_PREC_MIXED;
}

bool device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Largest barrier term l / s at which a MIXED factor object still solves the
// Newton systems; beyond it the driver switches to FP64.
constexpr double kIpmSwitch = 1e6;

}  // namespace

extern "C" int tlqr_ipm_box(const tlqr_plan_t* plan, tlqr_factor_t* f, const tlqr_problem* prob,
                            const double* u_lo, const double* u_hi, const tlqr_ipm_options* opts, double* x,
                            double* u, double* y, double* lam_lo, double* lam_hi, tlqr_ipm_info* info,
                            void* stream) {
  if (!plan || !f || !prob || !u_lo || !u_hi || !x || !u || !y || !lam_lo || !lam_hi) return TLQR_ERR_ARG;
  if (prob->mem != TLQR_MEM_DEVICE) return TLQR_ERR_ARG;
  const void* dev[] = {prob->Q, prob->q, prob->R, prob->r, prob->A, prob->B, prob->c, u_lo, u_hi, x, u, y,
                       lam_lo, lam_hi};
  for (const void* p : dev) if (!device_ptr(p)) return TLQR_ERR_ARG;
  tlqr_ipm_options o{};
  o.max_iter = 100; o.mu0 = 1.0; o.sigma = 0.1; o.tau = 0.995; o.tol = 1e-9;
  if (opts) {
    if (opts->max_iter > 0) o.max_iter = opts->max_iter;
    if (opts->mu0 > 0) o.mu0 = opts->mu0;
    if (opts->sigma > 0 && opts->sigma < 1) o.sigma = opts->sigma;
    if (opts->tau > 0 && opts->tau < 1) o.tau = opts->tau;
    if (opts->tol > 0) o.tol = opts->tol;
  }
  int32_t dims[3] = {0, 0, 0};                              // N, n, m of the factor object
  if (tlqr_factor_dims(f, dims) || dims[0] != plan->N) return TLQR_ERR_ARG;
  const size_t N = (size_t)dims[0];
  const int n = dims[1], m = dims[2];
  cudaStream_t st = (cudaStream_t)stream;
  // bounded components, counted on the host from the plan (roots carry no control)
  std::vector<unsigned char> edge(N);
  for (size_t j = 0; j < N; ++j) edge[j] = plan->parent[j] >= 0;
  std::vector<double> hlo(N * m), hhi(N * m);
  if (cudaMemcpyAsync(hlo.data(), u_lo, N * m * sizeof(double), cudaMemcpyDeviceToHost, st) ||
      cudaMemcpyAsync(hhi.data(), u_hi, N * m * sizeof(double), cudaMemcpyDeviceToHost, st) ||
      cudaStreamSynchronize(st))
    return TLQR_ERR_CUDA;
  size_t n_ineq = 0;
  for (size_t t = 0; t < N * m; ++t) {
    if (!edge[t / m]) continue;
    if (!(hlo[t] < hhi[t])) return TLQR_ERR_ARG;            // empty box (or NaN)
    n_ineq += std::isfinite(hlo[t]) + std::isfinite(hhi[t]);
  }
  // one workspace allocation for the whole run
  const size_t nm = N * m, nn = N * n;
  int dev_id = 0, sms = 1;
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
  const int threads = 256;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((std::max(nm, nn) + threads - 1) / threads,
                                                                (size_t)sms * 8));
  const size_t doubles = N * m * m + 5 * nm + 2 * nn + 3 + (size_t)blocks;
  unsigned char* ws = nullptr;
  if (cudaMalloc((void**)&ws, doubles * sizeof(double) + N * sizeof(int) + N)) {
    cudaGetLastError();
    return TLQR_ERR_OOM;
  }
  double* d = reinterpret_cast<double*>(ws);
  Ipm a{};
  a.N = (int)N; a.n = n; a.m = m;
  a.R = prob->R; a.r = prob->r; a.lo = u_lo; a.hi = u_hi;
  a.Rt = d; d += N * m * m;
  a.rt = d; d += nm;
  a.xp = d; d += nn;
  a.yp = d; d += nn;
  a.up = d; d += nm;
  a.du = d; d += nm;
  a.dl_lo = d; d += nm;
  a.dl_hi = d; d += nm;
  a.gap = d; d += 1;
  a.alpha_bits = reinterpret_cast<unsigned long long*>(d); d += 1;
  a.gap_part = d; d += blocks;
  a.smax_bits = reinterpret_cast<unsigned long long*>(d); d += 1;
  a.parent = reinterpret_cast<const int*>(d);
  a.edge = reinterpret_cast<unsigned char*>(d) + N * sizeof(int);
  a.x = x; a.u = u; a.y = y; a.l_lo = lam_lo; a.l_hi = lam_hi;
  int rc = TLQR_OK;
  auto fail = [&](int code) { cudaFree(ws); return code; };
  if (cudaMemcpyAsync((void*)a.edge, edge.data(), N, cudaMemcpyHostToDevice, st) ||
      cudaMemcpyAsync((void*)a.parent, plan->parent.data(), N * sizeof(int), cudaMemcpyHostToDevice, st))
    return fail(TLQR_ERR_CUDA);
  k_ipm_init<<<blocks, threads, 0, st>>>(a, o.mu0);
  if (cudaGetLastError()) return fail(TLQR_ERR_CUDA);
  tlqr_problem pt = *prob;
  pt.R = a.Rt;
  pt.r = a.rt;
  tlqr_solution sol{};
  sol.mem = TLQR_MEM_DEVICE;
  sol.x = a.xp; sol.u = a.up; sol.y = a.yp;
  double mu = o.mu0, mean_gap = INFINITY, alpha = 0.0;
  int it = 0, fp64_solves = 0;
  tlqr_info last{};
  // Near the solution the barrier terms S grow like 1 / mu, and a Newton system
  // can become too ill-conditioned for FP32 factors plus refinement; such a
  // system is solved again with an FP64 factor object of the same plan
  // (created once, on first need).
  tlqr_factor_t* f64 = nullptr;
  auto fail64 = [&](int code) { if (f64) tlqr_factor_destroy(f64); return fail(code); };
  bool use64 = false;                        // MIXED: Newton systems now solved in FP64
  bool stopped = false;                      // MIXED without FP64 fallback: a Newton system failed
  const bool mixed = o64_possible(f), allow64 = !(opts && opts->no_fp64_fallback);
  auto make64 = [&]() -> int {
    if (f64) return TLQR_OK;
    tlqr_options o64{};
    if (tlqr_factor_options(f, &o64)) return TLQR_ERR_ARG;
    o64.precision = TLQR_PREC_FP64;
    return tlqr_factor_create(plan, &o64, &f64);
  };
  for (it = 1; it <= o.max_iter; ++it) {
    k_ipm_form<<<blocks, threads, 0, st>>>(a, mu);
    if (cudaGetLastError()) return fail64(TLQR_ERR_CUDA);
    if (use64) {
      if ((rc = make64())) return fail64(rc);
      rc = tlqr_solve(f64, &pt, &sol, stream);
      last = tlqr_info{};
      ++fp64_solves;
    } else {
      rc = tlqr_solve(f, &pt, &sol, stream);
      tlqr_last_info(f, &last);
    }
    const bool precision_failure =
        rc == TLQR_ERR_NO_CONVERGENCE || rc == TLQR_ERR_NOT_PD || rc == TLQR_ERR_NONFINITE || rc == TLQR_ERR_SINGULAR;
    if (rc == TLQR_ERR_NO_CONVERGENCE && opts && opts->no_fp64_fallback) {
      rc = TLQR_OK;                           // inexact Newton step at the accuracy refinement reached
    } else if (precision_failure && !use64 && mixed && !allow64) {
      // the FP32 factors cannot take this Newton system (the barrier terms have outgrown
      // them) and no FP64 factor may be allocated: stop at the current iterate, which the
      // failed step has not touched; the call returns TLQR_ERR_NO_CONVERGENCE
      stopped = true;
      break;
    } else if (precision_failure && !use64 && mixed && allow64) {
      if ((rc = make64())) return fail64(rc);
      rc = tlqr_solve(f64, &pt, &sol, stream);
      last = tlqr_info{};
      ++fp64_solves;
      use64 = true;
    }
    if (rc) return fail64(rc);
    k_ipm_step<<<blocks, threads, 0, st>>>(a, mu, o.tau);
    k_ipm_update<<<blocks, threads, 0, st>>>(a);
    k_ipm_gap<<<1, 32, 0, st>>>(a, blocks);
    if (cudaGetLastError()) return fail64(TLQR_ERR_CUDA);
    double h[2] = {0, 0};
    unsigned long long ab = 0, sb = 0;
    if (cudaMemcpyAsync(&ab, a.alpha_bits, sizeof(ab), cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(&sb, a.smax_bits, sizeof(sb), cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(h, a.gap, sizeof(double), cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
      return fail64(TLQR_ERR_CUDA);
    std::memcpy(&alpha, &ab, sizeof(alpha));
    double smax = 0.0;
    std::memcpy(&smax, &sb, sizeof(smax));
    // FP32 factors stop resolving the Newton step on the active bounds once the
    // barrier terms l / s reach ~1e6 (measured: the step length then collapses
    // although each solve still meets its normwise tolerance); from there on
    // the Newton systems are solved in FP64
    if (mixed && allow64 && smax > kIpmSwitch) use64 = true;
    mean_gap = n_ineq ? h[0] / (double)n_ineq : 0.0;
    if (!std::isfinite(mean_gap)) return fail64(TLQR_ERR_NONFINITE);
    // stop after a full Newton step: the linear KKT rows then hold to solve accuracy
    if (mean_gap <= o.tol && alpha >= 1.0) break;
    mu = o.sigma * mean_gap;
  }
  const bool converged = !stopped && mean_gap <= o.tol && alpha >= 1.0;
  if (converged) {
    k_ipm_duals<<<blocks, threads, 0, st>>>(a, prob->M, prob->B);
    if (cudaGetLastError() || cudaStreamSynchronize(st)) return fail64(TLQR_ERR_CUDA);
  }
  if (info) {
    info->iterations = std::min(stopped ? it - 1 : it, o.max_iter);
    info->mu = mu;
    info->mean_gap = mean_gap;
    info->last_alpha = alpha;
    info->last_eta = last.eta;
    info->fp64_solves = fp64_solves;
  }
  if (f64) tlqr_factor_destroy(f64);
  cudaFree(ws);
  return converged ? TLQR_OK : TLQR_ERR_NO_CONVERGENCE;
}
