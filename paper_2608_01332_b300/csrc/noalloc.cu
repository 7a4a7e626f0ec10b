// Allocation-free variant of the FP64 KKT residual (tlqr_kkt_residual_noalloc).
//
// Who needs it: code that must not allocate device memory once it is running,
// for example a receding-horizon controller that re-checks its Newton step
// every few milliseconds (cudaMalloc/cudaFree may synchronise the device and
// take an unbounded time, which a hard control deadline cannot absorb), or a
// process whose device memory is handed out entirely by another framework's
// caching allocator.  Those callers cannot create a tlqr_factor_t (which owns
// cudaMalloc'd workspace) just to measure the residual of a candidate
// solution.
//
// How: the residual kernel's scratch -- the tree's parent and child lists, the
// three residual vectors and the four running maxima -- lives in one
// file-scope device array of fixed size, shared by every call on a GPU.  The
// kernel itself is the library's residual kernel, compiled into this file with
// internal linkage.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/tlqr.h"
#include "plan.hpp"

namespace {
#include "residual.cuh"
}  // namespace

namespace {

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TLQR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};   // device address of the array, per device

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

struct Layout {
  size_t maxes, parent, child_start, child_list, res_x, res_u, res_c, total;
};

Layout layout(size_t N, size_t n, size_t m) {
  Layout L;
  size_t o = 0;
  L.maxes = o;       o = up256(o + 4 * sizeof(unsigned long long));
  L.parent = o;      o = up256(o + N * sizeof(int32_t));
  L.child_start = o; o = up256(o + (N + 1) * sizeof(int32_t));
  L.child_list = o;  o = up256(o + std::max<size_t>(1, N - 1) * sizeof(int32_t));
  L.res_x = o;       o = up256(o + N * n * sizeof(double));
  L.res_u = o;       o = up256(o + N * m * sizeof(double));
  L.res_c = o;       o = up256(o + N * n * sizeof(double));
  L.total = o;
  return L;
}

// Device address of the scratch array on the current device.  The first call
// on a device resolves it (with that device current); later calls reuse it.
int scratch_on_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TLQR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return TLQR_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TLQR_OK;
}

}  // namespace

extern "C" int tlqr_kkt_residual_noalloc(const tlqr_plan_t* plan, int32_t n, int32_t m, const tlqr_problem* prob,
                                         const double* x, const double* u, const double* y, double* stats,
                                         void* stream) {
  if (!plan || !prob || !x || !u || !y || !stats) return TLQR_ERR_ARG;
  if (n < 1 || m < 1 || n > TLQR_MAX_DIM || m > TLQR_MAX_DIM) return TLQR_ERR_ARG;
  if (prob->mem != TLQR_MEM_DEVICE) return TLQR_ERR_ARG;          // host data would need staging memory
  if (!prob->Q || !prob->q || !prob->R || !prob->r || !prob->A || !prob->B || !prob->c) return TLQR_ERR_ARG;
  const size_t N = (size_t)plan->N;
  const Layout L = layout(N, (size_t)n, (size_t)m);
  if (L.total > (size_t)TLQR_NOALLOC_SCRATCH_BYTES) return TLQR_ERR_ARG;   // tree too large for the scratch
  unsigned char* base = nullptr;
  int rc = scratch_on_current_device(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* d_parent = reinterpret_cast<int32_t*>(base + L.parent);
  int32_t* d_cs = reinterpret_cast<int32_t*>(base + L.child_start);
  int32_t* d_cl = reinterpret_cast<int32_t*>(base + L.child_list);
  unsigned long long* d_maxes = reinterpret_cast<unsigned long long*>(base + L.maxes);
  cudaError_t e = cudaMemcpyAsync(d_parent, plan->parent.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(d_cs, plan->child_start.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (!e && N > 1)
    e = cudaMemcpyAsync(d_cl, plan->child_list.data(), (N - 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  // the maxima are accumulated with atomicMax and must start at zero on every call
  if (!e) e = cudaMemsetAsync(d_maxes, 0, 4 * sizeof(unsigned long long), st);
  if (e) return TLQR_ERR_CUDA;
  tlqr::ResidualArgs a{};
  a.N = (int)N; a.n = n; a.m = m; a.with_knorm = 1;
  a.parent = d_parent; a.child_start = d_cs; a.child_list = d_cl;
  a.Q = prob->Q; a.q = prob->q; a.M = prob->M; a.R = prob->R; a.r = prob->r; a.A = prob->A; a.B = prob->B;
  a.c = prob->c; a.Delta = prob->Delta;
  a.x = x; a.u = u; a.y = y;
  a.res_x = reinterpret_cast<double*>(base + L.res_x);
  a.res_u = reinterpret_cast<double*>(base + L.res_u);
  a.res_c = reinterpret_cast<double*>(base + L.res_c);
  a.maxes = d_maxes;
  const size_t rows = N * (2 * (size_t)n + (size_t)m);
  const int threads = 256;
  const int blocks = (int)std::min<size_t>((rows + threads - 1) / threads, 148 * 8);
  tlqr::k_residual<<<blocks, threads, 0, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) return TLQR_ERR_CUDA;
  unsigned long long hm[4] = {0, 0, 0, 0};
  e = cudaMemcpyAsync(hm, d_maxes, sizeof(hm), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return TLQR_ERR_CUDA;
  double v[4];
  for (int t = 0; t < 4; ++t) std::memcpy(&v[t], &hm[t], sizeof(double));
  const double den = v[3] * v[1] + v[2];
  stats[0] = v[0];
  stats[1] = !std::isfinite(v[0]) ? INFINITY : (den > 0 ? v[0] / den : v[0]);
  return TLQR_OK;
}
