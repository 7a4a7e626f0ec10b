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
// How: the residual kernel's scratch -- the tree's parent and child lists,
// the tree ordinal of every node of a forest, the three residual vectors, the
// four running maxima per tree and the two reduced statistics -- lives in one
// file-scope device array of fixed size, shared by every call on a GPU.  The
// kernels are the library's residual kernels, compiled into this file with
// internal linkage, and a one-block reduction of the per-tree maxima.
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
  size_t out, maxes, parent, child_start, child_list, tree, res_x, res_u, res_c, total;
};

// T = number of trees of the plan (a forest keeps four maxima per tree and the
// tree ordinal of every node).
Layout layout(size_t N, size_t n, size_t m, size_t T) {
  Layout L;
  size_t o = 0;
  L.out = o;         o = up256(o + 2 * sizeof(double));
  L.maxes = o;       o = up256(o + 4 * T * sizeof(unsigned long long));
  L.parent = o;      o = up256(o + N * sizeof(int32_t));
  L.child_start = o; o = up256(o + (N + 1) * sizeof(int32_t));
  L.child_list = o;  o = up256(o + std::max<size_t>(1, N - 1) * sizeof(int32_t));
  L.tree = o;        o = up256(o + (T > 1 ? N : 1) * sizeof(int32_t));
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

// True when the GPU can dereference p as device memory (device or managed
// allocations).  A host pointer -- pageable, pinned or unknown to CUDA -- is
// refused: handing one to the residual kernel would make it read host
// addresses as device addresses.  Nothing is allocated.
bool device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Per tree t: eta_t = r_t / (K_t z_t + b_t) from the slot-major maxima
// [4][T] (r, z, b, K); out[0] = max_t r_t, out[1] = max_t eta_t (+Inf when a
// residual is not finite) -- the same reduction the factor object applies to
// its own per-tree maxima.  One block.
__global__ void k_tree_eta_max(const unsigned long long* maxes, int T, double* out) {
  __shared__ unsigned long long red[2][32];
  unsigned long long ra = 0, re = 0;
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const double r = __longlong_as_double((long long)maxes[t]);
    const double z = __longlong_as_double((long long)maxes[(size_t)T + t]);
    const double b = __longlong_as_double((long long)maxes[2 * (size_t)T + t]);
    const double k = __longlong_as_double((long long)maxes[3 * (size_t)T + t]);
    const double den = k * z + b;
    double eta = den > 0 ? r / den : r;
    if (!isfinite(r)) eta = INFINITY;
    const unsigned long long a_bits = (unsigned long long)__double_as_longlong(r);
    const unsigned long long e_bits = (unsigned long long)__double_as_longlong(eta);
    ra = a_bits > ra ? a_bits : ra;
    re = e_bits > re ? e_bits : re;
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const unsigned long long oa = __shfl_xor_sync(0xffffffffu, ra, off);
    const unsigned long long oe = __shfl_xor_sync(0xffffffffu, re, off);
    ra = oa > ra ? oa : ra;
    re = oe > re ? oe : re;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) { red[0][warp] = ra; red[1][warp] = re; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      ra = red[0][w] > ra ? red[0][w] : ra;
      re = red[1][w] > re ? red[1][w] : re;
    }
    out[0] = __longlong_as_double((long long)ra);
    out[1] = __longlong_as_double((long long)re);
  }
}

}  // namespace

extern "C" int tlqr_kkt_residual_noalloc(const tlqr_plan_t* plan, int32_t n, int32_t m, const tlqr_problem* prob,
                                         const double* x, const double* u, const double* y, double* stats,
                                         void* stream) {
  if (!plan || !prob || !x || !u || !y || !stats) return TLQR_ERR_ARG;
  if (n < 1 || m < 1 || n > TLQR_MAX_DIM || m > TLQR_MAX_DIM) return TLQR_ERR_ARG;
  if (prob->mem != TLQR_MEM_DEVICE) return TLQR_ERR_ARG;          // host data would need staging memory
  if (!prob->Q || !prob->q || !prob->R || !prob->r || !prob->A || !prob->B || !prob->c) return TLQR_ERR_ARG;
  const size_t N = (size_t)plan->N, T = (size_t)std::max<int32_t>(1, plan->n_trees);
  const Layout L = layout(N, (size_t)n, (size_t)m, T);
  if (L.total > (size_t)TLQR_NOALLOC_SCRATCH_BYTES) return TLQR_ERR_ARG;   // tree too large for the scratch
  // every array must be device memory, whatever prob->mem claims
  const void* arrays[] = {prob->Q, prob->q, prob->R, prob->r, prob->A, prob->B, prob->c, x, u, y};
  for (const void* a : arrays)
    if (!device_pointer(a)) return TLQR_ERR_ARG;
  if ((prob->M && !device_pointer(prob->M)) || (prob->Delta && !device_pointer(prob->Delta))) return TLQR_ERR_ARG;
  unsigned char* base = nullptr;
  int rc = scratch_on_current_device(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* d_parent = reinterpret_cast<int32_t*>(base + L.parent);
  int32_t* d_cs = reinterpret_cast<int32_t*>(base + L.child_start);
  int32_t* d_cl = reinterpret_cast<int32_t*>(base + L.child_list);
  int32_t* d_tree = reinterpret_cast<int32_t*>(base + L.tree);
  unsigned long long* d_maxes = reinterpret_cast<unsigned long long*>(base + L.maxes);
  double* d_out = reinterpret_cast<double*>(base + L.out);
  cudaError_t e = cudaMemcpyAsync(d_parent, plan->parent.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(d_cs, plan->child_start.data(), (N + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (!e && N > 1)
    e = cudaMemcpyAsync(d_cl, plan->child_list.data(), (N - 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (!e && T > 1)
    e = cudaMemcpyAsync(d_tree, plan->tree_of.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  // the maxima are accumulated with atomicMax and must start at zero on every call
  if (!e) e = cudaMemsetAsync(d_maxes, 0, 4 * T * sizeof(unsigned long long), st);
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
  a.T = (int)T;
  a.tree = T > 1 ? d_tree : nullptr;
  int sms = 0;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) || sms < 1)
      return TLQR_ERR_CUDA;
  }
  const size_t rows = N * (2 * (size_t)n + (size_t)m);
  const int threads = 256;
  const int blocks = (int)std::min<size_t>((rows + threads - 1) / threads, (size_t)sms * 8);
  if (T > 1) tlqr::k_residual_trees<<<blocks, threads, 0, st>>>(a);
  else tlqr::k_residual<<<blocks, threads, 0, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) return TLQR_ERR_CUDA;
  k_tree_eta_max<<<1, 256, 0, st>>>(d_maxes, (int)T, d_out);
  if (cudaGetLastError() != cudaSuccess) return TLQR_ERR_CUDA;
  double v[2] = {0.0, 0.0};
  e = cudaMemcpyAsync(v, d_out, sizeof(v), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return TLQR_ERR_CUDA;
  stats[0] = v[0];
  stats[1] = v[1];
  return TLQR_OK;
}
