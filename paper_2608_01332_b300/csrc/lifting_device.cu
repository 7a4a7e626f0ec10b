// Node-control lifting and projection of Prop. 2 (Sec. III-B) on the device.
//
// The same map as the host version (lifting.cpp): node i keeps a predecision
// copy i- (label i) with state cost diag(Q_i, 0), q = (q_i, 0), c = (c_i, 0),
// Delta = diag(Delta_i, 0); the uncertainty edge parent(i)+ -> i- gets
// A = [[A_i, B_i], [0, 0]], B = 0 and a dummy control of cost R = I, r = 0
// (eq. (uncertainty-edge)); every nonterminal i gets a decision copy i+
// (labels N, N+1, ... in increasing i) reached through the decision edge
// eq. (decision-edge): A = [[I, 0], [0, 0]], B = [[0], [I]], M = [M_i; 0],
// R = R_i, r = r_i, zero node data.  The topology (parent, lifted parent, map)
// is computed on the host, where plans are built; every lifted data block is
// written once by a device kernel, so the node-form data never leave the GPU.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/tlqr.h"

namespace {

struct LiftArgs {
  int N, L, n, m;
  const int* parent;      // [N]
  const int* owner;       // [L - N]: node i of decision copy N + t
  const double *Q, *q, *Mv, *Rv, *rv, *Av, *Bv, *c, *Delta;
  double *lQ, *lq, *lM, *lR, *lr, *lA, *lB, *lc, *lDelta;
};

// One block per lifted node (grid-stride); threads over the entries of its blocks.
__global__ void k_lift(LiftArgs a) {
  const int n = a.n, m = a.m, s = n + m;
  const size_t ss = (size_t)s * s, sm = (size_t)s * m, nn = (size_t)n * n, nm = (size_t)n * m, mm = (size_t)m * m;
  for (int l = blockIdx.x; l < a.L; l += gridDim.x) {
    const bool pre = l < a.N;
    const int i = pre ? l : a.owner[l - a.N];
    const bool has_edge = pre ? a.parent[i] >= 0 : true;
    for (int e = threadIdx.x; e < (int)ss; e += blockDim.x) {
      const int r = e / s, col = e - (e / s) * s;
      double vQ = 0, vD = 0, vA = 0;
      if (pre) {
        if (r < n && col < n) {
          vQ = a.Q[i * nn + r * n + col];
          if (a.Delta) vD = a.Delta[i * nn + r * n + col];
        }
        if (has_edge && r < n) vA = col < n ? a.Av[i * nn + r * n + col] : a.Bv[i * nm + r * m + (col - n)];
      } else if (r < n && col == r) {
        vA = 1.0;
      }
      a.lQ[l * ss + e] = vQ;
      a.lDelta[l * ss + e] = vD;
      a.lA[l * ss + e] = vA;
    }
    for (int e = threadIdx.x; e < (int)sm; e += blockDim.x) {
      const int r = e / m, col = e - (e / m) * m;
      double vM = 0, vB = 0;
      if (!pre) {
        if (r < n) vM = a.Mv[i * nm + r * m + col];
        else if (r - n == col) vB = 1.0;
      }
      a.lM[l * sm + e] = vM;
      a.lB[l * sm + e] = vB;
    }
    for (int e = threadIdx.x; e < (int)mm; e += blockDim.x) {
      const int r = e / m, col = e - (e / m) * m;
      a.lR[l * mm + e] = pre ? ((has_edge && r == col) ? 1.0 : 0.0) : a.Rv[i * mm + e];
    }
    for (int e = threadIdx.x; e < m; e += blockDim.x) a.lr[(size_t)l * m + e] = pre ? 0.0 : a.rv[(size_t)i * m + e];
    for (int e = threadIdx.x; e < s; e += blockDim.x) {
      a.lq[(size_t)l * s + e] = (pre && e < n) ? a.q[(size_t)i * n + e] : 0.0;
      a.lc[(size_t)l * s + e] = (pre && e < n) ? a.c[(size_t)i * n + e] : 0.0;
    }
  }
}

__global__ void k_project(int N, int n, int m, const int* map, const double* lx, const double* lu, const double* ly,
                          double* x, double* v, double* y) {
  const int s = n + m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int im = map[i], ip = map[N + i];
    for (int e = 0; e < n; ++e) {
      x[(size_t)i * n + e] = lx[(size_t)im * s + e];
      y[(size_t)i * n + e] = ly[(size_t)im * s + e];
    }
    for (int e = 0; e < m; ++e) v[(size_t)i * m + e] = ip >= 0 ? lu[(size_t)ip * m + e] : 0.0;
  }
}

bool is_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int tlqr_lift_node_controls_device(const int32_t* parent, int32_t N, int32_t n, int32_t m,
                                              const double* Q, const double* q, const double* Mv,
                                              const double* Rv, const double* rv, const double* Av,
                                              const double* Bv, const double* c, const double* Delta,
                                              int32_t* Nl, int32_t* lifted_parent, double* lQ, double* lq,
                                              double* lM, double* lR, double* lr, double* lA, double* lB,
                                              double* lc, double* lDelta, int32_t* map, void* stream) {
  if (!parent || N < 1 || n < 1 || m < 1 || n > TLQR_MAX_DIM || m > TLQR_MAX_DIM || !Nl) return TLQR_ERR_ARG;
  // topology and sizes on the host (also validates parent[])
  int rc = tlqr_lift_node_controls(parent, N, n, m, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                   nullptr, nullptr, Nl, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                   nullptr, nullptr, nullptr, nullptr, nullptr);
  if (rc || !lifted_parent) return rc;
  const double* ins[] = {Q, q, Mv, Rv, rv, Av, Bv, c};
  double* outs[] = {lQ, lq, lM, lR, lr, lA, lB, lc, lDelta};
  for (const double* p : ins) if (!is_device(p)) return TLQR_ERR_ARG;
  for (double* p : outs) if (!is_device(p)) return TLQR_ERR_ARG;
  if (Delta && !is_device(Delta)) return TLQR_ERR_ARG;
  if (!map) return TLQR_ERR_ARG;
  const int L = *Nl;
  std::vector<char> nonterm(N, 0);
  for (int j = 0; j < N; ++j) if (parent[j] >= 0) nonterm[parent[j]] = 1;
  std::vector<int32_t> owner;
  std::vector<int32_t> plus(N, -1);
  for (int i = 0, t = N; i < N; ++i)
    if (nonterm[i]) { plus[i] = t++; owner.push_back(i); }
  for (int i = 0; i < N; ++i) {
    map[i] = i;
    map[N + i] = plus[i];
    lifted_parent[i] = parent[i] >= 0 ? plus[parent[i]] : -1;
    if (plus[i] >= 0) lifted_parent[plus[i]] = i;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* d_idx = nullptr;
  const size_t ni = (size_t)N + owner.size();
  if (cudaMallocAsync((void**)&d_idx, std::max<size_t>(1, ni) * sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return TLQR_ERR_OOM;
  }
  cudaError_t e = cudaMemcpyAsync(d_idx, parent, N * sizeof(int), cudaMemcpyHostToDevice, st);
  if (!e && !owner.empty())
    e = cudaMemcpyAsync(d_idx + N, owner.data(), owner.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  LiftArgs a{N, L, n, m, d_idx, d_idx + N, Q, q, Mv, Rv, rv, Av, Bv, c, Delta,
             lQ, lq, lM, lR, lr, lA, lB, lc, lDelta};
  if (!e) {
    const int blocks = std::min(L, 65535);
    k_lift<<<blocks, 128, 0, st>>>(a);
    e = cudaGetLastError();
  }
  // the host vectors above must stay alive until the copies have read them
  if (!e) e = cudaStreamSynchronize(st);
  cudaFreeAsync(d_idx, st);
  return e ? TLQR_ERR_CUDA : TLQR_OK;
}

extern "C" int tlqr_project_lifted_device(int32_t N, int32_t n, int32_t m, const int32_t* map, const double* lx,
                                          const double* lu, const double* ly, double* x, double* v, double* y,
                                          void* stream) {
  if (N < 1 || n < 1 || m < 1 || !map) return TLQR_ERR_ARG;
  const double* ins[] = {lx, lu, ly};
  double* outs[] = {x, v, y};
  for (const double* p : ins) if (!is_device(p)) return TLQR_ERR_ARG;
  for (double* p : outs) if (!is_device(p)) return TLQR_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* d_map = nullptr;
  if (cudaMallocAsync((void**)&d_map, 2 * (size_t)N * sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return TLQR_ERR_OOM;
  }
  cudaError_t e = cudaMemcpyAsync(d_map, map, 2 * (size_t)N * sizeof(int), cudaMemcpyHostToDevice, st);
  if (!e) {
    const int blocks = (int)std::min<long long>(((long long)N + 255) / 256, 65535);
    k_project<<<blocks, 256, 0, st>>>(N, n, m, d_map, lx, lu, ly, x, v, y);
    e = cudaGetLastError();
  }
  if (!e) e = cudaStreamSynchronize(st);
  cudaFreeAsync(d_map, st);
  return e ? TLQR_ERR_CUDA : TLQR_OK;
}
