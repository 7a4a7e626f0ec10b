// Kernels of the rake-compress factorisation and solve (Alg. 1, steps 2-6).
//
// Execution model: the host walks the plan's structural rounds and launches,
// per round, one kernel per operation kind; inside a kernel one warp performs
// one local operation (a rake, a sibling sum, a compression, a reconstruction,
// a local factor, a vector update) on n x n blocks staged in shared memory.
// Operations of one launch touch disjoint output slots (the plan guarantees a
// unique writer per slot per round), so no atomics are needed and results are
// independent of scheduling.
//
// Storage, all [N][..] blocks indexed by node (edge data by the child node):
//   U   node data U_i (eq. (initial-node-data)); after the reverse pass it holds
//       P_i (a raked node keeps U_j = P_j; a compressed one is overwritten by
//       eq. (value-reconstruction); the root keeps P_rho = U_rho).
//   Ea, Ec, Ep  current edge triple (A, C, P) of the edge entering the slot.
//       When centre j is compressed, slot j receives its tape
//       s_j = (A_r, C_r, P~_r) (eq. (quadratic-compress)) and slot k (the
//       child) the composed triple.
//   contrib  rake contributions m_{i<-j} (eq. (quadratic-rake)), by rake index.
//   K, Tm, W, Finv, LG  local factors (eq. (FW), (factor-local)); Tm is
//       overwritten by the composed transition matrices of eq. (transition-compose),
//       Tr keeps the outgoing map T_r of every compressed centre.
#pragma once
#include <cstdint>

#include "smallmat.cuh"

namespace tlqr {

enum : int { ST_OK = 0, ST_NOT_PD = 3, ST_SINGULAR = 4, ST_NONFINITE = 5, ST_TIMEOUT = 7 };

template <typename T>
struct Ws {
  int N, n, m;
  int has_M, has_delta;
  // problem data (FP64, device)
  const double *Q, *M, *R, *A, *B, *Delta;
  const double *q, *r, *c;
  // plan (device)
  const int *rake_leaf, *rake_parent, *seg_parent, *seg_start;
  const int *comp_j, *comp_i, *comp_k;
  const int *parent, *child_start, *child_list;
  // factor workspace
  T *U, *Ea, *Ec, *Ep, *contrib;
  T *K, *Tm, *Tr, *W, *Finv, *LG;
  unsigned char* dflag;   // per node: Delta_i has a nonzero entry
  // FP64 re-solves of ill-conditioned eliminations (FP32 compile-time-n
  // kernels): a ticket counter, the number of slots and the slots (slot
  // doubles each); redo_count == nullptr disables them
  int* redo_count;
  int redo_cap;
  double* redo_scratch;
  size_t redo_slot;
  // solve workspace
  T *h, *z, *s, *cv, *bv, *kv, *xs;
  int* status;
  // panel solves: nrhs right-hand sides at once; every vector above (and q, r,
  // c) is [nrhs][..] with these strides between right-hand sides
  int nrhs;
  size_t sv, sm, scv;          // n-vectors (N n), m-vectors (N m), rake contributions (rakes n)
  // the same workspace seen from right-hand side k of the panel
  __host__ __device__ Ws rhs(int k) const {
    Ws v = *this;
    if (k) {
      const size_t ov = (size_t)k * sv, om = (size_t)k * sm, oc = (size_t)k * scv;
      v.q = q + ov; v.c = c + ov; v.r = r + om;
      v.h = h + ov; v.z = z + ov; v.s = s + ov; v.bv = bv + ov; v.xs = xs + ov;
      v.kv = kv + om; v.cv = cv + oc;
    }
    return v;
  }
};

// A node is a root (of its tree in a forest) when its parent is -1.  Batched
// primitive calls have no tree (parent == nullptr) and no roots.
template <typename T>
__device__ __forceinline__ bool node_is_root(const Ws<T>& w, int j) { return w.parent ? (w.parent[j] < 0) : false; }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may be scheduled while its predecessor in the stream is still
// draining.  Every kernel of the factorisation and solve passes starts here:
// it waits until the predecessor grid has completed and its writes are
// visible, then allows its own successor to begin launching.  Without a
// programmatic predecessor both instructions return at once.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

__device__ __forceinline__ void set_status(int* status, int code) {
  if (lane_id() == 0) atomicCAS(status, 0, code);
}

// Per-warp shared-memory carve-out.
template <typename T>
__device__ __forceinline__ T* warp_smem(int warp_bytes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  return reinterpret_cast<T*>(smem_raw + (threadIdx.x >> 5) * warp_bytes);
}
__device__ __forceinline__ int warp_op() { return blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); }

// ---------------------------------------------------------------- tau
// Rake fold eq. (terminal-fold): out = P + A^T U (I + C U)^{-1} A.
// sm: 5 n^2 T + n ints.  U, A, C, P may be global (any type S); out global T.
template <typename T, typename S>
__device__ bool tau_warp(int n, const S* Ug, const S* Ag, const S* Cg, const S* Pg, T* out, T* sm) {
  const int nn = n * n;
  T *sU = sm, *sX = sm + nn, *sA = sm + 2 * nn, *sY = sm + 3 * nn, *sZ = sm + 4 * nn;
  int* piv = reinterpret_cast<int*>(sm + 5 * nn);
  wload(sU, Ug, nn);
  wload(sZ, Cg, nn);
  wload(sA, Ag, nn);
  wload(sY, Ag, nn);
  __syncwarp();
  wgemm<T, false, false>(n, n, n, sZ, n, sU, n, sX, n, T(1), (const T*)nullptr, 0);   // X = C U
  wadd_identity(sX, n, n);
  __syncwarp();
  if (!wlu(sX, n, n, piv)) return false;
  wlu_solve(sX, n, n, piv, sY, n, n);                                                   // Y = X^{-1} A
  wgemm<T, false, false>(n, n, n, sU, n, sY, n, sZ, n, T(1), (const T*)nullptr, 0);    // Z = U Y
  wgemm<T, true, false>(n, n, n, sA, n, sZ, n, out, n, T(1), Pg, n);                   // P + A^T Z
  return true;
}

// ---------------------------------------------------------------- condensation
// eq. (edge-components); also U_i <- Q_i (eq. (initial-node-data)) and the
// per-node "Delta nonzero" flag.  sm: 2 n^2 + m^2 + 2 n m T.
template <typename T>
__global__ void k_condense(Ws<T> w, int warp_bytes) {
  pdl_entry();
  const int i = warp_op();
  if (i >= w.N) return;
  const int n = w.n, m = w.m, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  wload(w.U + (size_t)i * nn, w.Q + (size_t)i * nn, nn);
  bool dnz = false;
  if (w.has_delta) {
    const double* D = w.Delta + (size_t)i * nn;
    for (int e = lane_id(); e < nn; e += 32) dnz |= (D[e] != 0.0);
    dnz = wany(dnz);
    if (lane_id() == 0) w.dflag[i] = dnz ? 1 : 0;
  }
  if (node_is_root(w, i)) return;
  T *sR = sm, *sX = sm + m * m, *sB = sX + 2 * n * m, *sM = sB + n * m;
  double* scratch = reinterpret_cast<double*>(
      reinterpret_cast<unsigned char*>(sm) + ((sizeof(T) * (m * m + 4 * n * m) + 15) / 16) * 16);
  const int nr = w.has_M ? 2 * n : n;    // X = R^{-1} [B^T | M^T]  (m x nr)
  wload(sR, w.R + (size_t)i * m * m, m * m);
  const double* Bg = w.B + (size_t)i * n * m;
  wload(sB, Bg, n * m);
  for (int e = lane_id(); e < n * m; e += 32) {
    const int a = e / m, b = e - (e / m) * m;   // B[a][b]
    sX[b * nr + a] = (T)Bg[e];
  }
  if (w.has_M) {
    const double* Mg = w.M + (size_t)i * n * m;
    wload(sM, Mg, n * m);
    for (int e = lane_id(); e < n * m; e += 32) {
      const int a = e / m, b = e - (e / m) * m;
      sX[b * nr + n + a] = (T)Mg[e];
    }
  }
  __syncwarp();
  if (!wchol_checked(sR, m, m, w.R + (size_t)i * m * m, (const T*)nullptr, 0, scratch)) {
    set_status(w.status, ST_NOT_PD);
    return;
  }
  wchol_solve(sR, m, m, sX, nr, nr);
  T* Ec = w.Ec + (size_t)i * nn;
  const double* Dg = (w.has_delta && dnz) ? w.Delta + (size_t)i * nn : nullptr;
  wgemm<T, false, false>(n, n, m, sB, m, sX, nr, Ec, n, T(1), Dg, n);             // C = Delta + B R^{-1} B^T
  if (w.has_M) {
    wgemm<T, false, false>(n, n, m, sB, m, sX + n, nr, w.Ea + (size_t)i * nn, n, T(-1), w.A + (size_t)i * nn, n);
    wgemm<T, false, false>(n, n, m, sM, m, sX + n, nr, w.Ep + (size_t)i * nn, n, T(-1), (const T*)nullptr, 0);
  } else {
    wload(w.Ea + (size_t)i * nn, w.A + (size_t)i * nn, nn);
    wzero(w.Ep + (size_t)i * nn, nn);
  }
}

// ---------------------------------------------------------------- rake
template <typename T>
__global__ void k_rake(Ws<T> w, int begin, int count, int warp_bytes) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int r = begin + t, j = w.rake_leaf[r], nn = w.n * w.n;
  T* sm = warp_smem<T>(warp_bytes);
  const size_t o = (size_t)j * nn;
  if (!tau_warp(w.n, w.U + o, w.Ea + o, w.Ec + o, w.Ep + o, w.contrib + (size_t)r * nn, sm))
    set_status(w.status, ST_SINGULAR);
}

// Ordered sibling sum + absorption: U_i += sum of the segment's contributions,
// in increasing leaf index (Sec. X-B, oplus = addition).
template <typename T>
__global__ void k_absorb(Ws<T> w, int seg_begin, int count) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int s = seg_begin + t, i = w.seg_parent[s], nn = w.n * w.n;
  const int b = w.seg_start[s], e = w.seg_start[s + 1];
  T* Ui = w.U + (size_t)i * nn;
  for (int x = lane_id(); x < nn; x += 32) {
    T acc = w.contrib[(size_t)b * nn + x];
    for (int r = b + 1; r < e; ++r) acc += w.contrib[(size_t)r * nn + x];
    Ui[x] += acc;
  }
}

// ---------------------------------------------------------------- compress
// eq. (compress-intermediates)-(composition), tape eq. (quadratic-compress).
// sm: 7 n^2 T + n ints.
template <typename T>
__global__ void k_compress(Ws<T> w, int begin, int count, int warp_bytes) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int r = begin + t, j = w.comp_j[r], k = w.comp_k[r];
  const int n = w.n, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  T *sPt = sm, *sS = sm + nn, *sAl = sm + 2 * nn, *sAr = sm + 3 * nn, *sY = sm + 4 * nn,
    *sTmp = sm + 6 * nn;
  int* piv = reinterpret_cast<int*>(sm + 7 * nn);
  const size_t oj = (size_t)j * nn, ok = (size_t)k * nn;
  wadd(sPt, w.Ep + ok, w.U + oj, nn);                 // P~ = P_r + U_j
  wload(sAl, w.Ea + oj, nn);
  wload(sAr, w.Ea + ok, nn);
  wload(sTmp, w.Ec + oj, nn);                         // C_l
  for (int e = lane_id(); e < nn; e += 32) {          // Y[:, 0:n] = A_l
    const int a = e / n, b = e - (e / n) * n;
    sY[a * 2 * n + b] = w.Ea[oj + e];
  }
  __syncwarp();
  wgemm<T, false, false>(n, n, n, sTmp, n, sPt, n, sS, n, T(1), (const T*)nullptr, 0);   // C_l P~
  wadd_identity(sS, n, n);
  wgemm<T, false, true>(n, n, n, sTmp, n, sAr, n, sY + n, 2 * n, T(1), (const T*)nullptr, 0);  // C_l A_r^T
  if (!wlu(sS, n, n, piv)) { set_status(w.status, ST_SINGULAR); return; }
  wlu_solve(sS, n, n, piv, sY, 2 * n, 2 * n);         // [Y1 | Y2] = S^{-1} [A_l | C_l A_r^T]
  // P_new = P_l + A_l^T (P~ Y1)  -> sS
  wgemm<T, false, false>(n, n, n, sPt, n, sY, 2 * n, sTmp, n, T(1), (const T*)nullptr, 0);
  wgemm<T, true, false>(n, n, n, sAl, n, sTmp, n, sS, n, T(1), w.Ep + oj, n);
  // A_new = A_r Y1 -> sTmp ; C_new = C_r + A_r Y2 -> sAl
  wgemm<T, false, false>(n, n, n, sAr, n, sY, 2 * n, sTmp, n, T(1), (const T*)nullptr, 0);
  wgemm<T, false, false>(n, n, n, sAr, n, sY + n, 2 * n, sAl, n, T(1), w.Ec + ok, n);
  // tape into slot j: (A_r, C_r, P~)
  for (int e = lane_id(); e < nn; e += 32) {
    w.Ea[oj + e] = sAr[e];
    w.Ec[oj + e] = w.Ec[ok + e];
    w.Ep[oj + e] = sPt[e];
  }
  __syncwarp();
  // composed edge into slot k
  for (int e = lane_id(); e < nn; e += 32) {
    w.Ea[ok + e] = sTmp[e];
    w.Ec[ok + e] = sAl[e];
    w.Ep[ok + e] = sS[e];
  }
}

// Reverse reconstruction at a compressed centre, eq. (quadratic-expand-compress):
// P_j = tau(s_j, P_k), written over U_j.
template <typename T>
__global__ void k_expand(Ws<T> w, int begin, int count, int warp_bytes) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int r = begin + t, j = w.comp_j[r], k = w.comp_k[r], nn = w.n * w.n;
  T* sm = warp_smem<T>(warp_bytes);
  const size_t oj = (size_t)j * nn;
  if (!tau_warp(w.n, w.U + (size_t)k * nn, w.Ea + oj, w.Ec + oj, w.Ep + oj, w.U + oj, sm))
    set_status(w.status, ST_SINGULAR);
}

// ---------------------------------------------------------------- local factors
// eq. (FW), (factor-local).  sm: 5 n^2 + 3 n m + m^2 T + n ints, then (FP32)
// B^T W B (m^2 T) and m^2 doubles for the FP64 fallback of the G Cholesky.
template <typename T>
__global__ void k_local_factor(Ws<T> w, int warp_bytes) {
  pdl_entry();
  const int j = warp_op();
  if (j >= w.N) return;
  const int n = w.n, m = w.m, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  T *sP = sm, *sF = sm + nn, *sFi = sm + 2 * nn, *sW = sm + 3 * nn, *sAcl = sm + 4 * nn;
  T *sB = sm + 5 * nn, *sWB = sB + n * m, *sH = sWB + n * m, *sG = sH + n * m;
  int* piv = reinterpret_cast<int*>(sG + m * m);
  unsigned char* tail = reinterpret_cast<unsigned char*>(sm) + ((sizeof(T) * (5 * nn + 3 * n * m + m * m) + 4 * n + 15) / 16) * 16;
  T* sBWB = reinterpret_cast<T*>(tail);
  double* scratch = reinterpret_cast<double*>(tail + ((sizeof(T) * m * m + 15) / 16) * 16);
  const size_t oj = (size_t)j * nn;
  wload(sP, w.U + oj, nn);
  const bool dnz = w.has_delta && w.dflag[j];
  __syncwarp();
  if (dnz) {
    // F = I + Delta P ; Finv = F^{-1} ; W = P F^{-1}
    const double* Dg = w.Delta + oj;
    wload(sAcl, Dg, nn);
    __syncwarp();
    wgemm<T, false, false>(n, n, n, sAcl, n, sP, n, sF, n, T(1), (const T*)nullptr, 0);
    wadd_identity(sF, n, n);
    wzero(sFi, nn);
    __syncwarp();
    wadd_identity(sFi, n, n);
    __syncwarp();
    if (!wlu(sF, n, n, piv)) { set_status(w.status, ST_SINGULAR); return; }
    wlu_solve(sF, n, n, piv, sFi, n, n);
    wload(w.Finv + oj, sFi, nn);
    wgemm<T, false, false>(n, n, n, sP, n, sFi, n, sW, n, T(1), (const T*)nullptr, 0);
    wload(w.W + oj, sW, nn);
  }
  if (node_is_root(w, j)) return;
  const T* Wuse = dnz ? sW : sP;
  const size_t onm = (size_t)j * n * m;
  wload(sB, w.B + onm, n * m);
  wload(sAcl, w.A + oj, nn);                       // A (becomes A_cl)
  wload(sG, w.R + (size_t)j * m * m, m * m);
  __syncwarp();
  wgemm<T, false, false>(n, m, n, Wuse, n, sB, m, sWB, m, T(1), (const T*)nullptr, 0);    // W B
  if constexpr (sizeof(T) == 8) {
    wgemm<T, true, false>(m, m, n, sB, m, sWB, m, sG, m, T(1), sG, m);                   // G = R + B^T W B
  } else {
    // keep B^T W B apart from R for a possible FP64 refactorisation of G
    wgemm<T, true, false>(m, m, n, sB, m, sWB, m, sBWB, m, T(1), (const T*)nullptr, 0);
    for (int e = lane_id(); e < m * m; e += 32) sG[e] += sBWB[e];
    __syncwarp();
  }
  // H = (W B)^T A + M^T  (B^T W A with W symmetric)
  wgemm<T, true, false>(m, n, n, sWB, m, sAcl, n, sH, n, T(1), (const T*)nullptr, 0);
  if (w.has_M) {
    const double* Mg = w.M + onm;
    for (int e = lane_id(); e < n * m; e += 32) {
      const int a = e / m, b = e - (e / m) * m;
      sH[b * n + a] += (T)Mg[e];
    }
    __syncwarp();
  }
  if (!wchol_checked(sG, m, m, w.R + (size_t)j * m * m, (const T*)sBWB, m, scratch)) {
    set_status(w.status, ST_NOT_PD);
    return;
  }
  wload(w.LG + (size_t)j * m * m, sG, m * m);
  wchol_solve(sG, m, m, sH, n, n);                 // G^{-1} H ; K = -G^{-1} H
  for (int e = lane_id(); e < m * n; e += 32) {
    sH[e] = -sH[e];
    w.K[onm + e] = sH[e];
  }
  __syncwarp();
  wgemm<T, false, false>(n, n, m, sB, m, sH, n, sAcl, n, T(1), sAcl, n);                 // A_cl = A + B K
  if (dnz)
    wgemm<T, false, false>(n, n, n, sFi, n, sAcl, n, w.Tm + oj, n, T(1), (const T*)nullptr, 0);  // T = F^{-1} A_cl
  else
    wload(w.Tm + oj, sAcl, nn);
}

// Composite transition matrices (eq. (transition-compose)) for every
// compression, in forward round order: Tr_j <- T_k ; T_k <- T_k T_j.
template <typename T>
__global__ void k_compose_T(Ws<T> w, int begin, int count, int warp_bytes) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int r = begin + t, j = w.comp_j[r], k = w.comp_k[r], n = w.n, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  T *sTk = sm, *sTj = sm + nn;
  wload(sTk, w.Tm + (size_t)k * nn, nn);
  wload(sTj, w.Tm + (size_t)j * nn, nn);
  __syncwarp();
  wload(w.Tr + (size_t)j * nn, sTk, nn);
  wgemm<T, false, false>(n, n, n, sTk, n, sTj, n, w.Tm + (size_t)k * nn, n, T(1), (const T*)nullptr, 0);
}

// ---------------------------------------------------------------- solve passes
// Affine edge data eq. (affine-edge) with h_i = q_i:
//   z_e = K^T r + A_cl^T W c_j = K^T (r + B^T w) + A^T w,  w = W_j c_j.
// sm: 2 n^2 + n m + m n + 4 (n + m) T.
template <typename T>
__global__ void k_aff_init(Ws<T> w, int warp_bytes) {
  pdl_entry();
  const int j = warp_op();
  if (j >= w.N) return;
  const int n = w.n, m = w.m, nn = n * n;
  wload(w.h + (size_t)j * n, w.q + (size_t)j * n, n);
  if (node_is_root(w, j)) return;
  T* sm = warp_smem<T>(warp_bytes);
  T *sWm = sm, *sA = sm + nn, *sB = sA + nn, *sK = sB + n * m, *vc = sK + m * n, *vw = vc + n,
    *vr = vw + n;
  const size_t oj = (size_t)j * nn, onm = (size_t)j * n * m;
  const bool dnz = w.has_delta && w.dflag[j];
  wload(sWm, dnz ? w.W + oj : w.U + oj, nn);
  wload(sA, w.A + oj, nn);
  wload(sB, w.B + onm, n * m);
  wload(sK, w.K + onm, m * n);
  wload(vc, w.c + (size_t)j * n, n);
  wload(vr, w.r + (size_t)j * m, m);
  __syncwarp();
  wgemv<T, false>(n, n, sWm, n, vc, vw, T(1), (const T*)nullptr);       // w = W c
  wgemv<T, true>(m, n, sB, m, vw, vr, T(1), vr);                          // r + B^T w
  wgemv<T, true>(n, n, sA, n, vw, vc, T(1), (const T*)nullptr);         // A^T w (into vc)
  wgemv<T, true>(n, m, sK, n, vr, w.z + (size_t)j * n, T(1), vc);        // K^T (.) + A^T w
}

// Affine rake eq. (affine-rake): contribution Z h_j + z, Z = T_j^T (current composite).
template <typename T>
__global__ void k_aff_rake(Ws<T> w, int begin, int count, int warp_bytes) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int r = begin + t, j = w.rake_leaf[r], n = w.n, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  T *sT = sm, *vh = sm + nn;
  wload(sT, w.Tm + (size_t)j * nn, nn);
  wload(vh, w.h + (size_t)j * n, n);
  __syncwarp();
  wgemv<T, true>(n, n, sT, n, vh, w.cv + (size_t)r * n, T(1), w.z + (size_t)j * n);
}

template <typename T>
__global__ void k_aff_absorb(Ws<T> w, int seg_begin, int count) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int s = seg_begin + t, i = w.seg_parent[s], n = w.n;
  const int b = w.seg_start[s], e = w.seg_start[s + 1];
  for (int x = lane_id(); x < n; x += 32) {
    T acc = w.cv[(size_t)b * n + x];
    for (int r = b + 1; r < e; ++r) acc += w.cv[(size_t)r * n + x];
    w.h[(size_t)i * n + x] += acc;
  }
}

// Affine compress eq. (affine-compose): s_j = h_j + z_r ; z_k <- z_l + Z_l s_j.
template <typename T>
__global__ void k_aff_compress(Ws<T> w, int begin, int count, int warp_bytes) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int r = begin + t, j = w.comp_j[r], k = w.comp_k[r], n = w.n, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  T *sT = sm, *vs = sm + nn;
  wload(sT, w.Tm + (size_t)j * nn, nn);
  wadd(vs, w.h + (size_t)j * n, w.z + (size_t)k * n, n);
  __syncwarp();
  wload(w.s + (size_t)j * n, vs, n);
  wgemv<T, true>(n, n, sT, n, vs, w.z + (size_t)k * n, T(1), w.z + (size_t)j * n);
}

// Affine expansion: p_j = Z_r p_k + s_j with Z_r = Tr_j^T (over h_j).
template <typename T>
__global__ void k_aff_expand(Ws<T> w, int begin, int count, int warp_bytes) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int r = begin + t, j = w.comp_j[r], k = w.comp_k[r], n = w.n, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  T *sT = sm, *vp = sm + nn;
  wload(sT, w.Tr + (size_t)j * nn, nn);
  wload(vp, w.h + (size_t)k * n, n);
  __syncwarp();
  wgemv<T, true>(n, n, sT, n, vp, w.h + (size_t)j * n, T(1), w.s + (size_t)j * n);
}

// Local affine solve eq. (local-affine-solve) and root state eq. (xroot):
//   f = Delta p - c, g = p - W f, k = -G^{-1}(r + B^T g), b = F^{-1}(B k - f).
template <typename T>
__global__ void k_local_solve(Ws<T> w, int warp_bytes) {
  pdl_entry();
  const int j = warp_op();
  if (j >= w.N) return;
  const int n = w.n, m = w.m, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  T *sMat = sm, *sB = sm + nn, *sL = sB + n * m, *vp = sL + m * m, *vf = vp + n, *vg = vf + n,
    *vk = vg + n, *vt = vk + m;
  const size_t oj = (size_t)j * nn;
  const bool dnz = w.has_delta && w.dflag[j];
  wload(vp, w.h + (size_t)j * n, n);
  if (dnz) wload(sMat, w.Delta + oj, nn);
  __syncwarp();
  if (dnz) wgemv<T, false>(n, n, sMat, n, vp, vf, T(1), (const T*)nullptr);
  else wzero(vf, n);
  __syncwarp();
  for (int a = lane_id(); a < n; a += 32) vf[a] -= (T)w.c[(size_t)j * n + a];
  __syncwarp();
  if (node_is_root(w, j)) {
    // x_rho = -F^{-1} f
    if (dnz) {
      wload(sMat, w.Finv + oj, nn);
      __syncwarp();
      wgemv<T, false>(n, n, sMat, n, vf, w.xs + (size_t)j * n, T(-1), (const T*)nullptr);
    } else {
      for (int a = lane_id(); a < n; a += 32) w.xs[(size_t)j * n + a] = -vf[a];
    }
    return;
  }
  // g = p - W f
  wload(sMat, dnz ? w.W + oj : w.U + oj, nn);
  wload(sB, w.B + (size_t)j * n * m, n * m);
  wload(sL, w.LG + (size_t)j * m * m, m * m);
  __syncwarp();
  wgemv<T, false>(n, n, sMat, n, vf, vg, T(-1), vp);
  // k = -G^{-1}(r + B^T g)
  wgemv<T, true>(m, n, sB, m, vg, vk, T(1), w.r + (size_t)j * m);
  wchol_solve(sL, m, m, vk, 1, 1);
  for (int a = lane_id(); a < m; a += 32) vk[a] = -vk[a];
  __syncwarp();
  wload(w.kv + (size_t)j * m, vk, m);
  // b = F^{-1}(B k - f)
  wgemv<T, false>(n, m, sB, m, vk, vt, T(1), (const T*)nullptr);
  for (int a = lane_id(); a < n; a += 32) vt[a] -= vf[a];
  __syncwarp();
  if (dnz) {
    wload(sMat, w.Finv + oj, nn);
    __syncwarp();
    wgemv<T, false>(n, n, sMat, n, vt, w.bv + (size_t)j * n, T(1), (const T*)nullptr);
  } else {
    wload(w.bv + (size_t)j * n, vt, n);
  }
}

// State-map compression eq. (transition-compose) (offsets only; the matrices
// were composed once in the factorisation): b_k <- T_r b_l + b_r, T_r = Tr_j.
template <typename T>
__global__ void k_state_compress(Ws<T> w, int begin, int count, int warp_bytes) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int r = begin + t, j = w.comp_j[r], k = w.comp_k[r], n = w.n, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  T *sT = sm, *vb = sm + nn;
  wload(sT, w.Tr + (size_t)j * nn, nn);
  wload(vb, w.bv + (size_t)j * n, n);
  __syncwarp();
  wgemv<T, false>(n, n, sT, n, vb, w.bv + (size_t)k * n, T(1), w.bv + (size_t)k * n);
}

// State expansion: x_j = T_j x_i + b_j with the current (composite) map of the
// edge that entered j when it was removed; `from` = comp_i or rake_parent.
template <typename T>
__global__ void k_state_expand(Ws<T> w, const int* nodes, const int* from, int begin, int count,
                               int warp_bytes) {
  pdl_entry();
  const int t = warp_op();
  if (t >= count) return;
  const int r = begin + t, j = nodes[r], i = from[r], n = w.n, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  T *sT = sm, *vx = sm + nn;
  wload(sT, w.Tm + (size_t)j * nn, nn);
  wload(vx, w.xs + (size_t)i * n, n);
  __syncwarp();
  wgemv<T, false>(n, n, sT, n, vx, w.xs + (size_t)j * n, T(1), w.bv + (size_t)j * n);
}

// Recovery eq. (recover): u_e = K_e x_i + k_e, y_i = P_i x_i + p_i; results in
// FP64, written or (accumulate = 1) added to x, u, y.
template <typename T>
__global__ void k_recover(Ws<T> w, double* x, double* u, double* y, int accumulate, int warp_bytes) {
  pdl_entry();
  const int j = warp_op();
  if (j >= w.N) return;
  const int n = w.n, m = w.m, nn = n * n;
  T* sm = warp_smem<T>(warp_bytes);
  T *sP = sm, *sK = sm + nn, *vx = sK + m * n, *vxp = vx + n, *vo = vxp + n;
  wload(sP, w.U + (size_t)j * nn, nn);
  wload(vx, w.xs + (size_t)j * n, n);
  const bool nonroot = !node_is_root(w, j);
  if (nonroot) {
    wload(sK, w.K + (size_t)j * m * n, m * n);
    wload(vxp, w.xs + (size_t)w.parent[j] * n, n);
  }
  __syncwarp();
  wgemv<T, false>(n, n, sP, n, vx, vo, T(1), w.h + (size_t)j * n);
  bool bad = false;
  for (int a = lane_id(); a < n; a += 32) {
    const size_t o = (size_t)j * n + a;
    bad |= !tfinite(vx[a]) || !tfinite(vo[a]);
    if (accumulate) { x[o] += (double)vx[a]; y[o] += (double)vo[a]; }
    else { x[o] = (double)vx[a]; y[o] = (double)vo[a]; }
  }
  __syncwarp();
  if (nonroot) {
    wgemv<T, false>(m, n, sK, n, vxp, vo, T(1), w.kv + (size_t)j * m);
    for (int a = lane_id(); a < m; a += 32) {
      const size_t o = (size_t)j * m + a;
      bad |= !tfinite(vo[a]);
      if (accumulate) u[o] += (double)vo[a]; else u[o] = (double)vo[a];
    }
  } else if (!accumulate) {
    for (int a = lane_id(); a < m; a += 32) u[(size_t)j * m + a] = 0.0;
  }
  if (wany(bad)) set_status(w.status, ST_NONFINITE);
}

// Widen P (= U after the reverse pass) and K to FP64 outputs.
template <typename T>
__global__ void k_export_PK(int N, int n, int m, const int* parent, const T* U, const T* K, double* P, double* Ko) {
  pdl_entry();
  const size_t nn = (size_t)n * n, mn = (size_t)m * n;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (P) for (size_t e = tid; e < (size_t)N * nn; e += stride) P[e] = (double)U[e];
  if (Ko)
    for (size_t e = tid; e < (size_t)N * mn; e += stride)
      Ko[e] = (parent[e / mn] < 0) ? 0.0 : (double)K[e];
}

}  // namespace tlqr
