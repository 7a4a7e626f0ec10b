// FP64 KKT residual of eq. (kkt) on the tree, and the quantities of the
// normwise backward error eta = ||K z - b||_inf / (||K||_inf ||z||_inf + ||b||_inf).
//
// One warp per node i computes
//   res_x[i] = Q_i x_i + q_i - y_i + sum_{children j} (M_j u_j + A_j^T y_j)
//   res_u[i] = M_i^T x_p + R_i u_i + r_i + B_i^T y_i                (i nonroot, p = parent)
//   res_c[i] = A_i x_p + B_i u_i + c_i - x_i - Delta_i y_i           (i nonroot)
//   res_c[rho] = c_rho - x_rho - Delta_rho y_rho
// and the absolute row sums of the KKT matrix for the same rows.  Maxima are
// combined with atomicMax on the bit patterns of nonnegative doubles, whose
// integer order equals their numeric order, so the result is deterministic.
#pragma once
#include <cstdint>

namespace tlqr {

struct ResidualArgs {
  int N, n, m, root;
  const int *parent, *child_start, *child_list;
  const double *Q, *q, *M, *R, *r, *A, *B, *c, *Delta;
  const double *x, *u, *y;
  double *res_x, *res_u, *res_c;
  unsigned long long* maxes;   // [0] ||res||, [1] ||z||, [2] ||b||, [3] ||K|| (row sums)
};

// running max of |v|; a NaN turns the maximum into +inf so that it is never hidden
__device__ __forceinline__ double amax(double acc, double v) { return isnan(v) ? INFINITY : fmax(acc, fabs(v)); }

__device__ __forceinline__ void warp_max_to(unsigned long long* dst, double v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_residual(ResidualArgs a) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= a.N) return;
  const int lane = threadIdx.x & 31, n = a.n, m = a.m;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m;
  double rmax = 0, zmax = 0, bmax = 0, kmax = 0;
  const double* xi = a.x + (size_t)i * n;
  const double* yi = a.y + (size_t)i * n;
  // node row (kkt-x)
  for (int r = lane; r < n; r += 32) {
    const double* Qr = a.Q + (size_t)i * nn + (size_t)r * n;
    double s = a.q[(size_t)i * n + r] - yi[r], rs = 1.0;
    for (int b = 0; b < n; ++b) { s = fma(Qr[b], xi[b], s); rs += fabs(Qr[b]); }
    for (int t = a.child_start[i]; t < a.child_start[i + 1]; ++t) {
      const int j = a.child_list[t];
      const double* Aj = a.A + (size_t)j * nn;
      const double* yj = a.y + (size_t)j * n;
      for (int b = 0; b < n; ++b) { s = fma(Aj[(size_t)b * n + r], yj[b], s); rs += fabs(Aj[(size_t)b * n + r]); }
      if (a.M) {
        const double* Mr = a.M + (size_t)j * nm + (size_t)r * m;
        const double* uj = a.u + (size_t)j * m;
        for (int b = 0; b < m; ++b) { s = fma(Mr[b], uj[b], s); rs += fabs(Mr[b]); }
      }
    }
    a.res_x[(size_t)i * n + r] = s;
    rmax = amax(rmax, s); kmax = fmax(kmax, rs);
    zmax = amax(amax(zmax, xi[r]), yi[r]);
    bmax = fmax(bmax, fmax(fabs(a.q[(size_t)i * n + r]), fabs(a.c[(size_t)i * n + r])));
  }
  const double* Di = a.Delta ? a.Delta + (size_t)i * nn : nullptr;
  if (i == a.root) {
    for (int r = lane; r < n; r += 32) {
      double s = a.c[(size_t)i * n + r] - xi[r], rs = 1.0;
      if (Di) for (int b = 0; b < n; ++b) { s = fma(-Di[(size_t)r * n + b], yi[b], s); rs += fabs(Di[(size_t)r * n + b]); }
      a.res_c[(size_t)i * n + r] = s;
      rmax = amax(rmax, s); kmax = fmax(kmax, rs);
    }
    for (int r = lane; r < m; r += 32) a.res_u[(size_t)i * m + r] = 0.0;
  } else {
    const int p = a.parent[i];
    const double* xp = a.x + (size_t)p * n;
    const double* ui = a.u + (size_t)i * m;
    const double* Ai = a.A + (size_t)i * nn;
    const double* Bi = a.B + (size_t)i * nm;
    const double* Ri = a.R + (size_t)i * m * m;
    const double* Mi = a.M ? a.M + (size_t)i * nm : nullptr;
    for (int r = lane; r < m; r += 32) {            // (kkt-u)
      double s = a.r[(size_t)i * m + r], rs = 0.0;
      if (Mi) for (int b = 0; b < n; ++b) { s = fma(Mi[(size_t)b * m + r], xp[b], s); rs += fabs(Mi[(size_t)b * m + r]); }
      for (int b = 0; b < m; ++b) { s = fma(Ri[(size_t)r * m + b], ui[b], s); rs += fabs(Ri[(size_t)r * m + b]); }
      for (int b = 0; b < n; ++b) { s = fma(Bi[(size_t)b * m + r], yi[b], s); rs += fabs(Bi[(size_t)b * m + r]); }
      a.res_u[(size_t)i * m + r] = s;
      rmax = amax(rmax, s); kmax = fmax(kmax, rs);
      zmax = amax(zmax, ui[r]);
      bmax = fmax(bmax, fabs(a.r[(size_t)i * m + r]));
    }
    for (int r = lane; r < n; r += 32) {            // (kkt-dyn)
      double s = a.c[(size_t)i * n + r] - xi[r], rs = 1.0;
      for (int b = 0; b < n; ++b) { s = fma(Ai[(size_t)r * n + b], xp[b], s); rs += fabs(Ai[(size_t)r * n + b]); }
      for (int b = 0; b < m; ++b) { s = fma(Bi[(size_t)r * m + b], ui[b], s); rs += fabs(Bi[(size_t)r * m + b]); }
      if (Di) for (int b = 0; b < n; ++b) { s = fma(-Di[(size_t)r * n + b], yi[b], s); rs += fabs(Di[(size_t)r * n + b]); }
      a.res_c[(size_t)i * n + r] = s;
      rmax = amax(rmax, s); kmax = fmax(kmax, rs);
    }
  }
  warp_max_to(a.maxes + 0, rmax);
  warp_max_to(a.maxes + 1, zmax);
  warp_max_to(a.maxes + 2, bmax);
  warp_max_to(a.maxes + 3, kmax);
}

}  // namespace tlqr
