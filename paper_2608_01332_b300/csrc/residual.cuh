// FP64 KKT residual of eq. (kkt) on the tree, and the quantities of the
// normwise backward error eta = ||K z - b||_inf / (||K||_inf ||z||_inf + ||b||_inf).
//
// One thread per KKT row (grid-stride over N n + N m + N n rows):
//   row (i, r) of (kkt-x):   Q_i x_i + q_i - y_i + sum_{children j} (M_j u_j + A_j^T y_j)
//   row (i, r) of (kkt-u):   M_i^T x_p + R_i u_i + r_i + B_i^T y_i          (i nonroot, p = parent)
//   row (i, r) of the constraint entering i:
//        A_i x_p + B_i u_i + c_i - x_i - Delta_i y_i                          (i nonroot)
//        c_rho - x_rho - Delta_rho y_rho                                       (root)
// Adjacent threads own adjacent rows of one block, so the column reads
// (A_j^T, B^T, M^T) are coalesced and the row reads are served from L1.
// The absolute row sums of the KKT matrix (||K||_inf) depend only on the
// matrices; they are formed when `with_knorm` is set and otherwise kept from an
// earlier call.  Maxima are combined with atomicMax on the bit patterns of
// nonnegative doubles (integer order = numeric order), so results are
// deterministic; a NaN turns a maximum into +inf.
#pragma once
#include <cstdint>

namespace tlqr {

struct ResidualArgs {
  int N, n, m, root, with_knorm;
  const int *parent, *child_start, *child_list;
  const double *Q, *q, *M, *R, *r, *A, *B, *c, *Delta;
  const double *x, *u, *y;
  double *res_x, *res_u, *res_c;
  unsigned long long* maxes;   // [0] ||res||, [1] ||z||, [2] ||b||, [3] ||K|| (row sums)
};

__device__ __forceinline__ double amax(double acc, double v) { return isnan(v) ? INFINITY : fmax(acc, fabs(v)); }

__device__ __forceinline__ void warp_max_to(unsigned long long* dst, double v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_residual(ResidualArgs a) {
  const int n = a.n, m = a.m;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m;
  const size_t rows_x = (size_t)a.N * n, rows_u = (size_t)a.N * m, total = 2 * rows_x + rows_u;
  double rmax = 0, zmax = 0, bmax = 0, kmax = 0;
  const bool ks = a.with_knorm;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    if (t < rows_x) {                                   // (kkt-x)
      const int i = (int)(t / n), r = (int)(t - (size_t)i * n);
      const double* Qr = a.Q + (size_t)i * nn + (size_t)r * n;
      const double* xi = a.x + (size_t)i * n;
      const double yir = a.y[t];
      double s = a.q[t] - yir, rs = 1.0;
      for (int b = 0; b < n; ++b) { s = fma(Qr[b], xi[b], s); if (ks) rs += fabs(Qr[b]); }
      for (int k = a.child_start[i]; k < a.child_start[i + 1]; ++k) {
        const int j = a.child_list[k];
        const double* Aj = a.A + (size_t)j * nn + r;
        const double* yj = a.y + (size_t)j * n;
        for (int b = 0; b < n; ++b) { s = fma(Aj[(size_t)b * n], yj[b], s); if (ks) rs += fabs(Aj[(size_t)b * n]); }
        if (a.M) {
          const double* Mr = a.M + (size_t)j * nm + (size_t)r * m;
          const double* uj = a.u + (size_t)j * m;
          for (int b = 0; b < m; ++b) { s = fma(Mr[b], uj[b], s); if (ks) rs += fabs(Mr[b]); }
        }
      }
      a.res_x[t] = s;
      rmax = amax(rmax, s);
      kmax = fmax(kmax, rs);
      zmax = amax(amax(zmax, a.x[t]), yir);
      bmax = fmax(bmax, fmax(fabs(a.q[t]), fabs(a.c[t])));
    } else if (t < rows_x + rows_u) {                   // (kkt-u)
      const size_t tu = t - rows_x;
      const int i = (int)(tu / m), r = (int)(tu - (size_t)i * m);
      if (i == a.root) { a.res_u[tu] = 0.0; continue; }
      const int p = a.parent[i];
      const double* xp = a.x + (size_t)p * n;
      const double* ui = a.u + (size_t)i * m;
      const double* yi = a.y + (size_t)i * n;
      const double* Bc = a.B + (size_t)i * nm + r;      // column r of B_i
      const double* Rr = a.R + (size_t)i * m * m + (size_t)r * m;
      double s = a.r[tu], rs = 0.0;
      if (a.M) {
        const double* Mc = a.M + (size_t)i * nm + r;
        for (int b = 0; b < n; ++b) { s = fma(Mc[(size_t)b * m], xp[b], s); if (ks) rs += fabs(Mc[(size_t)b * m]); }
      }
      for (int b = 0; b < m; ++b) { s = fma(Rr[b], ui[b], s); if (ks) rs += fabs(Rr[b]); }
      for (int b = 0; b < n; ++b) { s = fma(Bc[(size_t)b * m], yi[b], s); if (ks) rs += fabs(Bc[(size_t)b * m]); }
      a.res_u[tu] = s;
      rmax = amax(rmax, s);
      kmax = fmax(kmax, rs);
      zmax = amax(zmax, ui[r]);
      bmax = fmax(bmax, fabs(a.r[tu]));
    } else {                                            // constraint entering i
      const size_t tc = t - rows_x - rows_u;
      const int i = (int)(tc / n), r = (int)(tc - (size_t)i * n);
      const double* yi = a.y + (size_t)i * n;
      double s = a.c[tc] - a.x[tc], rs = 1.0;
      if (a.Delta) {
        const double* Dr = a.Delta + (size_t)i * nn + (size_t)r * n;
        for (int b = 0; b < n; ++b) { s = fma(-Dr[b], yi[b], s); if (ks) rs += fabs(Dr[b]); }
      }
      if (i != a.root) {
        const int p = a.parent[i];
        const double* xp = a.x + (size_t)p * n;
        const double* ui = a.u + (size_t)i * m;
        const double* Ar = a.A + (size_t)i * nn + (size_t)r * n;
        const double* Br = a.B + (size_t)i * nm + (size_t)r * m;
        for (int b = 0; b < n; ++b) { s = fma(Ar[b], xp[b], s); if (ks) rs += fabs(Ar[b]); }
        for (int b = 0; b < m; ++b) { s = fma(Br[b], ui[b], s); if (ks) rs += fabs(Br[b]); }
      }
      a.res_c[tc] = s;
      rmax = amax(rmax, s);
      kmax = fmax(kmax, rs);
    }
  }
  warp_max_to(a.maxes + 0, rmax);
  warp_max_to(a.maxes + 1, zmax);
  warp_max_to(a.maxes + 2, bmax);
  if (ks) warp_max_to(a.maxes + 3, kmax);
}

}  // namespace tlqr

namespace tlqr {

// ------------------------------------------------------------------ float-float residual
// The same residual rows as k_residual, evaluated in "float-float" arithmetic
// on the FP32 pipe: every FP64 operand a is split with integer bit operations
// into a_hi + a_lo (a_hi = a truncated to 24 significant bits, a_lo = the
// remaining 29 bits rounded to 24), products keep their exact rounding error
// through fma, and sums are accumulated with Knuth's two-sum.  About 47
// significant bits survive, i.e. the residual is accurate to ~1e-14 of the
// magnitude of its terms -- ample for driving eta below 1e-8 -- while B300's
// FP32 rate is ~60x its FP64 rate.  Operands with |a| >= 2^128 make the row
// infinite (reported as nonfinite); |a| < 2^-126 are taken as zero.
__device__ __forceinline__ void dsplit(double a, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const int e32 = (int)((b >> 52) & 0x7ffu) - 1023 + 127;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  if (e32 >= 1 && e32 <= 254) {
    hi = __uint_as_float(sign | ((unsigned)e32 << 23) | (unsigned)((b >> 29) & 0x7fffffu));
    float l = (float)(unsigned)(b & 0x1fffffffu);                 // low 29 mantissa bits
    l *= 2.220446049250313e-16f;                                    // 2^-52
    l *= __uint_as_float((unsigned)e32 << 23);                      // 2^(e32 - 127)
    lo = sign ? -l : l;
  } else if (e32 < 1) {
    hi = 0.f;
    lo = 0.f;
  } else {
    hi = __uint_as_float(sign | 0x7f800000u | (unsigned)((b >> 29) & 0x7fffffu));   // inf or nan
    lo = 0.f;
  }
}

struct FF { float h, l; };

// acc += a * x
__device__ __forceinline__ void ff_fma(FF& acc, double a, double x) {
  float ah, al, xh, xl;
  dsplit(a, ah, al);
  dsplit(x, xh, xl);
  const float p = ah * xh;
  float pe = fmaf(ah, xh, -p);
  pe = fmaf(ah, xl, pe);
  pe = fmaf(al, xh, pe);
  const float s = acc.h + p;
  const float bb = s - acc.h;
  const float err = (acc.h - (s - bb)) + (p - bb);
  acc.l += err + pe;
  acc.h = s;
}
// acc += a
__device__ __forceinline__ void ff_add(FF& acc, double a) {
  float ah, al;
  dsplit(a, ah, al);
  const float s = acc.h + ah;
  const float bb = s - acc.h;
  const float err = (acc.h - (s - bb)) + (ah - bb);
  acc.l += err + al;
  acc.h = s;
}
__device__ __forceinline__ double ff_value(const FF& v) { return (double)v.h + (double)v.l; }
__device__ __forceinline__ float absf_of(double a) {
  float h, l;
  dsplit(a, h, l);
  return fabsf(h);
}
// |v| as ordered bits (integer max), NaN sorts above +inf
__device__ __forceinline__ unsigned long long abits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ void warp_maxbits_to(unsigned long long* dst, unsigned long long v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  if ((threadIdx.x & 31) == 0 && v) atomicMax(dst, v);
}

__global__ void k_residual_ff(ResidualArgs a) {
  const int n = a.n, m = a.m;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m;
  const size_t rows_x = (size_t)a.N * n, rows_u = (size_t)a.N * m, total = 2 * rows_x + rows_u;
  unsigned long long rmax = 0, zmax = 0, bmax = 0;
  float kmax = 0.f;
  const bool ks = a.with_knorm;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    double out;
    if (t < rows_x) {                                   // (kkt-x)
      const int i = (int)(t / n), r = (int)(t - (size_t)i * n);
      const double* Qr = a.Q + (size_t)i * nn + (size_t)r * n;
      const double* xi = a.x + (size_t)i * n;
      const double yir = a.y[t];
      FF s{0.f, 0.f};
      ff_add(s, a.q[t]);
      ff_add(s, -yir);
      float rs = 1.f;
      for (int b = 0; b < n; ++b) { ff_fma(s, Qr[b], xi[b]); if (ks) rs += absf_of(Qr[b]); }
      for (int k = a.child_start[i]; k < a.child_start[i + 1]; ++k) {
        const int j = a.child_list[k];
        const double* Aj = a.A + (size_t)j * nn + r;
        const double* yj = a.y + (size_t)j * n;
        for (int b = 0; b < n; ++b) { ff_fma(s, Aj[(size_t)b * n], yj[b]); if (ks) rs += absf_of(Aj[(size_t)b * n]); }
        if (a.M) {
          const double* Mr = a.M + (size_t)j * nm + (size_t)r * m;
          const double* uj = a.u + (size_t)j * m;
          for (int b = 0; b < m; ++b) { ff_fma(s, Mr[b], uj[b]); if (ks) rs += absf_of(Mr[b]); }
        }
      }
      out = ff_value(s);
      a.res_x[t] = out;
      kmax = fmaxf(kmax, rs);
      const unsigned long long zx = abits(a.x[t]), zy = abits(yir);
      zmax = zx > zmax ? zx : zmax;
      zmax = zy > zmax ? zy : zmax;
      const unsigned long long bq = abits(a.q[t]), bc = abits(a.c[t]);
      bmax = bq > bmax ? bq : bmax;
      bmax = bc > bmax ? bc : bmax;
    } else if (t < rows_x + rows_u) {                   // (kkt-u)
      const size_t tu = t - rows_x;
      const int i = (int)(tu / m), r = (int)(tu - (size_t)i * m);
      if (i == a.root) { a.res_u[tu] = 0.0; continue; }
      const int p = a.parent[i];
      const double* xp = a.x + (size_t)p * n;
      const double* ui = a.u + (size_t)i * m;
      const double* yi = a.y + (size_t)i * n;
      const double* Bc = a.B + (size_t)i * nm + r;
      const double* Rr = a.R + (size_t)i * m * m + (size_t)r * m;
      FF s{0.f, 0.f};
      ff_add(s, a.r[tu]);
      float rs = 0.f;
      if (a.M) {
        const double* Mc = a.M + (size_t)i * nm + r;
        for (int b = 0; b < n; ++b) { ff_fma(s, Mc[(size_t)b * m], xp[b]); if (ks) rs += absf_of(Mc[(size_t)b * m]); }
      }
      for (int b = 0; b < m; ++b) { ff_fma(s, Rr[b], ui[b]); if (ks) rs += absf_of(Rr[b]); }
      for (int b = 0; b < n; ++b) { ff_fma(s, Bc[(size_t)b * m], yi[b]); if (ks) rs += absf_of(Bc[(size_t)b * m]); }
      out = ff_value(s);
      a.res_u[tu] = out;
      kmax = fmaxf(kmax, rs);
      const unsigned long long zu = abits(ui[r]), br = abits(a.r[tu]);
      zmax = zu > zmax ? zu : zmax;
      bmax = br > bmax ? br : bmax;
    } else {                                            // constraint entering i
      const size_t tc = t - rows_x - rows_u;
      const int i = (int)(tc / n), r = (int)(tc - (size_t)i * n);
      const double* yi = a.y + (size_t)i * n;
      FF s{0.f, 0.f};
      ff_add(s, a.c[tc]);
      ff_add(s, -a.x[tc]);
      float rs = 1.f;
      if (a.Delta) {
        const double* Dr = a.Delta + (size_t)i * nn + (size_t)r * n;
        for (int b = 0; b < n; ++b) { ff_fma(s, -Dr[b], yi[b]); if (ks) rs += absf_of(Dr[b]); }
      }
      if (i != a.root) {
        const int p = a.parent[i];
        const double* xp = a.x + (size_t)p * n;
        const double* ui = a.u + (size_t)i * m;
        const double* Ar = a.A + (size_t)i * nn + (size_t)r * n;
        const double* Br = a.B + (size_t)i * nm + (size_t)r * m;
        for (int b = 0; b < n; ++b) { ff_fma(s, Ar[b], xp[b]); if (ks) rs += absf_of(Ar[b]); }
        for (int b = 0; b < m; ++b) { ff_fma(s, Br[b], ui[b]); if (ks) rs += absf_of(Br[b]); }
      }
      out = ff_value(s);
      a.res_c[tc] = out;
      kmax = fmaxf(kmax, rs);
    }
    const unsigned long long ob = abits(out);
    rmax = ob > rmax ? ob : rmax;
  }
  warp_maxbits_to(a.maxes + 0, rmax);
  warp_maxbits_to(a.maxes + 1, zmax);
  warp_maxbits_to(a.maxes + 2, bmax);
  if (ks) warp_maxbits_to(a.maxes + 3, abits((double)kmax));
}

}  // namespace tlqr
