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
  int N, n, m, with_knorm;
  const int *parent, *child_start, *child_list;
  const double *Q, *q, *M, *R, *r, *A, *B, *c, *Delta;
  const double *x, *u, *y;
  double *res_x, *res_u, *res_c;
  unsigned long long* maxes;   // [0] ||res||, [1] ||z||, [2] ||b||, [3] ||K|| (row sums); slot-major [4][T]
  const int* tree;             // forest: tree ordinal of each node (null: one tree)
  int T;                       // number of trees (1 for a single tree)
  const unsigned char* dflag;  // per node: Delta_i has a nonzero entry (null: every Delta_i is read)
};

__device__ __forceinline__ double amax(double acc, double v) { return isnan(v) ? INFINITY : fmax(acc, fabs(v)); }

__device__ __forceinline__ void warp_max_to(unsigned long long* dst, double v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

// Block-wide maximum of nonnegative 64-bit keys, one atomicMax per block.
// Every thread of the block must call it (it synchronises the block).
__device__ __forceinline__ void block_maxbits_to(unsigned long long* dst, unsigned long long v) {
  __shared__ unsigned long long red[32];
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? red[lane] : 0ull;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
      v = o > v ? o : v;
    }
    if (lane == 0 && v) atomicMax(dst, v);
  }
}
__device__ __forceinline__ unsigned long long dbits_abs(double v) {
  return isnan(v) ? 0x7ff8000000000000ull : (unsigned long long)__double_as_longlong(fabs(v));
}

// Row t of eq. (kkt) in FP64.  Returns the residual entry (also stored) and
// sets rs = the row's absolute sum of KKT entries (when ks), zv = max |z| and
// bv = max |b| of the entries this row owns, and node = the node of the row.
// The u row of a root is empty: it stores 0 and contributes nothing.
__device__ __forceinline__ double fp64_row(const ResidualArgs& a, size_t t, bool ks, double& rs, double& zv,
                                           double& bv, int& node) {
  const int n = a.n, m = a.m;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m;
  const size_t rows_x = (size_t)a.N * n, rows_u = (size_t)a.N * m;
  rs = 0.0; zv = 0.0; bv = 0.0;
  if (t < rows_x) {                                   // (kkt-x)
    const int i = (int)(t / n), r = (int)(t - (size_t)i * n);
    node = i;
    const double* Qr = a.Q + (size_t)i * nn + (size_t)r * n;
    const double* xi = a.x + (size_t)i * n;
    const double yir = a.y[t];
    double s = a.q[t] - yir;
    rs = 1.0;
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
    zv = amax(amax(0.0, a.x[t]), yir);
    bv = fmax(fabs(a.q[t]), fabs(a.c[t]));
    return s;
  }
  if (t < rows_x + rows_u) {                          // (kkt-u)
    const size_t tu = t - rows_x;
    const int i = (int)(tu / m), r = (int)(tu - (size_t)i * m);
    node = i;
    if (a.parent[i] < 0) { a.res_u[tu] = 0.0; return 0.0; }
    const int p = a.parent[i];
    const double* xp = a.x + (size_t)p * n;
    const double* ui = a.u + (size_t)i * m;
    const double* yi = a.y + (size_t)i * n;
    const double* Bc = a.B + (size_t)i * nm + r;      // column r of B_i
    const double* Rr = a.R + (size_t)i * m * m + (size_t)r * m;
    double s = a.r[tu];
    if (a.M) {
      const double* Mc = a.M + (size_t)i * nm + r;
      for (int b = 0; b < n; ++b) { s = fma(Mc[(size_t)b * m], xp[b], s); if (ks) rs += fabs(Mc[(size_t)b * m]); }
    }
    for (int b = 0; b < m; ++b) { s = fma(Rr[b], ui[b], s); if (ks) rs += fabs(Rr[b]); }
    for (int b = 0; b < n; ++b) { s = fma(Bc[(size_t)b * m], yi[b], s); if (ks) rs += fabs(Bc[(size_t)b * m]); }
    a.res_u[tu] = s;
    zv = amax(0.0, ui[r]);
    bv = fabs(a.r[tu]);
    return s;
  }
  const size_t tc = t - rows_x - rows_u;              // constraint entering i
  const int i = (int)(tc / n), r = (int)(tc - (size_t)i * n);
  node = i;
  const double* yi = a.y + (size_t)i * n;
  double s = a.c[tc] - a.x[tc];
  rs = 1.0;
  if (a.Delta && (!a.dflag || a.dflag[i])) {
    const double* Dr = a.Delta + (size_t)i * nn + (size_t)r * n;
    for (int b = 0; b < n; ++b) { s = fma(-Dr[b], yi[b], s); if (ks) rs += fabs(Dr[b]); }
  }
  if (a.parent[i] >= 0) {
    const int p = a.parent[i];
    const double* xp = a.x + (size_t)p * n;
    const double* ui = a.u + (size_t)i * m;
    const double* Ar = a.A + (size_t)i * nn + (size_t)r * n;
    const double* Br = a.B + (size_t)i * nm + (size_t)r * m;
    for (int b = 0; b < n; ++b) { s = fma(Ar[b], xp[b], s); if (ks) rs += fabs(Ar[b]); }
    for (int b = 0; b < m; ++b) { s = fma(Br[b], ui[b], s); if (ks) rs += fabs(Br[b]); }
  }
  a.res_c[tc] = s;
  return s;
}

__global__ void k_residual(ResidualArgs a) {
  const size_t total = (size_t)a.N * (2 * a.n + a.m);
  double rmax = 0, zmax = 0, bmax = 0, kmax = 0;
  const bool ks = a.with_knorm;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    double rs, zv, bv;
    int node;
    const double s = fp64_row(a, t, ks, rs, zv, bv, node);
    rmax = amax(rmax, s);
    kmax = fmax(kmax, rs);
    zmax = fmax(zmax, zv);
    bmax = fmax(bmax, bv);
  }
  block_maxbits_to(a.maxes + 0, dbits_abs(rmax));
  block_maxbits_to(a.maxes + 1, dbits_abs(zmax));
  block_maxbits_to(a.maxes + 2, dbits_abs(bmax));
  if (ks) block_maxbits_to(a.maxes + 3, dbits_abs(kmax));
}

// ------------------------------------------------------------------ per-tree maxima (forests)
// A batch of trees needs eta tree by tree: each tree's solution must meet the
// tolerance on its own, as it would when solved alone.  The per-tree kernels
// give every warp one contiguous range of rows, walked 32 rows at a time.
// While all lanes' rows belong to one tree the four maxima stay in registers
// and are folded into maxes[slot * T + tree] when the warp moves to another
// tree; a step whose lanes straddle trees folds its rows one by one.
struct TreeAcc {
  int cur = -1;
  unsigned long long v[4] = {0ull, 0ull, 0ull, 0ull};

  // warp-uniform
  __device__ __forceinline__ void flush(const ResidualArgs& a, int nslots) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q >= nslots) break;
      unsigned long long w = v[q];
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, w, off);
        w = o > w ? o : w;
      }
      if ((threadIdx.x & 31) == 0 && cur >= 0 && w) atomicMax(a.maxes + (size_t)q * a.T + cur, w);
      v[q] = 0ull;
    }
  }
  // warp-uniform; r[] of an invalid lane is ignored
  __device__ __forceinline__ void add(const ResidualArgs& a, int nslots, bool valid, int tree,
                                      const unsigned long long (&r)[4]) {
    const int mine = valid ? tree : -1;
    const int lead = __shfl_sync(0xffffffffu, mine, 0);
    if (__all_sync(0xffffffffu, mine == lead || mine < 0)) {
      if (lead != cur) {
        flush(a, nslots);
        cur = lead;
      }
      if (valid) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nslots) v[q] = r[q] > v[q] ? r[q] : v[q];
      }
    } else if (valid) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < nslots && r[q]) atomicMax(a.maxes + (size_t)q * a.T + tree, r[q]);
    }
  }
};

// This warp's contiguous row range [beg, end) (32-row aligned chunks).
__device__ __forceinline__ void warp_rows(size_t total, size_t& beg, size_t& end) {
  const size_t wpb = blockDim.x >> 5, warps = (size_t)gridDim.x * wpb;
  const size_t gw = (size_t)blockIdx.x * wpb + (threadIdx.x >> 5);
  const size_t chunk = ((total + warps - 1) / warps + 31) & ~(size_t)31;
  beg = gw * chunk;
  end = beg + chunk < total ? beg + chunk : total;
}

__global__ void k_residual_trees(ResidualArgs a) {
  const size_t total = (size_t)a.N * (2 * a.n + a.m);
  const bool ks = a.with_knorm;
  const int nslots = ks ? 4 : 3;
  size_t beg, end;
  warp_rows(total, beg, end);
  TreeAcc acc;
  for (size_t base = beg; base < end; base += 32) {
    const size_t t = base + (threadIdx.x & 31);
    const bool valid = t < end;
    double s = 0, rs = 0, zv = 0, bv = 0;
    int node = 0;
    if (valid) s = fp64_row(a, t, ks, rs, zv, bv, node);
    const unsigned long long r[4] = {dbits_abs(isnan(s) ? INFINITY : s), dbits_abs(zv), dbits_abs(bv),
                                     dbits_abs(rs)};
    acc.add(a, nslots, valid, valid ? a.tree[node] : -1, r);
  }
  acc.flush(a, nslots);
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

// acc += (ah + al) * (xh + xl), keeping the rounding error of ah*xh exactly
__device__ __forceinline__ void ff_fma2(FF& acc, float ah, float al, float xh, float xl) {
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
// acc += a (FP64 constant, split here)
__device__ __forceinline__ void ff_add(FF& acc, double a) {
  float ah, al;
  dsplit(a, ah, al);
  const float s = acc.h + ah;
  const float bb = s - acc.h;
  const float err = (acc.h - (s - bb)) + (ah - bb);
  acc.l += err + al;
  acc.h = s;
}
// acc += (h + l) for an already split operand
__device__ __forceinline__ void ff_add2(FF& acc, float h, float l) {
  const float s = acc.h + h;
  const float bb = s - acc.h;
  const float err = (acc.h - (s - bb)) + (h - bb);
  acc.l += err + l;
  acc.h = s;
}
// Exact float -> double by bit manipulation (no FP64 instruction).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xffu, man = u & 0x7fffffu;
  if (e == 0) {
    if (man == 0) return __longlong_as_double((long long)sign);
    // subnormal float man * 2^-149: leading bit p becomes the implicit bit
    const int p = 31 - __clz(man);
    const unsigned m2 = (man << (23 - p)) & 0x7fffffu;
    const unsigned long long ex = (unsigned long long)(874 + p);   // 1023 - 149 + p
    return __longlong_as_double((long long)(sign | (ex << 52) | ((unsigned long long)m2 << 29)));
  }
  if (e == 0xffu) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | ((unsigned long long)man << 29)));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896) << 52) | ((unsigned long long)man << 29)));
}
// The residual value only feeds an FP32 correction solve and a max-norm: its
// float-float accumulation removes the cancellation, and the final h + l is
// rounded to FP32 and widened exactly.
__device__ __forceinline__ double ff_value(const FF& v) { return f2d_bits(v.h + v.l); }
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

// Split FP64 arrays into (hi, lo) FP32 pairs; up to 9 arrays in one launch.
// Optionally folds |.| maxima of the arrays into maxes[slot] (slot < 0: none).
struct SplitList {
  int count;
  const double* src[9];
  float *hi[9], *lo[9];
  size_t len[9];
  int slot[9];
  unsigned long long* maxes;
};

__global__ void k_split_ff(SplitList L) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int a = 0; a < L.count; ++a) {
    unsigned long long mx = 0;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < L.len[a]; t += stride) {
      const double v = L.src[a][t];
      if (L.hi[a]) {
        float h, l;
        dsplit(v, h, l);
        L.hi[a][t] = h;
        L.lo[a][t] = l;
      }
      const unsigned long long b = abits(v);
      mx = b > mx ? b : mx;
    }
    if (L.slot[a] >= 0) block_maxbits_to(L.maxes + L.slot[a], mx);
  }
}

// Pre-split vectors of the float-float residual (x, u, y as (hi, lo) FP32 pairs).
struct FFArgs {
  const float *xh, *xl, *uh, *ul, *yh, *yl;
};

// acc += a * (xh + xl) with the FP64 matrix entry a split on the fly; returns |a_hi|
__device__ __forceinline__ float ff_fma_d(FF& acc, double a, float xh, float xl) {
  float ah, al;
  dsplit(a, ah, al);
  ff_fma2(acc, ah, al, xh, xl);
  return fabsf(ah);
}

// Row t of eq. (kkt) in float-float arithmetic: matrix entries (FP64, read
// once per use) are split on the fly, the vectors x, u, y come pre-split.
// Returns the residual entry (also stored); rs = the row's FP32 absolute sum
// of KKT entries (when ks); zv, bv = max |z|, |b| of the FP64 entries the row
// owns (only read when want_zb); node = the node of the row.
__device__ __forceinline__ double ff_row(const ResidualArgs& a, const FFArgs& f, size_t t, bool ks, bool want_zb,
                                         float& rs, double& zv, double& bv, int& node) {
  const int n = a.n, m = a.m;
  const size_t nn = (size_t)n * n, nm = (size_t)n * m;
  const size_t rows_x = (size_t)a.N * n, rows_u = (size_t)a.N * m;
  rs = 0.f; zv = 0.0; bv = 0.0;
  if (t < rows_x) {                                   // (kkt-x)
    const int i = (int)(t / n), r = (int)(t - (size_t)i * n);
    node = i;
    const double* Qr = a.Q + (size_t)i * nn + (size_t)r * n;
    const size_t xo = (size_t)i * n;
    FF s{0.f, 0.f};
    ff_add(s, a.q[t]);
    ff_add2(s, -f.yh[t], -f.yl[t]);
    rs = 1.f;
#pragma unroll 4
    for (int b = 0; b < n; ++b) {
      const float aq = ff_fma_d(s, Qr[b], f.xh[xo + b], f.xl[xo + b]);
      if (ks) rs += aq;
    }
    for (int k = a.child_start[i]; k < a.child_start[i + 1]; ++k) {
      const int j = a.child_list[k];
      const double* Aj = a.A + (size_t)j * nn + r;
      const size_t yo = (size_t)j * n;
#pragma unroll 4
      for (int b = 0; b < n; ++b) {
        const float aa = ff_fma_d(s, Aj[(size_t)b * n], f.yh[yo + b], f.yl[yo + b]);
        if (ks) rs += aa;
      }
      if (a.M) {
        const double* Mr = a.M + (size_t)j * nm + (size_t)r * m;
        const size_t uo = (size_t)j * m;
        for (int b = 0; b < m; ++b) {
          const float am = ff_fma_d(s, Mr[b], f.uh[uo + b], f.ul[uo + b]);
          if (ks) rs += am;
        }
      }
    }
    const double out = ff_value(s);
    a.res_x[t] = out;
    if (want_zb) {
      zv = amax(amax(0.0, a.x[t]), a.y[t]);
      bv = fmax(fabs(a.q[t]), fabs(a.c[t]));
    }
    return out;
  }
  if (t < rows_x + rows_u) {                          // (kkt-u)
    const size_t tu = t - rows_x;
    const int i = (int)(tu / m), r = (int)(tu - (size_t)i * m);
    node = i;
    if (a.parent[i] < 0) { a.res_u[tu] = 0.0; return 0.0; }
    const int p = a.parent[i];
    const size_t xo = (size_t)p * n, uo = (size_t)i * m, yo = (size_t)i * n;
    const double* Bc = a.B + (size_t)i * nm + r;
    const double* Rr = a.R + (size_t)i * m * m + (size_t)r * m;
    FF s{0.f, 0.f};
    ff_add(s, a.r[tu]);
    if (a.M) {
      const double* Mc = a.M + (size_t)i * nm + r;
      for (int b = 0; b < n; ++b) {
        const float am = ff_fma_d(s, Mc[(size_t)b * m], f.xh[xo + b], f.xl[xo + b]);
        if (ks) rs += am;
      }
    }
    for (int b = 0; b < m; ++b) {
      const float ar = ff_fma_d(s, Rr[b], f.uh[uo + b], f.ul[uo + b]);
      if (ks) rs += ar;
    }
#pragma unroll 4
    for (int b = 0; b < n; ++b) {
      const float ab = ff_fma_d(s, Bc[(size_t)b * m], f.yh[yo + b], f.yl[yo + b]);
      if (ks) rs += ab;
    }
    const double out = ff_value(s);
    a.res_u[tu] = out;
    if (want_zb) {
      zv = amax(0.0, a.u[tu]);
      bv = fabs(a.r[tu]);
    }
    return out;
  }
  const size_t tc = t - rows_x - rows_u;              // constraint entering i
  const int i = (int)(tc / n), r = (int)(tc - (size_t)i * n);
  node = i;
  const size_t yo = (size_t)i * n;
  FF s{0.f, 0.f};
  ff_add(s, a.c[tc]);
  ff_add2(s, -f.xh[tc], -f.xl[tc]);
  rs = 1.f;
  if (a.Delta && (!a.dflag || a.dflag[i])) {
    const double* Dr = a.Delta + (size_t)i * nn + (size_t)r * n;
#pragma unroll 4
    for (int b = 0; b < n; ++b) {
      const float ad = ff_fma_d(s, Dr[b], -f.yh[yo + b], -f.yl[yo + b]);
      if (ks) rs += ad;
    }
  }
  if (a.parent[i] >= 0) {
    const int p = a.parent[i];
    const size_t xo = (size_t)p * n, uo = (size_t)i * m;
    const double* Ar = a.A + (size_t)i * nn + (size_t)r * n;
    const double* Br = a.B + (size_t)i * nm + (size_t)r * m;
#pragma unroll 4
    for (int b = 0; b < n; ++b) {
      const float aa = ff_fma_d(s, Ar[b], f.xh[xo + b], f.xl[xo + b]);
      if (ks) rs += aa;
    }
    for (int b = 0; b < m; ++b) {
      const float ab = ff_fma_d(s, Br[b], f.uh[uo + b], f.ul[uo + b]);
      if (ks) rs += ab;
    }
  }
  const double out = ff_value(s);
  a.res_c[tc] = out;
  return out;
}

// One tree: ||z|| and ||b|| maxima are formed by the split pass; this kernel
// adds ||res|| and (optionally) the FP32 row sums of ||K||.
__global__ void k_residual_ff(ResidualArgs a, FFArgs f) {
  const size_t total = (size_t)a.N * (2 * a.n + a.m);
  unsigned long long rmax = 0;
  float kmax = 0.f;
  const bool ks = a.with_knorm;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    float rs;
    double zv, bv;
    int node;
    const double out = ff_row(a, f, t, ks, false, rs, zv, bv, node);
    kmax = fmaxf(kmax, rs);
    const unsigned long long ob = abits(out);
    rmax = ob > rmax ? ob : rmax;
  }
  block_maxbits_to(a.maxes + 0, rmax);
  if (ks) block_maxbits_to(a.maxes + 3, abits(f2d_bits(kmax)));
}

// A forest: all four maxima per tree (the split pass folds none).
__global__ void k_residual_ff_trees(ResidualArgs a, FFArgs f) {
  const size_t total = (size_t)a.N * (2 * a.n + a.m);
  const bool ks = a.with_knorm;
  const int nslots = ks ? 4 : 3;
  size_t beg, end;
  warp_rows(total, beg, end);
  TreeAcc acc;
  for (size_t base = beg; base < end; base += 32) {
    const size_t t = base + (threadIdx.x & 31);
    const bool valid = t < end;
    float rs = 0.f;
    double out = 0, zv = 0, bv = 0;
    int node = 0;
    if (valid) out = ff_row(a, f, t, ks, true, rs, zv, bv, node);
    const unsigned long long r[4] = {abits(out), dbits_abs(zv), dbits_abs(bv), abits(f2d_bits(rs))};
    acc.add(a, nslots, valid, valid ? a.tree[node] : -1, r);
  }
  acc.flush(a, nslots);
}

}  // namespace tlqr
