// Warp-cooperative dense algebra on small row-major matrices held in shared
// memory (n, m <= 64).  One warp owns one local operation; every routine is
// called by all 32 lanes of that warp with identical arguments, distributes
// its elements over the lanes and ends with __syncwarp(), which also orders
// the warp's shared- and global-memory accesses.
//
// Factorisations follow the choices of the paper's local algebra: Cholesky for
// the SPD blocks R_e and G_e (Def. 1, Sec. V-C) and LU with partial pivoting
// for the nonsymmetric I + C U, I + C_l P~ and I + Delta P (Lemma 1, Sec. V-C).
#pragma once
#include <cstdint>

#define TLQR_FULL_MASK 0xffffffffu

namespace tlqr {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <typename T> __device__ __forceinline__ T tabs(T v) { return v < T(0) ? -v : v; }
__device__ __forceinline__ bool tfinite(double v) { return isfinite(v); }
__device__ __forceinline__ bool tfinite(float v) { return isfinite(v); }

// dst[0..count) = (T) src[0..count)
template <typename T, typename S>
__device__ __forceinline__ void wload(T* __restrict__ dst, const S* __restrict__ src, int count) {
  for (int e = lane_id(); e < count; e += 32) dst[e] = (T)src[e];
}
template <typename T>
__device__ __forceinline__ void wzero(T* dst, int count) {
  for (int e = lane_id(); e < count; e += 32) dst[e] = T(0);
}
// dst = a + b elementwise (any of them may be global)
template <typename T, typename SA, typename SB>
__device__ __forceinline__ void wadd(T* dst, const SA* a, const SB* b, int count) {
  for (int e = lane_id(); e < count; e += 32) dst[e] = (T)a[e] + (T)b[e];
}
template <typename T>
__device__ __forceinline__ void wadd_identity(T* a, int n, int lda) {
  for (int d = lane_id(); d < n; d += 32) a[d * lda + d] += T(1);
}

// C(r x c) = alpha * op(A) * op(B) [+ Add], op(A)(i,t) = TA ? A[t*lda+i] : A[i*lda+t].
// C must not alias A or B; Add may alias C (same element, read before write).
template <typename T, bool TA, bool TB, typename TC, typename TD>
__device__ __forceinline__ void wgemm(int r, int c, int k, const T* __restrict__ A, int lda,
                                      const T* __restrict__ B, int ldb, TC* C, int ldc, T alpha,
                                      const TD* Add, int ldadd) {
  const int total = r * c;
  for (int e = lane_id(); e < total; e += 32) {
    const int i = e / c, j = e - (e / c) * c;
    T s = T(0);
#pragma unroll 4
    for (int t = 0; t < k; ++t) {
      const T a = TA ? A[t * lda + i] : A[i * lda + t];
      const T b = TB ? B[j * ldb + t] : B[t * ldb + j];
      s = fma(a, b, s);
    }
    T v = alpha * s;
    if (Add) v += (T)Add[i * ldadd + j];
    C[i * ldc + j] = (TC)v;
  }
  __syncwarp();
}

// y(r) = alpha * op(A) x [+ add]; A is r x c (TA: A stored c x r).  One lane per row.
template <typename T, bool TA, typename TY, typename TD>
__device__ __forceinline__ void wgemv(int r, int c, const T* __restrict__ A, int lda,
                                      const T* __restrict__ x, TY* y, T alpha, const TD* add) {
  for (int i = lane_id(); i < r; i += 32) {
    T s = T(0);
    for (int t = 0; t < c; ++t) s = fma(TA ? A[t * lda + i] : A[i * lda + t], x[t], s);
    T v = alpha * s;
    if (add) v += (T)add[i];
    y[i] = (TY)v;
  }
  __syncwarp();
}

// In-place LU with partial pivoting of the n x n matrix a (leading dim lda);
// piv[k] = row exchanged with row k at step k.  Returns false (uniformly across
// the warp) on a zero or nonfinite pivot.
template <typename T>
__device__ bool wlu(T* a, int n, int lda, int* piv) {
  const int lane = lane_id();
  for (int k = 0; k < n; ++k) {
    T best = T(-1);
    int bi = n;
    for (int i = k + lane; i < n; i += 32) {
      const T v = tabs(a[i * lda + k]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const T ob = __shfl_xor_sync(TLQR_FULL_MASK, best, off);
      const int oi = __shfl_xor_sync(TLQR_FULL_MASK, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (!(best > T(0)) || !tfinite(best)) return false;
    if (lane == 0) piv[k] = bi;
    if (bi != k) {
      for (int j = lane; j < n; j += 32) {
        const T t = a[k * lda + j];
        a[k * lda + j] = a[bi * lda + j];
        a[bi * lda + j] = t;
      }
    }
    __syncwarp();
    const T inv = T(1) / a[k * lda + k];
    for (int i = k + 1 + lane; i < n; i += 32) a[i * lda + k] *= inv;
    __syncwarp();
    const int w = n - k - 1;
    for (int e = lane; e < w * w; e += 32) {
      const int i = k + 1 + e / w, j = k + 1 + (e - (e / w) * w);
      a[i * lda + j] = fma(-a[i * lda + k], a[k * lda + j], a[i * lda + j]);
    }
    __syncwarp();
  }
  return true;
}

// Solve (LU) X = B in place; B is n x nrhs with leading dim ldb.
template <typename T>
__device__ void wlu_solve(const T* lu, int n, int lda, const int* piv, T* b, int nrhs, int ldb) {
  const int lane = lane_id();
  for (int j = lane; j < nrhs; j += 32)
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k) { const T t = b[k * ldb + j]; b[k * ldb + j] = b[p * ldb + j]; b[p * ldb + j] = t; }
    }
  __syncwarp();
  for (int k = 0; k + 1 < n; ++k) {                       // unit lower
    const int w = n - k - 1;
    for (int e = lane; e < w * nrhs; e += 32) {
      const int i = k + 1 + e / nrhs, j = e - (e / nrhs) * nrhs;
      b[i * ldb + j] = fma(-lu[i * lda + k], b[k * ldb + j], b[i * ldb + j]);
    }
    __syncwarp();
  }
  for (int k = n - 1; k >= 0; --k) {                      // upper
    const T inv = T(1) / lu[k * lda + k];
    for (int j = lane; j < nrhs; j += 32) b[k * ldb + j] *= inv;
    __syncwarp();
    for (int e = lane; e < k * nrhs; e += 32) {
      const int i = e / nrhs, j = e - (e / nrhs) * nrhs;
      b[i * ldb + j] = fma(-lu[i * lda + k], b[k * ldb + j], b[i * ldb + j]);
    }
    __syncwarp();
  }
}

// In-place lower Cholesky (the strict upper part is left as is).  Returns false
// on a nonpositive or nonfinite pivot.
template <typename T>
__device__ bool wchol(T* a, int m, int lda) {
  const int lane = lane_id();
  for (int k = 0; k < m; ++k) {
    const T d = a[k * lda + k];
    if (!(d > T(0)) || !tfinite(d)) return false;
    const T s = sqrt(d);
    const T inv = T(1) / s;
    __syncwarp();
    if (lane == 0) a[k * lda + k] = s;
    for (int i = k + 1 + lane; i < m; i += 32) a[i * lda + k] *= inv;
    __syncwarp();
    const int w = m - k - 1;
    for (int e = lane; e < w * w; e += 32) {
      const int i = k + 1 + e / w, j = k + 1 + (e - (e / w) * w);
      if (j <= i) a[i * lda + j] = fma(-a[i * lda + k], a[j * lda + k], a[i * lda + j]);
    }
    __syncwarp();
  }
  return true;
}

// ------------------------------------------------------------ FP64 fallback
// In mixed precision the SPD blocks R_e and G_e = R_e + B_e^T W B_e are
// factored in FP32 first.  An FP32 Cholesky has a backward error of about
// eps_32 ||S||, i.e. a relative error ~ kappa(S) eps_32 in the directions of
// the small eigenvalues: beyond kappa ~ 1e5 the factors stop being a usable
// preconditioner for the FP64 refinement (and the factorisation may break
// down).  Such blocks are refactored in FP64 and the FP64 factor L is rounded
// to FP32; the rounding perturbs the preconditioned operator only by
// ~ kappa(L) eps_32 = sqrt(kappa(S)) eps_32, so FP32 triangular solves with the
// rounded L stay accurate to ~1e-3 up to kappa(S) ~ 1e8.
// A block counts as ill-conditioned when the FP32 factorisation fails or its
// largest diagonal entry of L exceeds kCholRatio times its smallest (pivot
// ratio > 1e4, a lower bound on kappa(S)).
constexpr float kCholRatio = 100.0f;

// In-place Cholesky of an m x m SPD matrix (row-major, lda) in FP64 by one
// thread, left-looking (row by row); the lower triangle receives L.  False
// when a pivot is not positive and finite.
// Not inlined: it runs rarely, on shared memory, and must not add registers to
// the kernels that call it.
__device__ __noinline__ bool chol64_serial(double* a, int m, int lda) {
#pragma unroll 1
  for (int k = 0; k < m; ++k) {
#pragma unroll 1
    for (int i = 0; i <= k; ++i) {
      double v = a[k * lda + i];
#pragma unroll 1
      for (int t = 0; t < i; ++t) v = fma(-a[k * lda + t], a[i * lda + t], v);
      if (i < k) {
        a[k * lda + i] = v / a[i * lda + i];
      } else {
        if (!(v > 0.0) || !isfinite(v)) return false;
        a[k * lda + k] = sqrt(v);
      }
    }
  }
  return true;
}

// Warp-cooperative Cholesky with the FP64 fallback.  On entry a (working
// precision) holds S = S64 + S32 rounded, where s64 (global, FP64, m x m
// row-major) and s32 (shared, working precision, lds; may be null) are the
// two parts of S kept separately; scratch holds m*m doubles of shared memory.
// On return a holds L (in the working precision).  False when S is not
// numerically PD even in FP64.
template <typename T>
__device__ bool wchol_checked(T* a, int m, int lda, const double* s64, const T* s32, int lds, double* scratch) {
  bool ok = wchol(a, m, lda);
  if constexpr (sizeof(T) == 8) {
    return ok;
  } else {
    float dmin = INFINITY, dmax = 0.f;
    if (ok) {
      for (int k = lane_id(); k < m; k += 32) {
        const float d = (float)a[k * lda + k];
        dmin = fminf(dmin, d);
        dmax = fmaxf(dmax, d);
      }
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        dmin = fminf(dmin, __shfl_xor_sync(TLQR_FULL_MASK, dmin, off));
        dmax = fmaxf(dmax, __shfl_xor_sync(TLQR_FULL_MASK, dmax, off));
      }
    }
    if (ok && dmax <= kCholRatio * dmin) return true;
    for (int e = lane_id(); e < m * m; e += 32) {
      const int i = e / m, j = e - (e / m) * m;
      scratch[e] = s64[e] + (s32 ? (double)s32[i * lds + j] : 0.0);
    }
    __syncwarp();
    bool ok64 = true;
    if (lane_id() == 0) ok64 = chol64_serial(scratch, m, m);
    ok64 = __shfl_sync(TLQR_FULL_MASK, ok64, 0);
    __syncwarp();
    for (int e = lane_id(); e < m * m; e += 32) {
      const int i = e / m, j = e - (e / m) * m;
      if (j <= i) a[i * lda + j] = (T)scratch[e];
    }
    __syncwarp();
    return ok64;
  }
}

// Solve L L^T X = B in place (L from wchol); B is m x nrhs, leading dim ldb.
template <typename T>
__device__ void wchol_solve(const T* l, int m, int lda, T* b, int nrhs, int ldb) {
  const int lane = lane_id();
  for (int k = 0; k < m; ++k) {                          // L w = b
    const T inv = T(1) / l[k * lda + k];
    for (int j = lane; j < nrhs; j += 32) b[k * ldb + j] *= inv;
    __syncwarp();
    const int w = m - k - 1;
    for (int e = lane; e < w * nrhs; e += 32) {
      const int i = k + 1 + e / nrhs, j = e - (e / nrhs) * nrhs;
      b[i * ldb + j] = fma(-l[i * lda + k], b[k * ldb + j], b[i * ldb + j]);
    }
    __syncwarp();
  }
  for (int k = m - 1; k >= 0; --k) {                     // L^T x = w
    const T inv = T(1) / l[k * lda + k];
    for (int j = lane; j < nrhs; j += 32) b[k * ldb + j] *= inv;
    __syncwarp();
    for (int e = lane; e < k * nrhs; e += 32) {
      const int i = e / nrhs, j = e - (e / nrhs) * nrhs;
      b[i * ldb + j] = fma(-l[k * lda + i], b[k * ldb + j], b[i * ldb + j]);
    }
    __syncwarp();
  }
}

// Warp-wide OR of a predicate.
__device__ __forceinline__ bool wany(bool p) { return __any_sync(TLQR_FULL_MASK, p); }

}  // namespace tlqr
