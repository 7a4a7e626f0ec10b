// Compile-time-dimension kernels for the n x n local operations of the
// contraction: rake fold, compression, reconstruction, transition composition,
// and the O(n^2) right-hand-side passes.  Same arithmetic as kernels.cuh
// (which handles any n at run time); used when n is one of the instantiated
// sizes.
//
// Mapping: a group of G lanes (G = smallest power of two >= n, at most 32)
// performs one operation, so a warp runs 32 / G operations side by side.  Lane
// r of a group holds row r of the block it is working on in registers.  The
// right operand of a product sits in shared memory (row stride LD, rows 16-byte
// aligned) and is read as whole 16-byte vectors that every lane of the group
// reads at the same address (broadcast): a lane performs W = 16 / sizeof(T)
// FMAs per shared-memory load.  The linear solves with S = I + C P~ and
// F = I + Delta P are Gauss-Jordan eliminations with partial pivoting that keep
// the rows where they are (implicit pivoting): the pivot is found with one
// unsigned-max reduction over the group and its row is broadcast through
// shared memory.  Loops over n are fully unrolled, so
// all register indexing is static.  At n = 16 and n = 32 in FP32 the block
// products run on the tensor cores instead (mma32.cuh); the eliminations stay
// on the FP32 pipe.
#pragma once
#include <cstdint>
#include <type_traits>

#include "kernels.cuh"
#include "mma32.cuh"

namespace tlqr {
namespace fx {

template <typename T> struct Vec;
template <> struct Vec<float> { using V = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using V = double2; static constexpr int W = 2; };

template <typename T, int N>
struct D {
  static constexpr int G = N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32;
  static constexpr int W = Vec<T>::W;
  static constexpr int NV = (N + W - 1) / W;          // vectors per row
  // padded row stride (elements): a whole number of 16-byte vectors, and an odd
  // one, so that the rows owned by consecutive lanes start in different
  // shared-memory bank quads (conflict-free 16-byte row accesses)
  static constexpr int LD = (NV % 2 == 1 ? NV : NV + 1) * W;
  static constexpr int OPS = 32 / G;                   // operations per warp
  static constexpr int MAT = N * LD;                   // elements of one staged matrix
};

// n = 16 (two operations per warp, one 16 x 16 product per half warp) and
// n = 32 (one operation per warp) in FP32: the n x n block products run on the
// tensor cores (3xTF32 mma.sync, mma32.cuh); the Gauss-Jordan solves stay on
// the FP32 pipe.
template <typename T, int N>
constexpr bool kTensorCores = std::is_same<T, float>::value && (N == 32 || N == 16);

template <typename T> __device__ __forceinline__ T vget(const typename Vec<T>::V& v, int i);
template <> __device__ __forceinline__ float vget<float>(const float4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
template <> __device__ __forceinline__ double vget<double>(const double2& v, int i) { return i == 0 ? v.x : v.y; }

__device__ __forceinline__ void vset(float4& v, int i, float x) {
  if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
}
__device__ __forceinline__ void vset(double2& v, int i, double x) { if (i == 0) v.x = x; else v.y = x; }

// Group context: lane within the group, group id within the block, validity.
struct Grp {
  int gl, gid;
  bool valid;
};

template <typename T, int N>
__device__ __forceinline__ Grp group_of(int count, int* op) {
  constexpr int G = D<T, N>::G, OPS = D<T, N>::OPS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Grp g;
  g.gl = lane & (G - 1);
  g.gid = warp * OPS + lane / G;
  const int o = blockIdx.x * (blockDim.x / G) + g.gid;
  g.valid = o < count;
  *op = g.valid ? o : count - 1;           // invalid groups shadow the last operation, store nothing
  return g;
}

// Copy ROWS x COLS contiguous global elements into shared rows of stride LDS.
template <typename T, int ROWS, int COLS, int LDS, int G, typename S>
__device__ __forceinline__ void gload(T* dst, const S* src, int gl) {
#pragma unroll
  for (int e = gl; e < ROWS * COLS; e += G) {
    const int r = e / COLS, c = e - (e / COLS) * COLS;
    dst[r * LDS + c] = (T)src[e];
  }
}
// Copy shared rows to contiguous global memory.
template <typename T, int ROWS, int COLS, int LDS, int G, typename S>
__device__ __forceinline__ void gstore(T* dst, const S* src, int gl) {
#pragma unroll
  for (int e = gl; e < ROWS * COLS; e += G) {
    const int r = e / COLS, c = e - (e / COLS) * COLS;
    dst[e] = (T)src[r * LDS + c];
  }
}

// a[0..N) <- shared row (vector loads)
template <typename T, int N>
__device__ __forceinline__ void row_load(T (&a)[N], const T* row) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
#pragma unroll
  for (int q = 0; q < D<T, N>::NV; ++q) {
    const V v = reinterpret_cast<const V*>(row)[q];
#pragma unroll
    for (int i = 0; i < W; ++i)
      if (q * W + i < N) a[q * W + i] = vget<T>(v, i);
  }
}
template <typename T, int N>
__device__ __forceinline__ void row_store(T* row, const T (&a)[N]) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
#pragma unroll
  for (int q = 0; q < D<T, N>::NV; ++q) {
    V v;
#pragma unroll
    for (int i = 0; i < W; ++i) vset(v, i, q * W + i < N ? a[q * W + i] : T(0));
    reinterpret_cast<V*>(row)[q] = v;
  }
}

// A length-N row of a node block in global memory (row-major, rows of N
// elements, blocks 256-byte aligned): 16-byte vector accesses when a row is a
// whole number of vectors, else element by element.
template <typename T, int N>
__device__ __forceinline__ void grow_load(T (&a)[N], const T* row) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
  if constexpr ((N * sizeof(T)) % 16 == 0) {
#pragma unroll
    for (int q = 0; q < N / W; ++q) {
      const V v = reinterpret_cast<const V*>(row)[q];
#pragma unroll
      for (int i = 0; i < W; ++i) a[q * W + i] = vget<T>(v, i);
    }
  } else {
#pragma unroll
    for (int c = 0; c < N; ++c) a[c] = row[c];
  }
}
template <typename T, int N>
__device__ __forceinline__ void grow_store(T* row, const T (&a)[N]) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
  if constexpr ((N * sizeof(T)) % 16 == 0) {
#pragma unroll
    for (int q = 0; q < N / W; ++q) {
      V v;
#pragma unroll
      for (int i = 0; i < W; ++i) vset(v, i, a[q * W + i]);
      reinterpret_cast<V*>(row)[q] = v;
    }
  } else {
#pragma unroll
    for (int c = 0; c < N; ++c) row[c] = a[c];
  }
}

// c[0..C) += sum_t a[t] * B[t][0..C)   (B in shared memory, row stride LDB, broadcast rows)
template <typename T, int K, int C, int LDB>
__device__ __forceinline__ void row_mm(T (&c)[C], const T (&a)[K], const T* B) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
#pragma unroll
  for (int t = 0; t < K; ++t) {
#pragma unroll
    for (int q = 0; q < (C + W - 1) / W; ++q) {
      const V v = reinterpret_cast<const V*>(B + t * LDB)[q];
#pragma unroll
      for (int i = 0; i < W; ++i)
        if (q * W + i < C) c[q * W + i] = fma(a[t], vget<T>(v, i), c[q * W + i]);
    }
  }
}
// c[0..C) += sum_t A[t][r] * B[t][0..C)   (column r of A from shared memory)
template <typename T, int K, int C, int LDA, int LDB>
__device__ __forceinline__ void col_mm(T (&c)[C], const T* A, int r, const T* B) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const T at = A[t * LDA + r];
#pragma unroll
    for (int q = 0; q < (C + W - 1) / W; ++q) {
      const V v = reinterpret_cast<const V*>(B + t * LDB)[q];
#pragma unroll
      for (int i = 0; i < W; ++i)
        if (q * W + i < C) c[q * W + i] = fma(at, vget<T>(v, i), c[q * W + i]);
    }
  }
}
// c[j] += sum_t a[t] * B[j][t]  for j < C  (rows of B from shared memory: a * B^T)
template <typename T, int K, int C, int LDB>
__device__ __forceinline__ void row_mmT(T (&c)[C], const T (&a)[K], const T* B) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    T s = c[j];
#pragma unroll
    for (int q = 0; q < (K + W - 1) / W; ++q) {
      const V v = reinterpret_cast<const V*>(B + j * LDB)[q];
#pragma unroll
      for (int i = 0; i < W; ++i)
        if (q * W + i < K) s = fma(a[q * W + i], vget<T>(v, i), s);
    }
    c[j] = s;
  }
}

// Pivot search key of a group lane: the bits of |v| (monotone for IEEE
// numbers of one sign; NaN maps to +Inf so a NaN column is picked and then
// rejected) with the low log2(G) bits replaced by G - 1 - gl, so that one
// unsigned max over the group returns the largest |v| and, among values
// equal in the remaining bits, the lowest lane.  Dropping those low mantissa
// bits lets the chosen pivot be up to 2^-18 (FP32) or 2^-15 (FP64, high word)
// below the true maximum in relative terms, which partial pivoting tolerates.
template <typename T> __device__ __forceinline__ unsigned pivot_bits(T v);
template <> __device__ __forceinline__ unsigned pivot_bits<float>(float v) {
  const unsigned u = __float_as_uint(v) & 0x7fffffffu;
  return u > 0x7f800000u ? 0x7f800000u : u;
}
template <> __device__ __forceinline__ unsigned pivot_bits<double>(double v) {
  const unsigned hi = (unsigned)__double2hiint(v) & 0x7fffffffu, lo = (unsigned)__double2loint(v);
  return (hi > 0x7ff00000u || (hi == 0x7ff00000u && lo != 0u)) ? 0x7ff00000u : hi;
}

// Unsigned max over the G lanes of each group of a warp.  Whole warp: one
// redux.sync.  Half warps: one full-warp redux per half (the other half
// contributes 0).  Smaller groups: a shuffle butterfly.  Called by all lanes.
template <int G>
__device__ __forceinline__ unsigned group_umax(unsigned key) {
  if constexpr (G == 32) {
    return __reduce_max_sync(TLQR_FULL_MASK, key);
  } else if constexpr (G == 16) {
    const bool upper = (threadIdx.x & 16) != 0;
    const unsigned lo = __reduce_max_sync(TLQR_FULL_MASK, upper ? 0u : key);
    const unsigned hi = __reduce_max_sync(TLQR_FULL_MASK, upper ? key : 0u);
    return upper ? hi : lo;
  } else {
#pragma unroll
    for (int off = G / 2; off; off >>= 1) key = max(key, __shfl_xor_sync(TLQR_FULL_MASK, key, off, G));
    return key;
  }
}

// Shared broadcast buffer of ggj: two rows (double buffering) of the pivot
// row of S (N entries, padded to whole vectors), of B (R entries, padded) and
// one vector holding 1 / pivot.
template <typename T, int N, int R>
struct GjBuf {
  static constexpr int W = Vec<T>::W;
  static constexpr int NP = (N + W - 1) / W * W, RP = (R + W - 1) / W * W;
  static constexpr int ROW = NP + RP + W;
  static constexpr int elems = 2 * ROW;
};

// Solve S X = B by Gauss-Jordan elimination with partial pivoting, for one
// group.  Lane gl < N holds row gl of S in a[] and row gl of B in b[]; rows
// stay in their lanes (implicit pivoting).  At step k the undone lane with the
// largest |a[k]| (group_umax of pivot keys) writes its row, unscaled, and
// 1 / a[k] to the shared buffer; every other lane, pivots of earlier steps
// included, subtracts l = a[k] / pivot times that row from columns > k of S
// and from all of B.  After N steps the lane that was pivot k holds row k of
// X once it divides its B row by its own pivot: on return lane gl holds row
// kpos of X in b[].  N serial steps, against 3N for an LU followed by forward
// and backward substitution; every lane issues the same N^2/2 + N R FMAs as
// there (a lane owns a whole row, so the triangular sweeps saved no per-lane
// work).  Double-buffered broadcast rows need one __syncwarp per step.
// bc: GjBuf<T, N, R>::elems shared elements of this group, 16-byte aligned.
// Returns false (uniformly in the group) on a zero or nonfinite pivot.
// ratio (the same in every lane of the group): a lower bound on the condition
// number of S, the larger of (largest |pivot|) / (smallest |pivot|) and
// ||S||_inf ||X||_inf / ||B||_inf (since ||X|| <= ||S^{-1}|| ||B||).  The pivot
// ratio alone can stay far below kappa(S) when S = I + (low-rank, large).
template <typename T, int N, int G, int R>
__device__ __forceinline__ bool ggj(T (&a)[N], T (&b)[R], int gl, T* bc, int& kpos, float& ratio) {
  using Bf = GjBuf<T, N, R>;
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
  bool done = gl >= N;
  kpos = N;
  bool ok = true;
  T myinv = T(1);
  T imin = T(INFINITY), imax = T(0);
  // row sums of |S| and |B| (this lane's row; FP32 kernels only, where the
  // estimate decides on a re-solve)
  float s_norm = 0.f, b_norm = 0.f;
  if constexpr (sizeof(T) == 4) {
    float sn = 0.f, bn = 0.f;
    if (gl < N) {
#pragma unroll
      for (int c = 0; c < N; ++c) sn += fabsf(a[c]);
#pragma unroll
      for (int c = 0; c < R; ++c) bn += fabsf(b[c]);
    }
    s_norm = __uint_as_float(group_umax<G>(__float_as_uint(sn)));
    b_norm = __uint_as_float(group_umax<G>(__float_as_uint(bn)));
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T* row = bc + (k & 1) * Bf::ROW;
    const unsigned key = done ? 0u : ((pivot_bits<T>(a[k]) & ~unsigned(G - 1)) | unsigned(G - 1 - gl));
    const unsigned mx = group_umax<G>(key);
    const int p = G - 1 - (int)(mx & unsigned(G - 1));
    if (gl == p) {
      kpos = k;
      done = true;
      myinv = T(1) / a[k];
#pragma unroll
      for (int q = k / W; q < Bf::NP / W; ++q) {
        V v;
#pragma unroll
        for (int i = 0; i < W; ++i) vset(v, i, q * W + i < N ? a[q * W + i] : T(0));
        reinterpret_cast<V*>(row)[q] = v;
      }
#pragma unroll
      for (int q = 0; q < Bf::RP / W; ++q) {
        V v;
#pragma unroll
        for (int i = 0; i < W; ++i) vset(v, i, q * W + i < R ? b[q * W + i] : T(0));
        reinterpret_cast<V*>(row + Bf::NP)[q] = v;
      }
      row[Bf::NP + Bf::RP] = myinv;
    }
    __syncwarp();
    const T inv = row[Bf::NP + Bf::RP];
    ok = ok && tfinite(inv) && inv != T(0);
    imin = fmin(imin, fabs(inv));
    imax = fmax(imax, fabs(inv));
    if (gl != p && gl < N) {
      const T l = a[k] * inv;
#pragma unroll
      for (int q = (k + 1) / W; q < Bf::NP / W; ++q) {
        const V v = reinterpret_cast<const V*>(row)[q];
#pragma unroll
        for (int i = 0; i < W; ++i)
          if (q * W + i > k && q * W + i < N) a[q * W + i] = fma(-l, vget<T>(v, i), a[q * W + i]);
      }
#pragma unroll
      for (int q = 0; q < Bf::RP / W; ++q) {
        const V v = reinterpret_cast<const V*>(row + Bf::NP)[q];
#pragma unroll
        for (int i = 0; i < W; ++i)
          if (q * W + i < R) b[q * W + i] = fma(-l, vget<T>(v, i), b[q * W + i]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < R; ++c) b[c] *= myinv;
  float est = 0.f;
  if constexpr (sizeof(T) == 4) {
    float xn = 0.f;
    if (gl < N) {
#pragma unroll
      for (int c = 0; c < R; ++c) xn += fabsf(b[c]);
    }
    const float x_norm = __uint_as_float(group_umax<G>(__float_as_uint(xn)));
    est = b_norm > 0.f ? s_norm * x_norm / b_norm : 0.f;
  }
  __syncwarp();
  ratio = fmaxf((float)(imax / imin), est);
  return ok;
}
template <typename T, int N, int G, int R>
__device__ __forceinline__ bool ggj(T (&a)[N], T (&b)[R], int gl, T* bc, int& kpos) {
  float ratio;
  return ggj<T, N, G, R>(a, b, gl, bc, kpos, ratio);
}

// ---------------------------------------------------------------- FP64 re-solves
// An FP32 elimination whose pivots span more than kSolveRatio (a lower bound
// on the condition number of S = I + C P~, I + C U or F = I + Delta P) has
// lost about log10(ratio) of FP32's seven digits.  Such a group solves the
// system again in FP64: S and the right-hand side are formed in FP64 from the
// operands (FP32 workspace blocks, FP64 problem data), written to a slot of a
// global scratch (one slot per re-solve of a factorisation, handed out by an
// atomic ticket), eliminated there by the group's lanes, and the solution is
// rounded to FP32.  When the slots run out the FP32 solution stands.  The
// functions below are not inlined: they run rarely and must not add registers
// to the kernels that call them.
constexpr float kSolveRatio = 1e4f;

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
}

// A slot for this group (leader takes the ticket), or null when none is left.
template <int G>
__device__ __forceinline__ double* redo_slot(int* count, int cap, double* scratch, size_t slot, int gl) {
  int t = 0;
  if (gl == 0) t = atomicAdd(count, 1);
  t = __shfl_sync(group_mask<G>(), t, 0, G);
  return t < cap ? scratch + (size_t)t * slot : nullptr;
}

// Gauss-Jordan elimination with partial pivoting of a (n x n, row stride lda)
// against b (n x nb, row stride ldb) in global memory by the G lanes of a
// group, rows kept in place (lane gl < n owns row gl).  On return lane gl's
// row of b holds row *kpos of X = a^{-1} b.  False on a zero or nonfinite pivot.
template <int G>
__device__ __forceinline__ bool gj64_rows(double* a, int lda, double* b, int ldb, int n, int nb, int gl, int& kpos) {
  const unsigned mask = group_mask<G>();
  bool done = gl >= n, ok = true;
  int kp = n;
  double myinv = 1.0;
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    double best = done ? -1.0 : fabs(a[gl * lda + k]);
    if (isnan(best)) best = INFINITY;
    int bl = gl;
#pragma unroll
    for (int off = G / 2; off; off >>= 1) {
      const double ov = __shfl_xor_sync(mask, best, off, G);
      const int ol = __shfl_xor_sync(mask, bl, off, G);
      if (ov > best || (ov == best && ol < bl)) { best = ov; bl = ol; }
    }
    if (gl == bl) {
      kp = k;
      done = true;
      myinv = 1.0 / a[gl * lda + k];
    }
    const double pinv = __shfl_sync(mask, myinv, bl, G);
    ok = ok && isfinite(pinv) && pinv != 0.0;
    __syncwarp(mask);
    if (gl != bl && gl < n) {
      const double l = a[gl * lda + k] * pinv;
#pragma unroll 1
      for (int c = k + 1; c < n; ++c) a[gl * lda + c] = fma(-l, a[bl * lda + c], a[gl * lda + c]);
#pragma unroll 1
      for (int c = 0; c < nb; ++c) b[gl * ldb + c] = fma(-l, b[bl * ldb + c], b[gl * ldb + c]);
    }
    __syncwarp(mask);
  }
  if (gl < n) {
#pragma unroll 1
    for (int c = 0; c < nb; ++c) b[gl * ldb + c] *= myinv;
  }
  __syncwarp(mask);
  kpos = kp;
  return ok;
}

// Forms rows gl < N of the system in the slot, eliminates it, writes the
// solution X, rounded to FP32, into the shared rows `dst` (row stride ldd)
// where the FP32 elimination would have put it, and forms in FP64 the product
// with the right factor that follows every one of these solves -- R X -- whose
// large-times-small terms (R large along the directions where X is small) FP32
// cannot resolve, writing it rounded into `wdst` (row stride ldwd):
//   kind 0 (rake, reconstruction): S = I + L R, B = B1, X = S^{-1} A, R X = U Y
//   kind 1 (compression):          S = I + L R, B = [B1 | L B2^T] (the second
//                                  block of X goes to column col2), R X1 = P~ Y1
//   kind 2 (local factor):         S = I + L64 R, B = I, X = F^{-1}, R X = P F^{-1}
// L, R, B1, B2: FP32 rows (shared or global memory, leading dimensions);
// L64: FP64 rows (problem data).  Slot layout: S (N x N), then B (N x nb);
// wdst may alias R (the product is staged in the slot first).
enum : int { RS_TAU = 0, RS_COMPRESS = 1, RS_LOCAL = 2 };
template <int N, int G>
__device__ __noinline__ bool resolve64(double* sc, int kind, const float* L, int ldl, const double* L64,
                                       const float* R, int ldr, const float* B1, int ldb1, const float* B2,
                                       int ldb2, float* dst, int ldd, int col2, float* wdst, int ldwd, int gl) {
  const unsigned mask = group_mask<G>();
  const int nb = kind == RS_COMPRESS ? 2 * N : N;
  double *a = sc, *b = sc + N * N;
  if (gl < N) {
#pragma unroll 1
    for (int c = 0; c < N; ++c) {
      double v = c == gl ? 1.0 : 0.0;
#pragma unroll 1
      for (int t = 0; t < N; ++t) {
        const double l = kind == RS_LOCAL ? L64[gl * ldl + t] : (double)L[gl * ldl + t];
        v = fma(l, (double)R[t * ldr + c], v);
      }
      a[gl * N + c] = v;
    }
#pragma unroll 1
    for (int c = 0; c < N; ++c) b[gl * nb + c] = kind == RS_LOCAL ? (c == gl ? 1.0 : 0.0) : (double)B1[gl * ldb1 + c];
    if (kind == RS_COMPRESS) {
#pragma unroll 1
      for (int c = 0; c < N; ++c) {
        double v = 0.0;
#pragma unroll 1
        for (int t = 0; t < N; ++t) v = fma((double)L[gl * ldl + t], (double)B2[c * ldb2 + t], v);
        b[gl * nb + N + c] = v;
      }
    }
  }
  __syncwarp(mask);
  int kp;
  const bool ok = gj64_rows<G>(a, N, b, nb, N, nb, gl, kp);
  // rows of X by index (first N columns) into the slot's S block, rounded X into dst
  if (gl < N) {
#pragma unroll 1
    for (int c = 0; c < N; ++c) {
      a[kp * N + c] = b[gl * nb + c];
      dst[kp * ldd + c] = (float)b[gl * nb + c];
    }
    if (kind == RS_COMPRESS) {
#pragma unroll 1
      for (int c = 0; c < N; ++c) dst[kp * ldd + col2 + c] = (float)b[gl * nb + N + c];
    }
  }
  __syncwarp(mask);
  // row gl of R X in FP64 (into the lane's own row of the B block), then rounded into wdst
  if (gl < N) {
#pragma unroll 1
    for (int c = 0; c < N; ++c) {
      double v = 0.0;
#pragma unroll 1
      for (int t = 0; t < N; ++t) v = fma((double)R[gl * ldr + t], a[t * N + c], v);
      b[gl * nb + c] = v;
    }
  }
  __syncwarp(mask);
  if (gl < N) {
#pragma unroll 1
    for (int c = 0; c < N; ++c) wdst[gl * ldwd + c] = (float)b[gl * nb + c];
  }
  __syncwarp(mask);
  return ok;
}

template <typename T, int N>
__device__ __forceinline__ void zero(T (&a)[N]) {
#pragma unroll
  for (int j = 0; j < N; ++j) a[j] = T(0);
}

// ---------------------------------------------------------------- tau
// out = P + A^T U (I + C U)^{-1} A  (eq. terminal-fold) for one group.
// sm (group): U, A, Y matrices + the Gauss-Jordan broadcast rows.
template <typename T, int N>
struct TauSmem {
  // U, A, Y; on the tensor-core path A stays in global memory (fewer bytes per
  // warp, more resident warps)
  static constexpr int mats = kTensorCores<T, N> ? 2 : 3;
  static constexpr int elems = mats * D<T, N>::MAT + GjBuf<T, N, N>::elems;
  static constexpr int bytes = ((elems * (int)sizeof(T) + 15) / 16) * 16;
};

// Tensor-core version (n = 16, 32, FP32): U and C staged, C U on the tensor
// cores, A read from global memory twice -- rows for the elimination's
// right-hand side and as the transposed left operand of the last product -- so
// that a warp holds two staged matrices instead of three.
template <typename T, int N>
__device__ __forceinline__ bool tau_group_tc(const Ws<T>& w, const Grp& g, const T* Ug, const T* Ag, const T* Cg,
                                             const T* Pg, T* out, T* sm) {
  using Dm = D<T, N>;
  constexpr int G = Dm::G, LD = Dm::LD, MAT = Dm::MAT;
  T *sU = sm, *sY = sm + MAT, *bc = sm + 2 * MAT;
  gload<T, N, N, LD, G>(sU, Ug, g.gl);
  gload<T, N, N, LD, G>(sY, Cg, g.gl);      // C staged in sY
  __syncwarp();
  const int r = g.gl < N ? g.gl : 0;
  T x[N], b[N];
  tc::gemm<N, false, false>(sY, LD, sU, LD, nullptr, 0, sY, LD, true);   // C U over C
  row_load<T, N>(x, sY + r * LD);
#pragma unroll
  for (int c = 0; c < N; ++c) x[c] += (c == r) ? T(1) : T(0);
  grow_load<T, N>(b, Ag + r * N);               // row r of A (right-hand side)
  __syncwarp();
  int kpos;
  float pr;
  bool ok = ggj<T, N, G, N>(x, b, g.gl, bc, kpos, pr);   // Y = (I + C U)^{-1} A, row kpos in b
  bool stored = false;
  if (w.redo_count && g.valid && !(pr <= kSolveRatio)) {
    if (double* sc = redo_slot<G>(w.redo_count, w.redo_cap, w.redo_scratch, w.redo_slot, g.gl)) {
      ok = resolve64<N, G>(sc, RS_TAU, Cg, N, nullptr, sU, LD, Ag, N, nullptr, 0, sY, LD, 0, sU, LD, g.gl);
      stored = true;                            // Y in sY and Z = U Y (FP64) in sU
    }
  }
  if (!stored && g.gl < N) row_store<T, N>(sY + kpos * LD, b);
  __syncwarp();
  tc::gemm<N, false, false>(sU, LD, sY, LD, nullptr, 0, sU, LD, !stored);   // Z = U Y over U
  tc::gemm<N, true, false>(Ag, N, sU, LD, Pg, N, out, N, g.valid);      // P + A^T Z
  return ok;
}

template <typename T, int N>
__device__ __forceinline__ bool tau_group(const Ws<T>& w, const Grp& g, const T* Ug, const T* Ag, const T* Cg,
                                          const T* Pg, T* out, T* sm) {
  if constexpr (kTensorCores<T, N>) return tau_group_tc<T, N>(w, g, Ug, Ag, Cg, Pg, out, sm);
  using Dm = D<T, N>;
  constexpr int G = Dm::G, LD = Dm::LD, MAT = Dm::MAT;
  T *sU = sm, *sA = sm + MAT, *sY = sm + 2 * MAT, *bc = sm + 3 * MAT;
  gload<T, N, N, LD, G>(sU, Ug, g.gl);
  gload<T, N, N, LD, G>(sA, Ag, g.gl);
  gload<T, N, N, LD, G>(sY, Cg, g.gl);      // C staged in sY
  __syncwarp();
  const int r = g.gl < N ? g.gl : 0;
  T x[N], b[N];
  {
    T crow[N];
    row_load<T, N>(crow, sY + r * LD);
    zero(x);
    row_mm<T, N, N, LD>(x, crow, sU);           // row r of C U
#pragma unroll
    for (int c = 0; c < N; ++c) x[c] += (c == r) ? T(1) : T(0);
  }
  row_load<T, N>(b, sA + r * LD);               // row r of A (right-hand side)
  __syncwarp();
  int kpos;
  float pr;
  bool ok = ggj<T, N, G, N>(x, b, g.gl, bc, kpos, pr);   // Y = (I + C U)^{-1} A, row kpos in b
  bool stored = false;
  if constexpr (sizeof(T) == 4) {
    if (w.redo_count && g.valid && !(pr <= kSolveRatio)) {
      if (double* sc = redo_slot<G>(w.redo_count, w.redo_cap, w.redo_scratch, w.redo_slot, g.gl)) {
        ok = resolve64<N, G>(sc, RS_TAU, Cg, N, nullptr, sU, LD, sA, LD, nullptr, 0, sY, LD, 0, sU, LD, g.gl);
        stored = true;                          // Y in sY and Z = U Y (FP64) in sU
      }
    }
  }
  if (!stored && g.gl < N) row_store<T, N>(sY + kpos * LD, b);
  __syncwarp();
  T z[N];
  {
    T urow[N];
    row_load<T, N>(urow, sU + r * LD);
    zero(z);
    row_mm<T, N, N, LD>(z, urow, sY);           // row r of Z = U Y
  }
  __syncwarp();
  if (!stored && g.gl < N) row_store<T, N>(sU + r * LD, z); // Z over U
  __syncwarp();
  T o[N];
  grow_load<T, N>(o, Pg + r * N);
  col_mm<T, N, N, LD, LD>(o, sA, r, sU);        // P + A^T Z
  if (g.valid && g.gl < N) grow_store<T, N>(out + r * N, o);
  return ok;
}

// 128-thread blocks; resident blocks per SM the register budget must allow:
// five for the n = 32 tensor-core version (two staged matrices per warp, so
// shared memory allows five) and for FP64, eight for the other FP32 group
// kernels (n = 16 included)
template <typename T, int N>
constexpr int kRakeBlocks = (sizeof(T) == 8 || N >= 32) ? 5 : 8;

template <typename T, int N>
__global__ void __launch_bounds__(128, kRakeBlocks<T, N>) kf_rake(Ws<T> w, int begin, int count) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int op;
  const Grp g = group_of<T, N>(count, &op);
  T* sm = reinterpret_cast<T*>(smem_raw + g.gid * TauSmem<T, N>::bytes);
  const int rr = begin + op, j = w.rake_leaf[rr];
  const size_t o = (size_t)j * N * N;
  const bool ok = tau_group<T, N>(w, g, w.U + o, w.Ea + o, w.Ec + o, w.Ep + o, w.contrib + (size_t)rr * N * N, sm);
  if (!ok && g.valid && g.gl == 0) atomicCAS(w.status, 0, ST_SINGULAR);
}

template <typename T, int N>
__global__ void __launch_bounds__(128, kRakeBlocks<T, N>) kf_expand(Ws<T> w, int begin, int count) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int op;
  const Grp g = group_of<T, N>(count, &op);
  T* sm = reinterpret_cast<T*>(smem_raw + g.gid * TauSmem<T, N>::bytes);
  const int rr = begin + op, j = w.comp_j[rr], k = w.comp_k[rr];
  const size_t oj = (size_t)j * N * N;
  const bool ok = tau_group<T, N>(w, g, w.U + (size_t)k * N * N, w.Ea + oj, w.Ec + oj, w.Ep + oj, w.U + oj, sm);
  if (!ok && g.valid && g.gl == 0) atomicCAS(w.status, 0, ST_SINGULAR);
}

// ---------------------------------------------------------------- compress
// eq. (compress-intermediates)-(composition) with the tape of
// eq. (quadratic-compress).  sm (group): Pt, Al, Cl, Ar, Y (2 matrices of
// 2N columns), the Gauss-Jordan broadcast rows.
template <typename T, int N>
struct CompSmem {
  // [Y1 | Y2]: Y2 at column YW (N rounded up to whole vectors); row stride an
  // odd number of vectors (conflict-free row stores)
  static constexpr int YW = D<T, N>::NV * D<T, N>::W;
  static constexpr int LD2 = (2 * D<T, N>::NV + 1) * D<T, N>::W;
  // P~, A_l, C_l, A_r; on the tensor-core path A_l and A_r stay in global memory
  static constexpr int mats = kTensorCores<T, N> ? 2 : 4;
  static constexpr int elems = mats * D<T, N>::MAT + N * LD2 + GjBuf<T, N, 2 * YW>::elems;
  static constexpr int bytes = ((elems * (int)sizeof(T) + 15) / 16) * 16;
};

// Tensor-core compression (n = 16, 32, FP32): P~ and C_l staged, the block products
// on the tensor cores, A_l and A_r read from global memory (so a warp holds two
// staged matrices and the [Y1 | Y2] panel instead of four and the panel).  The
// order keeps every read ahead of the write that replaces it: A_l (slot j) is
// last read by P_new, before the tape overwrites slot j; A_r (slot k) is last
// read by A_new, which replaces it.
template <typename T, int N>
__device__ __forceinline__ bool compress_op_tc(const Ws<T>& w, int rr, const Grp& g, T* sm) {
  using Dm = D<T, N>;
  constexpr int G = Dm::G, LD = Dm::LD, MAT = Dm::MAT, LD2 = CompSmem<T, N>::LD2, YW = CompSmem<T, N>::YW;
  constexpr int NN = N * N;
  T *sPt = sm, *sCl = sm + MAT, *sY = sm + 2 * MAT, *bc = sm + 2 * MAT + N * LD2;
  const int j = w.comp_j[rr], k = w.comp_k[rr];
  const size_t oj = (size_t)j * NN, ok_ = (size_t)k * NN;
  const T *Al = w.Ea + oj, *Ar = w.Ea + ok_;
  const int gl = g.gl, r = gl < N ? gl : 0;
#pragma unroll
  for (int e = gl; e < NN; e += G) {
    const int a = e / N, c = e - (e / N) * N;
    sPt[a * LD + c] = w.Ep[ok_ + e] + w.U[oj + e];                     // P~ = P_r + U_j
  }
  gload<T, N, N, LD, G>(sCl, w.Ec + oj, gl);
  __syncwarp();
  tc::gemm<N, false, false>(sCl, LD, sPt, LD, nullptr, 0, sY, LD2, true);   // C_l P~ -> Y1 columns
  tc::gemm<N, false, true>(sCl, LD, Ar, N, nullptr, 0, sY + YW, LD2, true);  // C_l A_r^T -> Y2 columns
  T s[N], b[2 * YW], t1[N], t2[N];
  row_load<T, N>(s, sY + r * LD2);
#pragma unroll
  for (int c = 0; c < N; ++c) s[c] += (c == r) ? T(1) : T(0);         // S = I + C_l P~
  grow_load<T, N>(t1, Al + r * N);
  row_load<T, N>(t2, sY + r * LD2 + YW);
#pragma unroll
  for (int c = 0; c < 2 * YW; ++c) b[c] = c < N ? t1[c] : (c >= YW && c < YW + N) ? t2[c - YW] : T(0);
  __syncwarp();
  int kpos;
  float pr;
  bool okf = ggj<T, N, G, 2 * YW>(s, b, gl, bc, kpos, pr);   // [Y1 | Y2] = S^{-1} [A_l | C_l A_r^T]
  bool stored = false;
  if (w.redo_count && g.valid && !(pr <= kSolveRatio)) {
    if (double* sc = redo_slot<G>(w.redo_count, w.redo_cap, w.redo_scratch, w.redo_slot, gl)) {
      okf = resolve64<N, G>(sc, RS_COMPRESS, sCl, LD, nullptr, sPt, LD, Al, N, Ar, N, sY, LD2, YW, sCl, LD, gl);
      stored = true;                            // [Y1 | Y2] in sY and W = P~ Y1 (FP64) in sCl
    }
  }
  if (!stored && gl < N) row_store<T, 2 * YW>(sY + kpos * LD2, b);
  __syncwarp();
  tc::gemm<N, false, false>(sPt, LD, sY, LD2, nullptr, 0, sCl, LD, !stored);          // W = P~ Y1 over C_l
  tc::gemm<N, true, false>(Al, N, sCl, LD, w.Ep + oj, N, w.Ep + ok_, N, g.valid);   // P_new = P_l + A_l^T W
  if (g.valid && gl < N) {
    // tape into slot j: (A_r, C_r, P~), read before slot k is rewritten
    T v[N];
    grow_load<T, N>(v, Ar + r * N);
    grow_store<T, N>(w.Ea + oj + r * N, v);
    grow_load<T, N>(v, w.Ec + ok_ + r * N);
    grow_store<T, N>(w.Ec + oj + r * N, v);
    row_load<T, N>(v, sPt + r * LD);
    grow_store<T, N>(w.Ep + oj + r * N, v);
  }
  __syncwarp();
  tc::gemm<N, false, false>(Ar, N, sY + YW, LD2, w.Ec + ok_, N, w.Ec + ok_, N, g.valid);   // C_new = C_r + A_r Y2
  tc::gemm<N, false, false>(Ar, N, sY, LD2, nullptr, 0, w.Ea + ok_, N, g.valid);          // A_new = A_r Y1
  return okf;
}

template <typename T, int N>
__device__ __forceinline__ bool compress_op(const Ws<T>& w, int rr, const Grp& g, T* sm) {
  if constexpr (kTensorCores<T, N>) return compress_op_tc<T, N>(w, rr, g, sm);
  using Dm = D<T, N>;
  constexpr int G = Dm::G, LD = Dm::LD, MAT = Dm::MAT, LD2 = CompSmem<T, N>::LD2, YW = CompSmem<T, N>::YW;
  constexpr int NN = N * N;
  T *sPt = sm, *sAl = sm + MAT, *sCl = sm + 2 * MAT, *sAr = sm + 3 * MAT, *sY = sm + 4 * MAT,
    *bc = sm + 4 * MAT + N * LD2;
  const int j = w.comp_j[rr], k = w.comp_k[rr];
  const size_t oj = (size_t)j * NN, ok_ = (size_t)k * NN;
  const int gl = g.gl, r = gl < N ? gl : 0;
  // stage; P~ = P_r + U_j
#pragma unroll
  for (int e = gl; e < NN; e += G) {
    const int a = e / N, c = e - (e / N) * N;
    sPt[a * LD + c] = w.Ep[ok_ + e] + w.U[oj + e];
  }
  gload<T, N, N, LD, G>(sAl, w.Ea + oj, gl);
  gload<T, N, N, LD, G>(sCl, w.Ec + oj, gl);
  gload<T, N, N, LD, G>(sAr, w.Ea + ok_, gl);
  __syncwarp();
  T s[N], b[2 * YW];
  {
    T cl[N], t1[N], t2[N];
    row_load<T, N>(cl, sCl + r * LD);
    zero(s);
    row_mm<T, N, N, LD>(s, cl, sPt);            // row r of C_l P~
#pragma unroll
    for (int c = 0; c < N; ++c) s[c] += (c == r) ? T(1) : T(0);   // S = I + C_l P~
    row_load<T, N>(t1, sAl + r * LD);
    zero(t2);
    row_mmT<T, N, N, LD>(t2, cl, sAr);          // row r of C_l A_r^T
#pragma unroll
    for (int c = 0; c < 2 * YW; ++c)
      b[c] = c < N ? t1[c] : (c >= YW && c < YW + N) ? t2[c - YW] : T(0);
  }
  __syncwarp();
  int kpos;
  float pr;
  bool okf = ggj<T, N, G, 2 * YW>(s, b, gl, bc, kpos, pr);   // [Y1 | Y2] = S^{-1} [A_l | C_l A_r^T], row kpos
  bool stored = false;
  if constexpr (sizeof(T) == 4) {
    if (w.redo_count && g.valid && !(pr <= kSolveRatio)) {
      if (double* sc = redo_slot<G>(w.redo_count, w.redo_cap, w.redo_scratch, w.redo_slot, gl)) {
        okf = resolve64<N, G>(sc, RS_COMPRESS, sCl, LD, nullptr, sPt, LD, sAl, LD, sAr, LD, sY, LD2, YW, sCl, LD,
                              gl);
        stored = true;                          // [Y1 | Y2] in sY and W = P~ Y1 (FP64) in sCl
      }
    }
  }
  if (!stored && gl < N) row_store<T, 2 * YW>(sY + kpos * LD2, b);
  __syncwarp();
  // A_new = A_r Y1, C_new = C_r + A_r Y2  (rows r); C_r read before slot k is overwritten
  T an[N], cn[N];
  {
    T ar[N];
    row_load<T, N>(ar, sAr + r * LD);
    zero(an);
    row_mm<T, N, N, LD2>(an, ar, sY);
    grow_load<T, N>(cn, w.Ec + ok_ + r * N);
    row_mm<T, N, N, LD2>(cn, ar, sY + YW);
  }
  // W = P~ Y1 (rows r) -> over C_l ; P_new = P_l + A_l^T W
  {
    T pt[N], wr[N];
    row_load<T, N>(pt, sPt + r * LD);
    zero(wr);
    row_mm<T, N, N, LD2>(wr, pt, sY);
    __syncwarp();
    if (!stored && gl < N) row_store<T, N>(sCl + r * LD, wr);
  }
  __syncwarp();
  T pn[N];
  grow_load<T, N>(pn, w.Ep + oj + r * N);                      // P_l, read before slot j is overwritten
  col_mm<T, N, N, LD, LD>(pn, sAl, r, sCl);
  __syncwarp();
  if (g.valid && gl < N) {
    // tape into slot j: (A_r, C_r, P~); composed edge into slot k
    T v[N];
    row_load<T, N>(v, sAr + r * LD);
    grow_store<T, N>(w.Ea + oj + r * N, v);
    grow_load<T, N>(v, w.Ec + ok_ + r * N);
    grow_store<T, N>(w.Ec + oj + r * N, v);
    row_load<T, N>(v, sPt + r * LD);
    grow_store<T, N>(w.Ep + oj + r * N, v);
  }
  __syncwarp();
  if (g.valid && gl < N) {
    grow_store<T, N>(w.Ea + ok_ + r * N, an);
    grow_store<T, N>(w.Ec + ok_ + r * N, cn);
    grow_store<T, N>(w.Ep + ok_ + r * N, pn);
  }
  __syncwarp();
  return okf;
}

template <typename T, int N>
__global__ void kf_compress(Ws<T> w, int begin, int count) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int op;
  const Grp g = group_of<T, N>(count, &op);
  T* sm = reinterpret_cast<T*>(smem_raw + g.gid * CompSmem<T, N>::bytes);
  const bool okf = compress_op<T, N>(w, begin + op, g, sm);
  if (!okf && g.valid && g.gl == 0) atomicCAS(w.status, 0, ST_SINGULAR);
}

// ================================================================ level-asynchronous contraction
// The late structural rounds hold few operations each, and executing them
// round by round puts one kernel launch and one operation latency on the
// critical path per phase.  Here the rakes, absorptions and compressions of
// rounds [r0, R) and the expansions of the same compressions run in ONE
// persistent launch without round barriers: each operation starts as soon as
// the data it reads are final, following the dependency DAG of
// eq. (earliest-level) (Sec. X-B, "Static dependency levels").
//
// The host lists the operations sorted by dependency level (so every
// operation comes after the ones it depends on) with runs of one kind padded
// to whole warps, and gives each operation at most three (flag, target)
// dependencies.  A warp takes the next OPS operations from a global counter;
// each of its lanes polls the flags of its group's operation with
// ld.acquire.gpu until they reach their targets, the warp runs the operations
// (all groups of a warp run the same kind, so the warp-wide collectives stay
// converged) and then publishes completion with st.release.gpu on the
// operation's flag; a rake also adds 1 to its sibling segment's counter, on
// which the absorption of that segment waits.  No deadlock is possible: an
// operation is only taken by a running warp, and its dependencies were taken
// earlier.  Every wait is bounded (spin_limit polls with backoff): when one
// runs out the kernel records ST_TIMEOUT, raises `abort` so that all warps
// leave, and returns -- the context stays usable and the host reports
// TLQR_ERR_TIMEOUT.
enum : int { AK_RAKE = 0, AK_ABSORB = 1, AK_COMPRESS = 2, AK_EXPAND = 3 };
// kinds of the state pass (kf_async_vec); the affine pass reuses the four above
enum : int { SK_COMPOSE = 4, SK_EXPAND_C = 5, SK_EXPAND_R = 6 };
constexpr int kAsyncPad = 0x0fffffff;       // index field of a padding slot

struct AsyncArgs {
  const int* op;            // [n_ops] kind << 28 | index (rake, segment or compression index)
  const int* dep_flag;      // [3 n_ops] flag indices, -1 = none
  const int* dep_target;    // [3 n_ops] value each flag must reach
  const int* signal;        // [n_ops] extra flag to increment on completion (-1 = none)
  int* flags;               // [n_flags]: done flag of op p at p, segment counters after them
  int* counter;             // next operation to hand out
  int* abort;               // set when a wait gave up
  int n_ops;                // multiple of the operations per warp
  int spin_limit;           // polls per wait before giving up
  int withhold;             // testing: the operation at this position never signals (-1 = none)
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_gpu(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) {
  int v;
  asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait until the operation at `pos` may start: every lane polls every one of
// its dependency flags with ld.acquire.gpu itself.  Returns true (uniformly in
// the warp) when a wait ran out or another warp gave up: the caller returns.
__device__ __forceinline__ bool async_wait(const AsyncArgs& a, int pos, int* status) {
  bool gave_up = false;
#pragma unroll 1
  for (int d = 0; d < 3 && !gave_up; ++d) {
    const int f = a.dep_flag[3 * pos + d];
    if (f < 0) continue;
    const int target = a.dep_target[3 * pos + d];
    int polls = 0;
    while (ld_acquire_gpu(a.flags + f) < target) {
      if (++polls > a.spin_limit || ld_volatile(a.abort)) { gave_up = true; break; }
      if (polls > 16) __nanosleep(polls < 128 ? 32 : 256);
    }
  }
  if (__any_sync(TLQR_FULL_MASK, gave_up)) {
    if ((threadIdx.x & 31) == 0) {
      atomicCAS(status, 0, ST_TIMEOUT);
      atomicExch(a.abort, 1);
    }
    return true;
  }
  return false;
}

// Publish the completion of the operation at `pos`: every lane's writes are
// fenced, then the group's first lane releases the flag (and a rake adds to
// its segment's counter).
__device__ __forceinline__ void async_publish(const AsyncArgs& a, int pos, bool valid, int gl) {
  __threadfence();
  __syncwarp();
  if (valid && gl == 0 && pos != a.withhold) {
    st_release_gpu(a.flags + pos, 1);
    const int sig = a.signal[pos];
    if (sig >= 0) red_release_add_gpu(a.flags + sig, 1);
  }
}

template <typename T, int N>
struct AsyncSmem {
  static constexpr int bytes = TauSmem<T, N>::bytes > CompSmem<T, N>::bytes ? TauSmem<T, N>::bytes
                                                                            : CompSmem<T, N>::bytes;
};

template <typename T, int N>
__global__ void kf_async(Ws<T> w, AsyncArgs a) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Dm = D<T, N>;
  constexpr int G = Dm::G, OPS = Dm::OPS, NN = N * N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane & (G - 1), gsub = lane / G;
  T* sm = reinterpret_cast<T*>(smem_raw + (warp * OPS + gsub) * AsyncSmem<T, N>::bytes);
  for (;;) {
    int base = 0;
    if (lane == 0) base = atomicAdd(a.counter, OPS);
    base = __shfl_sync(TLQR_FULL_MASK, base, 0);
    if (base >= a.n_ops) break;
    const int pos = base + gsub;
    const int word = a.op[pos];
    const int kind = word >> 28;                       // one kind per warp (host padding)
    int idx = word & kAsyncPad;
    const bool valid = idx != kAsyncPad;
    if (async_wait(a, pos, w.status)) return;
    // a padding group repeats the warp's first operation and stores nothing
    const int idx0 = __shfl_sync(TLQR_FULL_MASK, idx, 0);
    if (!valid) idx = idx0;
    const Grp g{gl, warp * OPS + gsub, valid};
    bool ok = true;
    if (kind == AK_RAKE) {
      const int j = w.rake_leaf[idx];
      const size_t o = (size_t)j * NN;
      ok = tau_group<T, N>(w, g, w.U + o, w.Ea + o, w.Ec + o, w.Ep + o, w.contrib + (size_t)idx * NN, sm);
    } else if (kind == AK_ABSORB) {
      const int i = w.seg_parent[idx], b = w.seg_start[idx], e = w.seg_start[idx + 1];
      T* Ui = w.U + (size_t)i * NN;
#pragma unroll 1
      for (int x = gl; x < NN; x += G) {
        T acc = w.contrib[(size_t)b * NN + x];
        for (int t = b + 1; t < e; ++t) acc += w.contrib[(size_t)t * NN + x];
        if (valid) Ui[x] += acc;
      }
    } else if (kind == AK_COMPRESS) {
      ok = compress_op<T, N>(w, idx, g, sm);
    } else {
      const int j = w.comp_j[idx], k = w.comp_k[idx];
      const size_t oj = (size_t)j * NN;
      ok = tau_group<T, N>(w, g, w.U + (size_t)k * NN, w.Ea + oj, w.Ec + oj, w.Ep + oj, w.U + oj, sm);
    }
    if (!ok && valid && gl == 0) atomicCAS(w.status, 0, ST_SINGULAR);
    async_publish(a, pos, valid, gl);
  }
}


// ---------------------------------------------------------------- composite transitions
// Tr_j <- T_k ; T_k <- T_k T_j  (eq. transition-compose), one group per compression.
template <typename T, int N>
struct ComposeSmem {
  static constexpr int bytes = D<T, N>::MAT * (int)sizeof(T);
};

template <typename T, int N>
__device__ __forceinline__ void compose_op(const Ws<T>& w, int rr, const Grp& g, T* sTj) {
  using Dm = D<T, N>;
  constexpr int G = Dm::G, LD = Dm::LD, NN = N * N;
  const int j = w.comp_j[rr], k = w.comp_k[rr];
  const int gl = g.gl, r = gl < N ? gl : 0;
  gload<T, N, N, LD, G>(sTj, w.Tm + (size_t)j * NN, gl);
  T tk[N], o[N];
  grow_load<T, N>(tk, w.Tm + (size_t)k * NN + r * N);
  if constexpr (kTensorCores<T, N>) {
    __syncwarp();
    if (g.valid && gl < N) grow_store<T, N>(w.Tr + (size_t)j * NN + r * N, tk);
    __syncwarp();
    tc::gemm<N, false, false>(w.Tm + (size_t)k * NN, N, sTj, LD, nullptr, 0, w.Tm + (size_t)k * NN, N, g.valid);
    return;
  }
  __syncwarp();
  zero(o);
  row_mm<T, N, N, LD>(o, tk, sTj);
  if (g.valid && gl < N) {
    grow_store<T, N>(w.Tr + (size_t)j * NN + r * N, tk);
    grow_store<T, N>(w.Tm + (size_t)k * NN + r * N, o);
  }
  __syncwarp();
}

template <typename T, int N>
__global__ void kf_compose_T(Ws<T> w, int begin, int count) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int op;
  const Grp g = group_of<T, N>(count, &op);
  compose_op<T, N>(w, begin + op, g, reinterpret_cast<T*>(smem_raw + g.gid * ComposeSmem<T, N>::bytes));
}

// ---------------------------------------------------------------- vector passes
// One group per operation; lane r owns entry r of the output vector.  Each
// operation is a device function so that the per-round kernels (one launch per
// phase) and the tail kernel (all small rounds in one block) share it.
template <typename T, int N>
__device__ __forceinline__ void vec_load(T (&v)[N], const T* src) {
#pragma unroll
  for (int c = 0; c < N; ++c) v[c] = src[c];
}

// contribution cv_rr = T_j^T h_j + z_j  (eq. affine-rake).  Every vector op
// below loads its block row or column once and applies it to the w.nrhs
// right-hand sides of a panel.
template <typename T, int N>
__device__ __forceinline__ void aff_rake_op(const Ws<T>& w, int rr, bool valid, int gl) {
  const int j = w.rake_leaf[rr], r = gl < N ? gl : 0;
  const T* Tj = w.Tm + (size_t)j * N * N;
  T col[N];
#pragma unroll
  for (int t = 0; t < N; ++t) col[t] = Tj[t * N + r];
  for (int k = 0; k < w.nrhs; ++k) {
    const Ws<T> v = w.rhs(k);
    T h[N];
    vec_load(h, v.h + (size_t)j * N);
    T s = v.z[(size_t)j * N + r];
#pragma unroll
    for (int t = 0; t < N; ++t) s = fma(col[t], h[t], s);
    if (valid && gl < N) v.cv[(size_t)rr * N + r] = s;
  }
}
// h_i += sum of the segment's contributions, in sibling order
template <typename T, int N>
__device__ __forceinline__ void aff_absorb_op(const Ws<T>& w, int sidx, bool valid, int gl) {
  const int i = w.seg_parent[sidx], b = w.seg_start[sidx], e = w.seg_start[sidx + 1], r = gl < N ? gl : 0;
  for (int k = 0; k < w.nrhs; ++k) {
    const Ws<T> v = w.rhs(k);
    T acc = v.cv[(size_t)b * N + r];
    for (int t = b + 1; t < e; ++t) acc += v.cv[(size_t)t * N + r];
    if (valid && gl < N) v.h[(size_t)i * N + r] += acc;
  }
}
// s_j = h_j + z_k ; z_k <- z_j + T_j^T s_j  (eq. affine-compose)
template <typename T, int N>
__device__ __forceinline__ void aff_compress_op(const Ws<T>& w, int rr, bool valid, int gl) {
  const int j = w.comp_j[rr], k = w.comp_k[rr], r = gl < N ? gl : 0;
  const T* Tj = w.Tm + (size_t)j * N * N;
  T col[N];
#pragma unroll
  for (int t = 0; t < N; ++t) col[t] = Tj[t * N + r];
  for (int q = 0; q < w.nrhs; ++q) {
    const Ws<T> v = w.rhs(q);
    T sv[N];
#pragma unroll
    for (int c = 0; c < N; ++c) sv[c] = v.h[(size_t)j * N + c] + v.z[(size_t)k * N + c];
    T acc = v.z[(size_t)j * N + r];
#pragma unroll
    for (int t = 0; t < N; ++t) acc = fma(col[t], sv[t], acc);
    const T sr = v.h[(size_t)j * N + r] + v.z[(size_t)k * N + r];
    __syncwarp();
    if (valid && gl < N) {
      v.s[(size_t)j * N + r] = sr;
      v.z[(size_t)k * N + r] = acc;
    }
  }
}
// p_j = Tr_j^T p_k + s_j  (affine expansion)
template <typename T, int N>
__device__ __forceinline__ void aff_expand_op(const Ws<T>& w, int rr, bool valid, int gl) {
  const int j = w.comp_j[rr], k = w.comp_k[rr], r = gl < N ? gl : 0;
  const T* Trj = w.Tr + (size_t)j * N * N;
  T col[N];
#pragma unroll
  for (int t = 0; t < N; ++t) col[t] = Trj[t * N + r];
  for (int q = 0; q < w.nrhs; ++q) {
    const Ws<T> v = w.rhs(q);
    T p[N];
    vec_load(p, v.h + (size_t)k * N);
    T acc = v.s[(size_t)j * N + r];
#pragma unroll
    for (int t = 0; t < N; ++t) acc = fma(col[t], p[t], acc);
    if (valid && gl < N) v.h[(size_t)j * N + r] = acc;
  }
}
// b_k <- Tr_j b_j + b_k  (state-map composition of the offsets)
template <typename T, int N>
__device__ __forceinline__ void state_compress_op(const Ws<T>& w, int rr, bool valid, int gl) {
  const int j = w.comp_j[rr], k = w.comp_k[rr], r = gl < N ? gl : 0;
  const T* Trj = w.Tr + (size_t)j * N * N + r * N;
  T row[N];
#pragma unroll
  for (int t = 0; t < N; ++t) row[t] = Trj[t];
  for (int q = 0; q < w.nrhs; ++q) {
    const Ws<T> v = w.rhs(q);
    T b[N];
    vec_load(b, v.bv + (size_t)j * N);
    T acc = v.bv[(size_t)k * N + r];
#pragma unroll
    for (int t = 0; t < N; ++t) acc = fma(row[t], b[t], acc);
    __syncwarp();
    if (valid && gl < N) v.bv[(size_t)k * N + r] = acc;
  }
}
// x_j = T_j x_i + b_j  (state expansion)
template <typename T, int N>
__device__ __forceinline__ void state_expand_op(const Ws<T>& w, const int* nodes, const int* from, int rr,
                                                bool valid, int gl) {
  const int j = nodes[rr], i = from[rr], r = gl < N ? gl : 0;
  const T* Tj = w.Tm + (size_t)j * N * N + r * N;
  T row[N];
#pragma unroll
  for (int t = 0; t < N; ++t) row[t] = Tj[t];
  for (int q = 0; q < w.nrhs; ++q) {
    const Ws<T> v = w.rhs(q);
    T x[N];
    vec_load(x, v.xs + (size_t)i * N);
    T acc = v.bv[(size_t)j * N + r];
#pragma unroll
    for (int t = 0; t < N; ++t) acc = fma(row[t], x[t], acc);
    if (valid && gl < N) v.xs[(size_t)j * N + r] = acc;
  }
}

template <typename T, int N>
__global__ void kf_aff_rake(Ws<T> w, int begin, int count) {
  pdl_entry();
  int op;
  const Grp g = group_of<T, N>(count, &op);
  aff_rake_op<T, N>(w, begin + op, g.valid, g.gl);
}
template <typename T, int N>
__global__ void kf_aff_absorb(Ws<T> w, int begin, int count) {
  pdl_entry();
  int op;
  const Grp g = group_of<T, N>(count, &op);
  aff_absorb_op<T, N>(w, begin + op, g.valid, g.gl);
}
template <typename T, int N>
__global__ void kf_aff_compress(Ws<T> w, int begin, int count) {
  pdl_entry();
  int op;
  const Grp g = group_of<T, N>(count, &op);
  aff_compress_op<T, N>(w, begin + op, g.valid, g.gl);
}
template <typename T, int N>
__global__ void kf_aff_expand(Ws<T> w, int begin, int count) {
  pdl_entry();
  int op;
  const Grp g = group_of<T, N>(count, &op);
  aff_expand_op<T, N>(w, begin + op, g.valid, g.gl);
}
template <typename T, int N>
__global__ void kf_state_compress(Ws<T> w, int begin, int count) {
  pdl_entry();
  int op;
  const Grp g = group_of<T, N>(count, &op);
  state_compress_op<T, N>(w, begin + op, g.valid, g.gl);
}
template <typename T, int N>
__global__ void kf_state_expand(Ws<T> w, const int* nodes, const int* from, int begin, int count) {
  pdl_entry();
  int op;
  const Grp g = group_of<T, N>(count, &op);
  state_expand_op<T, N>(w, nodes, from, begin + op, g.valid, g.gl);
}

// Right-hand-side passes, level-asynchronous: the affine pass (kinds AK_*: its
// dependency structure is that of the factorisation, on h for U, z for the
// edge slots and s for the tape) or the state pass (kinds SK_*), all rounds in
// one launch.  The operations are the O(n^2) vector maps of the per-round
// kernels; no shared memory.
template <typename T, int N>
__global__ void kf_async_vec(Ws<T> w, AsyncArgs a) {
  pdl_entry();
  constexpr int G = D<T, N>::G, OPS = D<T, N>::OPS;
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1), gsub = lane / G;
  for (;;) {
    int base = 0;
    if (lane == 0) base = atomicAdd(a.counter, OPS);
    base = __shfl_sync(TLQR_FULL_MASK, base, 0);
    if (base >= a.n_ops) break;
    const int pos = base + gsub;
    const int word = a.op[pos];
    const int kind = word >> 28;
    int idx = word & kAsyncPad;
    const bool valid = idx != kAsyncPad;
    if (async_wait(a, pos, w.status)) return;
    const int idx0 = __shfl_sync(TLQR_FULL_MASK, idx, 0);
    if (!valid) idx = idx0;
    switch (kind) {
      case AK_RAKE: aff_rake_op<T, N>(w, idx, valid, gl); break;
      case AK_ABSORB: aff_absorb_op<T, N>(w, idx, valid, gl); break;
      case AK_COMPRESS: aff_compress_op<T, N>(w, idx, valid, gl); break;
      case AK_EXPAND: aff_expand_op<T, N>(w, idx, valid, gl); break;
      case SK_COMPOSE: state_compress_op<T, N>(w, idx, valid, gl); break;
      case SK_EXPAND_C: state_expand_op<T, N>(w, w.comp_j, w.comp_i, idx, valid, gl); break;
      default: state_expand_op<T, N>(w, w.rake_leaf, w.rake_parent, idx, valid, gl); break;
    }
    async_publish(a, pos, valid, gl);
  }
}

// ---------------------------------------------------------------- tail kernels
// The late structural rounds hold few operations each; running them as one
// launch per phase costs a kernel launch per handful of operations.  A tail
// kernel runs rounds [r0, R) of a pass -- and the matching backward rounds --
// inside ONE block: its groups stride over each phase's operations and the
// phases are separated by __syncthreads().  No block waits for another.
struct RoundDesc { int rb, re, sb, se, cb, ce; };

// Threads of the single-block tail kernels; __launch_bounds__ keeps their
// register use within one block of this size.
constexpr int kTailBlock = 1024;

// Loop `count` operations over the block's groups with uniform trip counts.
#define TLQR_BLOCK_OPS(count, ...)                                             \
  do {                                                                         \
    const int cnt_ = (count);                                                  \
    for (int base_ = 0; base_ < cnt_; base_ += gpb) {                          \
      const int o_ = base_ + gid;                                              \
      const bool valid = o_ < cnt_;                                            \
      const int op = valid ? o_ : cnt_ - 1;                                    \
      __VA_ARGS__;                                                             \
    }                                                                          \
  } while (0)

// Affine pass tail: forward rounds r0..R-1 (rake, absorb, compress), then the
// backward rounds R-1..r0 (expand).
template <typename T, int N>
__global__ void __launch_bounds__(kTailBlock) kf_aff_tail(Ws<T> w, const RoundDesc* rounds, int r0, int R) {
  pdl_entry();
  constexpr int G = D<T, N>::G;
  const int gl = threadIdx.x & (G - 1), gid = threadIdx.x / G, gpb = blockDim.x / G;
  for (int r = r0; r < R; ++r) {
    const RoundDesc d = rounds[r];
    TLQR_BLOCK_OPS(d.re - d.rb, aff_rake_op<T, N>(w, d.rb + op, valid, gl));
    __syncthreads();
    TLQR_BLOCK_OPS(d.se - d.sb, aff_absorb_op<T, N>(w, d.sb + op, valid, gl));
    __syncthreads();
    TLQR_BLOCK_OPS(d.ce - d.cb, aff_compress_op<T, N>(w, d.cb + op, valid, gl));
    __syncthreads();
  }
  for (int r = R - 1; r >= r0; --r) {
    const RoundDesc d = rounds[r];
    TLQR_BLOCK_OPS(d.ce - d.cb, aff_expand_op<T, N>(w, d.cb + op, valid, gl));
    __syncthreads();
  }
}

// State pass tail: forward compositions r0..R-1, then expansion R-1..r0
// (compressed centres before the leaves raked in the same round).
template <typename T, int N>
__global__ void __launch_bounds__(kTailBlock) kf_state_tail(Ws<T> w, const RoundDesc* rounds, int r0, int R) {
  pdl_entry();
  constexpr int G = D<T, N>::G;
  const int gl = threadIdx.x & (G - 1), gid = threadIdx.x / G, gpb = blockDim.x / G;
  for (int r = r0; r < R; ++r) {
    const RoundDesc d = rounds[r];
    TLQR_BLOCK_OPS(d.ce - d.cb, state_compress_op<T, N>(w, d.cb + op, valid, gl));
    __syncthreads();
  }
  for (int r = R - 1; r >= r0; --r) {
    const RoundDesc d = rounds[r];
    TLQR_BLOCK_OPS(d.ce - d.cb, state_expand_op<T, N>(w, w.comp_j, w.comp_i, d.cb + op, valid, gl));
    __syncthreads();
    TLQR_BLOCK_OPS(d.re - d.rb, state_expand_op<T, N>(w, w.rake_leaf, w.rake_parent, d.rb + op, valid, gl));
    __syncthreads();
  }
}

}  // namespace fx
}  // namespace tlqr

namespace tlqr {
namespace fx {

// ================================================================ (n, m) kernels
// One group per node; lane r < N owns row r.  The m x m blocks (R, G) are
// factored redundantly by every lane of the group (m <= 8).

// Broadcast a length-N vector whose entry r lives in lane r of the group.
template <typename T, int N, int G>
__device__ __forceinline__ void gather_vec(T (&v)[N], T mine) {
#pragma unroll
  for (int t = 0; t < N; ++t) v[t] = __shfl_sync(TLQR_FULL_MASK, mine, t, G);
}

// In-register Cholesky of an M x M block (lower), returns false if not PD.
template <typename T, int M>
__device__ __forceinline__ bool chol_reg(T (&g)[M][M]) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    T d = g[k][k];
#pragma unroll
    for (int t = 0; t < k; ++t) d = fma(-g[k][t], g[k][t], d);
    ok = ok && d > T(0) && tfinite(d);
    const T s = sqrt(d > T(0) ? d : T(1));
    g[k][k] = s;
    const T inv = T(1) / s;
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      T v = g[i][k];
#pragma unroll
      for (int t = 0; t < k; ++t) v = fma(-g[i][t], g[k][t], v);
      g[i][k] = v * inv;
    }
  }
  return ok;
}
// FP64 fallback of chol_reg (see kCholRatio): when a group's FP32 factor of
// S = S64 + S32 failed or is ill-conditioned, the group's first lane
// refactors S in FP64 in `scratch` (M*M doubles of the group's shared memory)
// and writes the rounded L to lout (M rows of stride ldo); every lane of the
// group then reloads L from there.  s32 (shared, stride lds) may be null.
// Called by all lanes of the warp (warp-uniform); skip = this group has no
// block to factor (a root's empty edge slot).
template <typename T, int M, int G>
__device__ __forceinline__ bool chol_reg_checked(T (&l)[M][M], bool ok, bool skip, int gl, const double* s64,
                                                 const T* s32, int lds, double* scratch, T* lout, int ldo) {
  if constexpr (sizeof(T) == 8) {
    return ok;
  } else {
    float dmin = INFINITY, dmax = 0.f;
#pragma unroll
    for (int k = 0; k < M; ++k) { dmin = fminf(dmin, l[k][k]); dmax = fmaxf(dmax, l[k][k]); }
    const bool ill = !skip && (!ok || dmax > kCholRatio * dmin);
    if (!__any_sync(TLQR_FULL_MASK, ill)) return ok;
    bool ok64 = true;
    if (ill && gl == 0) {
#pragma unroll 1
      for (int e = 0; e < M * M; ++e) {
        const int i = e / M, j = e - (e / M) * M;
        scratch[e] = s64[e] + (s32 ? (double)s32[i * lds + j] : 0.0);
      }
      ok64 = chol64_serial(scratch, M, M);
#pragma unroll 1
      for (int e = 0; e < M * M; ++e) {
        const int i = e / M, j = e - (e / M) * M;
        lout[i * ldo + j] = j <= i ? (T)scratch[e] : T(0);
      }
    }
    const int leader = (threadIdx.x & 31) & ~(G - 1);
    ok64 = __shfl_sync(TLQR_FULL_MASK, ok64, leader);
    __syncwarp();
    if (ill) {
#pragma unroll
      for (int a = 0; a < M; ++a) {
        T row[M];
        row_load<T, M>(row, lout + a * ldo);
#pragma unroll
        for (int b = 0; b < M; ++b) l[a][b] = row[b];
      }
      ok = ok64;
    }
    __syncwarp();
    return ok;
  }
}

// Solve L L^T x = b in registers.
template <typename T, int M>
__device__ __forceinline__ void chol_solve_reg(const T (&l)[M][M], T (&b)[M]) {
#pragma unroll
  for (int i = 0; i < M; ++i) {
    T v = b[i];
#pragma unroll
    for (int t = 0; t < i; ++t) v = fma(-l[i][t], b[t], v);
    b[i] = v / l[i][i];
  }
#pragma unroll
  for (int i = M - 1; i >= 0; --i) {
    T v = b[i];
#pragma unroll
    for (int t = i + 1; t < M; ++t) v = fma(-l[t][i], b[t], v);
    b[i] = v / l[i][i];
  }
}

// Copy COUNT contiguous global elements into shared rows of stride LDS
// (COLS columns per row), converting S -> T.  Uses 16-byte loads when the
// block is a whole number of vectors and the rows are unpadded.
template <typename T, typename S, int ROWS, int COLS, int LDS, int G>
__device__ __forceinline__ void stage(T* dst, const S* src, int gl) {
  constexpr int COUNT = ROWS * COLS;
  constexpr int SW = 16 / (int)sizeof(S);
  if constexpr (COLS == LDS && COUNT % SW == 0) {
    using VS = typename Vec<S>::V;
#pragma unroll
    for (int v = gl; v < COUNT / SW; v += G) {
      const VS x = reinterpret_cast<const VS*>(src)[v];
#pragma unroll
      for (int i = 0; i < SW; ++i) dst[v * SW + i] = (T)vget<S>(x, i);
    }
  } else {
    gload<T, ROWS, COLS, LDS, G>(dst, src, gl);
  }
}

template <typename T, int M> struct MPad { static constexpr int LD = (M + Vec<T>::W - 1) / Vec<T>::W * Vec<T>::W; };

template <typename T, int N, int M>
struct CondSmem {
  static constexpr int MLD = MPad<T, M>::LD;
  // B, M, B R^{-1}, M R^{-1} (N rows of MLD each), R (M rows of MLD)
  static constexpr int elems = 4 * N * MLD + M * MLD;
  static constexpr int bytes = ((elems * (int)sizeof(T) + 15) / 16) * 16;
};

// Condensation eq. (edge-components), U_i <- Q_i, Delta flag.  All groups of a
// warp run the same instruction sequence; the root's group computes on its
// (ignored) edge slot and stores nothing but U and the flag.
template <typename T, int N, int M>
__global__ void kf_condense(Ws<T> w, int count) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int G = D<T, N>::G, NN = N * N, NM = N * M, MLD = CondSmem<T, N, M>::MLD;
  int i;
  const Grp g = group_of<T, N>(count, &i);
  T* sB = reinterpret_cast<T*>(smem_raw + g.gid * CondSmem<T, N, M>::bytes);
  T *sM = sB + N * MLD, *sBR = sM + N * MLD, *sMR = sBR + N * MLD, *sR = sMR + N * MLD;
  const int gl = g.gl, r = gl < N ? gl : 0;
  const size_t oi = (size_t)i * NN, om = (size_t)i * NM;
  const bool is_root = node_is_root(w, i);
  bool dnz = false;
  if (w.has_delta) {
    bool mine = false;
#pragma unroll
    for (int e = gl; e < NN; e += G) mine |= (w.Delta[oi + e] != 0.0);
    const unsigned bal = __ballot_sync(TLQR_FULL_MASK, mine);
    const int base = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gm = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
    dnz = ((bal >> base) & gm) != 0;
  }
  if (g.valid) {
#pragma unroll
    for (int e = gl; e < NN; e += G) w.U[oi + e] = (T)w.Q[oi + e];
    if (w.has_delta && gl == 0) w.dflag[i] = dnz ? 1 : 0;
  }
  stage<T, double, N, M, MLD, G>(sB, w.B + om, gl);
  if (w.has_M) stage<T, double, N, M, MLD, G>(sM, w.M + om, gl);
  stage<T, double, M, M, MLD, G>(sR, w.R + (size_t)i * M * M, gl);
  __syncwarp();
  T Rl[M][M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    T row[M];
    row_load<T, M>(row, sR + a * MLD);
#pragma unroll
    for (int b = 0; b < M; ++b) Rl[a][b] = row[b];
  }
  bool ok = chol_reg<T, M>(Rl);
  static_assert(2 * N * CondSmem<T, N, M>::MLD * sizeof(T) >= 8 * M * M, "FP64 scratch does not fit");
  __syncwarp();
  ok = chol_reg_checked<T, M, G>(Rl, ok, is_root || !g.valid, gl, w.R + (size_t)i * M * M, (const T*)nullptr, 0,
                                 reinterpret_cast<double*>(sBR), sR, MLD);
  T br[M];
  row_load<T, M>(br, sB + r * MLD);
  chol_solve_reg<T, M>(Rl, br);                 // row r of B R^{-1}
  if (gl < N) row_store<T, M>(sBR + r * MLD, br);
  if (w.has_M) {
    T mr[M];
    row_load<T, M>(mr, sM + r * MLD);
    chol_solve_reg<T, M>(Rl, mr);               // row r of M R^{-1}
    if (gl < N) row_store<T, M>(sMR + r * MLD, mr);
  }
  __syncwarp();
  // outputs element by element (coalesced): C = Delta + B R^{-1} B^T, A - B R^{-1} M^T, -M R^{-1} M^T
  if (g.valid && !is_root) {
#pragma unroll
    for (int e = gl; e < NN; e += G) {
      const int a = e / N, c = e - (e / N) * N;
      T x[M], y[M];
      row_load<T, M>(x, sBR + a * MLD);
      row_load<T, M>(y, sB + c * MLD);
      T cb = dnz ? (T)w.Delta[oi + e] : T(0);
#pragma unroll
      for (int b = 0; b < M; ++b) cb = fma(x[b], y[b], cb);
      w.Ec[oi + e] = cb;
      T ab = (T)w.A[oi + e], pb = T(0);
      if (w.has_M) {
        T mm[M], mr[M];
        row_load<T, M>(mm, sM + c * MLD);
        row_load<T, M>(mr, sMR + a * MLD);
#pragma unroll
        for (int b = 0; b < M; ++b) { ab = fma(-x[b], mm[b], ab); pb = fma(-mr[b], mm[b], pb); }
      }
      w.Ea[oi + e] = ab;
      w.Ep[oi + e] = pb;
    }
  }
  if (!ok && g.valid && !is_root && gl == 0) atomicCAS(w.status, 0, ST_NOT_PD);
}

template <typename T, int N, int M>
struct LfSmem {
  static constexpr int MAT = D<T, N>::MAT, LD = D<T, N>::LD, MLD = MPad<T, M>::LD;
  // P, Finv, A (-> A_cl), Delta, K (M x LD), B, W B, M (N x MLD), G (M x MLD), Gauss-Jordan rows
  static constexpr int elems = 4 * MAT + M * LD + 3 * N * MLD + M * MLD + GjBuf<T, N, N>::elems;
  static constexpr int bytes = ((elems * (int)sizeof(T) + 15) / 16) * 16;
};

// Local factors eq. (FW), (factor-local).  The F = I + Delta P branch runs in
// every group of a warp when any of them needs it (a group without Delta then
// factors F = I and ignores the result), so the warp stays converged.
template <typename T, int N, int M>
__global__ void kf_local_factor(Ws<T> w, int count) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using Dm = D<T, N>;
  using L = LfSmem<T, N, M>;
  constexpr int G = Dm::G, LD = Dm::LD, MAT = Dm::MAT, NN = N * N, NM = N * M, MLD = L::MLD;
  int j;
  const Grp g = group_of<T, N>(count, &j);
  unsigned char* gbase = smem_raw + g.gid * L::bytes;
  T* sm = reinterpret_cast<T*>(gbase);
  T *sP = sm, *sFi = sm + MAT, *sA = sm + 2 * MAT, *sD = sm + 3 * MAT, *sK = sm + 4 * MAT, *sB = sK + M * LD,
    *sWB = sB + N * MLD, *sMm = sWB + N * MLD, *sG = sMm + N * MLD, *bc = sG + M * MLD;
  const int gl = g.gl, r = gl < N ? gl : 0;
  const size_t oj = (size_t)j * NN, om = (size_t)j * NM;
  const bool is_root = node_is_root(w, j);
  const bool dnz = w.has_delta && w.dflag[j];
  const bool any_dnz = __any_sync(TLQR_FULL_MASK, dnz);
  stage<T, T, N, N, LD, G>(sP, w.U + oj, gl);
  stage<T, double, N, N, LD, G>(sA, w.A + oj, gl);
  stage<T, double, N, M, MLD, G>(sB, w.B + om, gl);
  if (w.has_M) stage<T, double, N, M, MLD, G>(sMm, w.M + om, gl);
  if (dnz) stage<T, double, N, N, LD, G>(sD, w.Delta + oj, gl);
  __syncwarp();
  T wrow[N];
  row_load<T, N>(wrow, sP + r * LD);            // W = P unless Delta_j != 0
  bool ok = true;
  if (any_dnz) {
    T f[N], e[N];
    zero(f);
    if (dnz) {
      T dr[N];
      row_load<T, N>(dr, sD + r * LD);
      row_mm<T, N, N, LD>(f, dr, sP);           // row r of Delta P
    }
#pragma unroll
    for (int c = 0; c < N; ++c) { f[c] += (c == r) ? T(1) : T(0); e[c] = (c == r) ? T(1) : T(0); }
    int kpos;
    float pr;
    ok = ggj<T, N, G, N>(f, e, gl, bc, kpos, pr);  // rows of F^{-1}
    bool stored = false;
    if constexpr (sizeof(T) == 4) {
      if (w.redo_count && dnz && g.valid && !(pr <= kSolveRatio)) {
        if (double* sc = redo_slot<G>(w.redo_count, w.redo_cap, w.redo_scratch, w.redo_slot, gl)) {
          ok = resolve64<N, G>(sc, RS_LOCAL, nullptr, N, w.Delta + oj, sP, LD, nullptr, 0, nullptr, 0, sFi, LD, 0,
                               sD, LD, gl);
          stored = true;                        // F^{-1} in sFi and W = P F^{-1} (FP64) in sD
        }
      }
    }
    if (!stored && gl < N) row_store<T, N>(sFi + kpos * LD, e);
    __syncwarp();
    if (dnz) {
      zero(wrow);
      T pr[N];
      row_load<T, N>(pr, sP + r * LD);
      row_mm<T, N, N, LD>(wrow, pr, sFi);       // row r of W = P F^{-1}
      if (stored) row_load<T, N>(wrow, sD + r * LD);
      if (g.valid) {
#pragma unroll
        for (int e2 = gl; e2 < NN; e2 += G) {
          const int a = e2 / N, c = e2 - (e2 / N) * N;
          w.Finv[oj + e2] = sFi[a * LD + c];
        }
        if (gl < N) {
#pragma unroll
          for (int c = 0; c < N; ++c) w.W[oj + r * N + c] = wrow[c];
        }
      }
    }
  }
  // row r of W B
  T wb[M];
#pragma unroll
  for (int a = 0; a < M; ++a) wb[a] = T(0);
  row_mm<T, N, M, MLD>(wb, wrow, sB);
  if (gl < N) row_store<T, M>(sWB + r * MLD, wb);
  __syncwarp();
  // G = R + B^T (W B): entry (a, b) by lane a*M + b, then factored in every
  // lane; in FP32, B^T W B is also kept apart (in the Delta tile, free by now)
  // for the FP64 fallback of the factorisation
  T* sBWB = sD;
  double* scratch = reinterpret_cast<double*>(sD + M * M);
  static_assert(MAT * sizeof(T) >= 4 * M * M + 8 * M * M, "FP64 scratch does not fit");
#pragma unroll
  for (int e2 = gl; e2 < M * M; e2 += G) {
    const int a = e2 / M, b = e2 - (e2 / M) * M;
    if constexpr (sizeof(T) == 8) {
      T v = (T)w.R[(size_t)j * M * M + e2];
#pragma unroll
      for (int t = 0; t < N; ++t) v = fma(sB[t * MLD + a], sWB[t * MLD + b], v);
      sG[a * MLD + b] = v;
    } else {
      T v = T(0);
#pragma unroll
      for (int t = 0; t < N; ++t) v = fma(sB[t * MLD + a], sWB[t * MLD + b], v);
      sBWB[e2] = v;
      sG[a * MLD + b] = (T)w.R[(size_t)j * M * M + e2] + v;
    }
  }
  __syncwarp();
  T Gl[M][M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    T row[M];
    row_load<T, M>(row, sG + a * MLD);
#pragma unroll
    for (int b = 0; b < M; ++b) Gl[a][b] = row[b];
  }
  bool okg = chol_reg<T, M>(Gl);
  __syncwarp();
  okg = chol_reg_checked<T, M, G>(Gl, okg, is_root || !g.valid, gl, w.R + (size_t)j * M * M, (const T*)sBWB, M,
                                  scratch, sG, MLD);
  // column r of H = (W B)^T A + M^T;  K(:, r) = -G^{-1} H(:, r)
  T hc[M];
  if (w.has_M) row_load<T, M>(hc, sMm + r * MLD);
  else {
#pragma unroll
    for (int a = 0; a < M; ++a) hc[a] = T(0);
  }
#pragma unroll
  for (int t = 0; t < N; ++t) {
    const T at = sA[t * LD + r];
    T wbt[M];
    row_load<T, M>(wbt, sWB + t * MLD);
#pragma unroll
    for (int a = 0; a < M; ++a) hc[a] = fma(wbt[a], at, hc[a]);
  }
  chol_solve_reg<T, M>(Gl, hc);
  if (gl < N) {
#pragma unroll
    for (int a = 0; a < M; ++a) sK[a * LD + r] = -hc[a];
  }
  __syncwarp();
  // row r of A_cl = A + B K
  T ac[N], brow[M];
  row_load<T, N>(ac, sA + r * LD);
  row_load<T, M>(brow, sB + r * MLD);
  row_mm<T, M, N, LD>(ac, brow, sK);
  const bool store = g.valid && !is_root;
  if (store) {
#pragma unroll
    for (int e2 = gl; e2 < M * N; e2 += G) {
      const int a = e2 / N, c = e2 - (e2 / N) * N;
      w.K[om + e2] = sK[a * LD + c];
    }
#pragma unroll
    for (int e2 = gl; e2 < M * M; e2 += G) {
      const int a = e2 / M, b = e2 - (e2 / M) * M;
      T v = T(0);
#pragma unroll
      for (int aa = 0; aa < M; ++aa)
#pragma unroll
        for (int bb = 0; bb < M; ++bb) v = (aa == a && bb == b) ? Gl[aa][bb] : v;
      w.LG[(size_t)j * M * M + e2] = v;
    }
  }
  __syncwarp();
  if (gl < N) row_store<T, N>(sA + r * LD, ac);
  __syncwarp();
  T t[N];
  if (any_dnz) {
    T fr[N];
    row_load<T, N>(fr, sFi + r * LD);
    zero(t);
    row_mm<T, N, N, LD>(t, fr, sA);             // T = F^{-1} A_cl
  }
  if (store && gl < N) {
#pragma unroll
    for (int c = 0; c < N; ++c) w.Tm[oj + r * N + c] = dnz ? t[c] : ac[c];
  }
  if (g.valid && gl == 0) {
    if (dnz && !ok) atomicCAS(w.status, 0, ST_SINGULAR);
    else if (!is_root && !okg) atomicCAS(w.status, 0, ST_NOT_PD);
  }
}

template <typename T, int N, int M>
struct AiSmem {
  static constexpr int LD = D<T, N>::LD, MLD = MPad<T, M>::LD;
  // W, A (N x LD), K (M x LD), B (N x MLD), c, w (LD), r (MLD)
  static constexpr int elems = 2 * N * LD + M * LD + N * MLD + 2 * LD + MLD;
  static constexpr int bytes = ((elems * (int)sizeof(T) + 15) / 16) * 16;
};

// Affine edge data eq. (affine-edge): h = q, z = K^T (r + B^T w) + A^T w, w = W c.
template <typename T, int N, int M>
__global__ void kf_aff_init(Ws<T> w, int count) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using A_ = AiSmem<T, N, M>;
  constexpr int G = D<T, N>::G, LD = A_::LD, MLD = A_::MLD, NN = N * N, NM = N * M;
  int j;
  const Grp g = group_of<T, N>(count, &j);
  T* sW = reinterpret_cast<T*>(smem_raw + g.gid * A_::bytes);
  T *sA = sW + N * LD, *sK = sA + N * LD, *sB = sK + M * LD, *vc = sB + N * MLD, *vw = vc + LD, *vr = vw + LD;
  const int gl = g.gl, r = gl < N ? gl : 0;
  const bool is_root = node_is_root(w, j);
  const size_t oj = (size_t)j * NN, om = (size_t)j * NM;
  const bool dnz = w.has_delta && w.dflag[j];
  stage<T, T, N, N, LD, G>(sW, dnz ? w.W + oj : w.U + oj, gl);
  stage<T, double, N, N, LD, G>(sA, w.A + oj, gl);
  stage<T, T, M, N, LD, G>(sK, w.K + om, gl);
  stage<T, double, N, M, MLD, G>(sB, w.B + om, gl);
  for (int k = 0; k < w.nrhs; ++k) {           // right-hand sides of a panel, blocks staged once
    const Ws<T> q = w.rhs(k);
    if (g.valid && gl < N) q.h[(size_t)j * N + r] = (T)q.q[(size_t)j * N + r];
    if (gl < N) vc[gl] = (T)q.c[(size_t)j * N + gl];
    if (gl < M) vr[gl] = (T)q.r[(size_t)j * M + gl];
    if (gl >= N && gl < LD) vc[gl] = T(0);
    __syncwarp();
    T row[N], cv[N];
    row_load<T, N>(row, sW + r * LD);
    row_load<T, N>(cv, vc);
    T wr = T(0);
#pragma unroll
    for (int t = 0; t < N; ++t) wr = fma(row[t], cv[t], wr);     // w = W c
    if (gl < N) vw[gl] = wr;
    __syncwarp();
    T wv[N], v[M];
    row_load<T, N>(wv, vw);
    row_load<T, M>(v, vr);
    row_mm<T, N, M, MLD>(v, wv, sB);              // v = r + B^T w
    T z = T(0);
#pragma unroll
    for (int a = 0; a < M; ++a) z = fma(sK[a * LD + r], v[a], z);
#pragma unroll
    for (int t = 0; t < N; ++t) z = fma(sA[t * LD + r], wv[t], z);
    if (g.valid && !is_root && gl < N) q.z[(size_t)j * N + r] = z;
    __syncwarp();
  }
}

template <typename T, int N, int M>
struct LsSmem {
  static constexpr int LD = D<T, N>::LD, MLD = MPad<T, M>::LD;
  // W, Delta, Finv (N x LD), B (N x MLD), LG (M x MLD), p, f, g, t (LD), r (MLD)
  static constexpr int elems = 3 * N * LD + N * MLD + M * MLD + 4 * LD + MLD;
  static constexpr int bytes = ((elems * (int)sizeof(T) + 15) / 16) * 16;
};

// Local affine solve eq. (local-affine-solve) and the root state eq. (xroot).
template <typename T, int N, int M>
__global__ void kf_local_solve(Ws<T> w, int count) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using L = LsSmem<T, N, M>;
  constexpr int G = D<T, N>::G, LD = L::LD, MLD = L::MLD, NN = N * N, NM = N * M;
  int j;
  const Grp g = group_of<T, N>(count, &j);
  T* sW = reinterpret_cast<T*>(smem_raw + g.gid * L::bytes);
  T *sD = sW + N * LD, *sFi = sD + N * LD, *sB = sFi + N * LD, *sL = sB + N * MLD, *vp = sL + M * MLD,
    *vf = vp + LD, *vg = vf + LD, *vt = vg + LD, *vr = vt + LD;
  const int gl = g.gl, r = gl < N ? gl : 0;
  const size_t oj = (size_t)j * NN, om = (size_t)j * NM;
  const bool dnz = w.has_delta && w.dflag[j];
  const bool is_root = node_is_root(w, j);
  stage<T, T, N, N, LD, G>(sW, dnz ? w.W + oj : w.U + oj, gl);
  stage<T, double, N, M, MLD, G>(sB, w.B + om, gl);
  if (!is_root) stage<T, T, M, M, MLD, G>(sL, w.LG + (size_t)j * M * M, gl);
  if (dnz) {
    stage<T, double, N, N, LD, G>(sD, w.Delta + oj, gl);
    stage<T, T, N, N, LD, G>(sFi, w.Finv + oj, gl);
  }
  for (int kq = 0; kq < w.nrhs; ++kq) {         // right-hand sides of a panel, blocks staged once
    const Ws<T> q = w.rhs(kq);
    if (gl < LD) vp[gl] = gl < N ? q.h[(size_t)j * N + gl] : T(0);
    if (gl < M) vr[gl] = (T)q.r[(size_t)j * M + gl];
    __syncwarp();
    T p[N];
    row_load<T, N>(p, vp);
    T pr = p[0];
#pragma unroll
    for (int t = 0; t < N; ++t) pr = (t == r) ? p[t] : pr;
    T fr = -(T)q.c[(size_t)j * N + r];
    if (dnz) {
      T dr[N];
      row_load<T, N>(dr, sD + r * LD);
#pragma unroll
      for (int t = 0; t < N; ++t) fr = fma(dr[t], p[t], fr);   // f = Delta p - c
    }
    if (gl < LD) vf[gl] = gl < N ? fr : T(0);
    __syncwarp();
    T f[N];
    row_load<T, N>(f, vf);
    // root: x = -F^{-1} f ; others: g = p - W f
    T xr = -fr;
    if (dnz) {
      T fi[N];
      row_load<T, N>(fi, sFi + r * LD);
      xr = T(0);
#pragma unroll
      for (int t = 0; t < N; ++t) xr = fma(-fi[t], f[t], xr);
    }
    T wrow[N];
    row_load<T, N>(wrow, sW + r * LD);
    T gr = pr;
#pragma unroll
    for (int t = 0; t < N; ++t) gr = fma(-wrow[t], f[t], gr);
    if (gl < LD) vg[gl] = gl < N ? gr : T(0);
    __syncwarp();
    // k = -G^{-1}(r + B^T g) (every lane)
    T gv[N], k[M];
    row_load<T, N>(gv, vg);
    row_load<T, M>(k, vr);
    row_mm<T, N, M, MLD>(k, gv, sB);
    T Lg[M][M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      T row[M];
      row_load<T, M>(row, sL + a * MLD);
#pragma unroll
      for (int b = 0; b < M; ++b) Lg[a][b] = is_root ? ((a == b) ? T(1) : T(0)) : row[b];
    }
    chol_solve_reg<T, M>(Lg, k);
#pragma unroll
    for (int a = 0; a < M; ++a) k[a] = -k[a];
    // b = F^{-1}(B k - f)
    T brow[M];
    row_load<T, M>(brow, sB + r * MLD);
    T tr = -fr;
#pragma unroll
    for (int a = 0; a < M; ++a) tr = fma(brow[a], k[a], tr);
    if (gl < LD) vt[gl] = gl < N ? tr : T(0);
    __syncwarp();
    T b = tr;
    if (dnz) {
      T tv[N], fi[N];
      row_load<T, N>(tv, vt);
      row_load<T, N>(fi, sFi + r * LD);
      b = T(0);
#pragma unroll
      for (int t = 0; t < N; ++t) b = fma(fi[t], tv[t], b);
    }
    if (g.valid) {
      if (is_root) {
        if (gl < N) q.xs[(size_t)j * N + r] = xr;
      } else {
        if (gl < M) {
          T kk = k[0];
#pragma unroll
          for (int a = 0; a < M; ++a) kk = (a == gl) ? k[a] : kk;
          q.kv[(size_t)j * M + gl] = kk;
        }
        if (gl < N) q.bv[(size_t)j * N + r] = b;
      }
    }
    __syncwarp();
  }
}

// Recovery eq. (recover) into FP64 x, u, y (written or accumulated).
template <typename T, int N, int M>
__global__ void kf_recover(Ws<T> w, double* x, double* u, double* y, int accumulate, int count) {
  pdl_entry();
  constexpr int NN = N * N, NM = N * M;
  int j;
  const Grp g = group_of<T, N>(count, &j);
  const int gl = g.gl, r = gl < N ? gl : 0;
  for (int kq = 0; kq < w.nrhs; ++kq) {         // right-hand sides of a panel
    const Ws<T> q = w.rhs(kq);
    double *qx = x + (size_t)kq * w.sv, *qu = u + (size_t)kq * w.sm, *qy = y + (size_t)kq * w.sv;
    T xv[N];
#pragma unroll
    for (int t = 0; t < N; ++t) xv[t] = q.xs[(size_t)j * N + t];
    T xr = xv[0];
#pragma unroll
    for (int t = 0; t < N; ++t) xr = (t == r) ? xv[t] : xr;
    T yr = q.h[(size_t)j * N + r];
#pragma unroll
    for (int t = 0; t < N; ++t) yr = fma(w.U[(size_t)j * NN + t * N + r], xv[t], yr);   // P symmetric
    bool bad = !tfinite(xr) || !tfinite(yr);
    const bool nonroot = !node_is_root(w, j);
    T ur = T(0);
    if (nonroot && gl < M) {
      const int par = w.parent[j];
      ur = q.kv[(size_t)j * M + gl];
#pragma unroll
      for (int t = 0; t < N; ++t) ur = fma(w.K[(size_t)j * NM + gl * N + t], q.xs[(size_t)par * N + t], ur);
      bad |= !tfinite(ur);
    }
    if (g.valid) {
      if (gl < N) {
        const size_t o = (size_t)j * N + r;
        if (accumulate) { qx[o] += (double)xr; qy[o] += (double)yr; }
        else { qx[o] = (double)xr; qy[o] = (double)yr; }
      }
      if (gl < M) {
        const size_t o = (size_t)j * M + gl;
        if (nonroot) { if (accumulate) qu[o] += (double)ur; else qu[o] = (double)ur; }
        else if (!accumulate) qu[o] = 0.0;
      }
      if (bad) atomicCAS(w.status, 0, ST_NONFINITE);
    }
  }
}

}  // namespace fx
}  // namespace tlqr
