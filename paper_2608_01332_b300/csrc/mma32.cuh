// Warp-level block products on the tensor cores for the n = 32 group kernels
// (one warp per local operation, 32 x 32 x 32) and the n = 16 ones (two
// operations per warp, 16 x 16 x 16 each): C = op(A) op(B) (+ Cin) with
// mma.sync m16n8k8 TF32 instructions and the "3xTF32" split: every FP32
// operand x = big + small with big = tf32(x) and small = tf32(x - big), and
// A B = A_big B_big + A_big B_small + A_small B_big (the small x small term is
// dropped), accumulated in FP32.  The result is accurate to a few FP32 ulps of
// the terms, like the SIMT products it replaces.
//
// Operands are read through generic pointers (shared or global memory), row
// major with leading dimensions; TA / TB read A / B transposed.  The output is
// written through a generic pointer only when `store` is true (all 32 lanes
// take part either way: the mma instructions are warp-collective).  Reads of
// A, B and Cin all happen before the first write of C, with a __syncwarp()
// between, so C may alias any input.
//
// Fragment layout of m16n8k8 (g = lane / 4, t = lane % 4):
//   A (16 x 8):  a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4)
//   B (8 x 8):   b0 (t, g), b1 (t + 4, g)
//   C (16 x 8):  c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1)
#pragma once
#include <cstdint>

namespace tlqr {
namespace tc {

__device__ __forceinline__ unsigned tf32_of(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, unsigned& big, unsigned& small) {
  big = tf32_of(x);
  small = tf32_of(x - __uint_as_float(big));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <bool TA, bool TB>
__device__ __forceinline__ void gemm32(const float* A, int lda, const float* B, int ldb, const float* Cin, int ldcin,
                                       float* C, int ldc, bool store) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int r0 = mt * 16 + g, c0 = nt * 8 + 2 * t;
      if (Cin) {
        acc[mt][nt][0] = Cin[r0 * ldcin + c0];
        acc[mt][nt][1] = Cin[r0 * ldcin + c0 + 1];
        acc[mt][nt][2] = Cin[(r0 + 8) * ldcin + c0];
        acc[mt][nt][3] = Cin[(r0 + 8) * ldcin + c0 + 1];
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
      }
    }
  auto a_at = [&](int i, int k) { return TA ? A[k * lda + i] : A[i * lda + k]; };
  auto b_at = [&](int k, int j) { return TB ? B[j * ldb + k] : B[k * ldb + j]; };
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const int k0 = kk * 8;
    unsigned ab[2][4], as[2][4], bb[4][2], bs[4][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int i0 = mt * 16 + g;
      tf32_split(a_at(i0, k0 + t), ab[mt][0], as[mt][0]);
      tf32_split(a_at(i0 + 8, k0 + t), ab[mt][1], as[mt][1]);
      tf32_split(a_at(i0, k0 + t + 4), ab[mt][2], as[mt][2]);
      tf32_split(a_at(i0 + 8, k0 + t + 4), ab[mt][3], as[mt][3]);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int j0 = nt * 8 + g;
      tf32_split(b_at(k0 + t, j0), bb[nt][0], bs[nt][0]);
      tf32_split(b_at(k0 + t + 4, j0), bb[nt][1], bs[nt][1]);
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        mma_tf32(acc[mt][nt], as[mt][0], as[mt][1], as[mt][2], as[mt][3], bb[nt][0], bb[nt][1]);
        mma_tf32(acc[mt][nt], ab[mt][0], ab[mt][1], ab[mt][2], ab[mt][3], bs[nt][0], bs[nt][1]);
        mma_tf32(acc[mt][nt], ab[mt][0], ab[mt][1], ab[mt][2], ab[mt][3], bb[nt][0], bb[nt][1]);
      }
  }
  __syncwarp();
  if (store) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int r0 = mt * 16 + g, c0 = nt * 8 + 2 * t;
        C[r0 * ldc + c0] = acc[mt][nt][0];
        C[r0 * ldc + c0 + 1] = acc[mt][nt][1];
        C[(r0 + 8) * ldc + c0] = acc[mt][nt][2];
        C[(r0 + 8) * ldc + c0 + 1] = acc[mt][nt][3];
      }
  }
  __syncwarp();
}

// Two 16 x 16 x 16 products per warp for the n = 16 group kernels (two
// operations per warp, one per half warp): lanes 0-15 pass the operands of
// their group's product, lanes 16-31 those of theirs; every lane takes part in
// both products, whose operand addresses it obtains by shuffles.  Leading
// dimensions and whether Cin is given must be the same in both halves; `store`
// may differ.  Same split, accumulation and aliasing rules as gemm32.
__device__ __forceinline__ const float* shfl_ptr(const float* p, int src) {
  return reinterpret_cast<const float*>(
      __shfl_sync(0xffffffffu, (unsigned long long)reinterpret_cast<uintptr_t>(p), src));
}

template <bool TA, bool TB>
__device__ __forceinline__ void gemm16x2(const float* A, int lda, const float* B, int ldb, const float* Cin, int ldcin,
                                         float* C, int ldc, bool store) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[2][2][4];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float* Ap = shfl_ptr(A, 16 * p);
    const float* Bp = shfl_ptr(B, 16 * p);
    const float* Cp = Cin ? shfl_ptr(Cin, 16 * p) : nullptr;
    auto a_at = [&](int i, int k) { return TA ? Ap[k * lda + i] : Ap[i * lda + k]; };
    auto b_at = [&](int k, int j) { return TB ? Bp[j * ldb + k] : Bp[k * ldb + j]; };
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const int c0 = nt * 8 + 2 * t;
      if (Cp) {
        acc[p][nt][0] = Cp[g * ldcin + c0];
        acc[p][nt][1] = Cp[g * ldcin + c0 + 1];
        acc[p][nt][2] = Cp[(g + 8) * ldcin + c0];
        acc[p][nt][3] = Cp[(g + 8) * ldcin + c0 + 1];
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][nt][q] = 0.f;
      }
    }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int k0 = kk * 8;
      unsigned ab[4], as[4];
      tf32_split(a_at(g, k0 + t), ab[0], as[0]);
      tf32_split(a_at(g + 8, k0 + t), ab[1], as[1]);
      tf32_split(a_at(g, k0 + t + 4), ab[2], as[2]);
      tf32_split(a_at(g + 8, k0 + t + 4), ab[3], as[3]);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        unsigned bb[2], bs[2];
        tf32_split(b_at(k0 + t, nt * 8 + g), bb[0], bs[0]);
        tf32_split(b_at(k0 + t + 4, nt * 8 + g), bb[1], bs[1]);
        mma_tf32(acc[p][nt], as[0], as[1], as[2], as[3], bb[0], bb[1]);
        mma_tf32(acc[p][nt], ab[0], ab[1], ab[2], ab[3], bs[0], bs[1]);
        mma_tf32(acc[p][nt], ab[0], ab[1], ab[2], ab[3], bb[0], bb[1]);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    float* Cd = const_cast<float*>(shfl_ptr(C, 16 * p));
    const bool st = __shfl_sync(0xffffffffu, store, 16 * p);
    if (st) {
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int c0 = nt * 8 + 2 * t;
        Cd[g * ldc + c0] = acc[p][nt][0];
        Cd[g * ldc + c0 + 1] = acc[p][nt][1];
        Cd[(g + 8) * ldc + c0] = acc[p][nt][2];
        Cd[(g + 8) * ldc + c0 + 1] = acc[p][nt][3];
      }
    }
  }
  __syncwarp();
}

// The n x n block product of the group kernels on the tensor cores: one
// warp-wide 32 x 32 product (n = 32) or one 16 x 16 product per half warp (n = 16).
template <int N, bool TA, bool TB>
__device__ __forceinline__ void gemm(const float* A, int lda, const float* B, int ldb, const float* Cin, int ldcin,
                                     float* C, int ldc, bool store) {
  static_assert(N == 16 || N == 32, "tensor-core products for n = 16 and n = 32");
  if constexpr (N == 32) gemm32<TA, TB>(A, lda, B, ldb, Cin, ldcin, C, ldc, store);
  else gemm16x2<TA, TB>(A, lda, B, ldb, Cin, ldcin, C, ldc, store);
}

}  // namespace tc
}  // namespace tlqr
