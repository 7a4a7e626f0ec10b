// Float-float KKT residual of eq. (kkt), organised by node for compile-time
// (n, m): one group of G lanes per node, lane r owning row r.  Each node's
// FP64 blocks are copied into shared memory with asynchronous 8-byte copies
// (cp.async), double-buffered so that the next node's blocks are in flight
// while the current node is computed; every FP64 matrix entry is read from HBM
// exactly once per evaluation (the row-per-thread kernels of residual.cuh read
// A_j and B_j twice and walk Q by strided rows).
//
// Two launches:
//   edge pass, node j:  the constraint row entering j
//                          A_j x_p + B_j u_j + c_j - x_j - Delta_j y_j
//                       the control row of the edge into j
//                          M_j^T x_p + R_j u_j + r_j + B_j^T y_j
//                       and the message to the parent's stationarity row
//                          w_j = A_j^T y_j + M_j u_j        (float-float, stored)
//   node pass, node i:  Q_i x_i + q_i - y_i + sum_{children j} w_j
// Absolute row sums of the KKT matrix (||K||_inf) follow the same split; the
// maxima ||res||, ||z||, ||b||, ||K|| are folded per block (one tree) or per
// tree (a forest), exactly as the row kernels do.
#pragma once
#include "residual.cuh"

namespace tlqr {
namespace rn {

template <int N>
struct RG {
  static constexpr int G = N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32;
  static constexpr int OPS = 32 / G;          // nodes per warp
};

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

// Asynchronous copy of an R x C FP64 block (contiguous rows) into shared rows
// of stride LDS, by the G lanes of a group.
template <int R, int C, int LDS, int G>
__device__ __forceinline__ void stage_async(double* dst, const double* src, int gl) {
#pragma unroll 4
  for (int e = gl; e < R * C; e += G) {
    const int a = e / C, b = e - (e / C) * C;
    cp_async8(dst + a * LDS + b, src + e);
  }
}

// s += sum_b a[b * STRIDE] * (xh[b] + xl[b]) (sign -1: minus), with four
// independent float-float accumulators to shorten the dependent chain; returns
// the FP32 sum of |a_hi| for the absolute row sums.
template <int K, int STRIDE>
__device__ __forceinline__ float ff_dot(FF& s, const double* a, const float* xh, const float* xl, float sign = 1.f) {
  FF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  float rs = 0.f;
#pragma unroll
  for (int b = 0; b < K; ++b) rs += ff_fma_d(acc[b & 3], a[b * STRIDE], sign * xh[b], sign * xl[b]);
#pragma unroll
  for (int q = 0; q < 4; ++q) ff_add2(s, acc[q].h, acc[q].l);
  return rs;
}

// Warp-contiguous node ranges: warp w handles nodes [w*C, (w+1)*C), OPS at a time.
struct NodeRange {
  int begin, end;
};
template <int OPS>
__device__ __forceinline__ NodeRange warp_nodes(int N) {
  const int wpb = blockDim.x >> 5, warps = gridDim.x * wpb, gw = blockIdx.x * wpb + (threadIdx.x >> 5);
  int c = (N + warps - 1) / warps;
  c = (c + OPS - 1) / OPS * OPS;
  const long long b = (long long)gw * c;
  NodeRange r;
  r.begin = (int)(b < N ? b : N);
  r.end = (int)(b + c < N ? b + c : N);
  return r;
}

struct NodeArgs {
  float *wh, *wl;     // [N][n] float-float message w_j to the parent row
  float* wk;          // [N][n] absolute column sums of [A_j^T | M_j] (when with_knorm)
};

struct Maxima {
  unsigned long long v[4] = {0ull, 0ull, 0ull, 0ull};
  __device__ __forceinline__ void take(const unsigned long long (&r)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = r[q] > v[q] ? r[q] : v[q];
  }
};

// Shared-memory layout of one edge-pass buffer (doubles): A, [Delta], B, [M], R.
template <int N, int M>
struct EdgeBuf {
  static constexpr int LDA = N + 1, LDB = M + 1;
  __host__ __device__ static constexpr int doubles(bool has_delta, bool has_M) {
    return N * LDA * (has_delta ? 2 : 1) + N * LDB * (has_M ? 2 : 1) + M * LDB;
  }
  // per group: two buffers + the float-float vectors x_p, y_j (N each), u_j (M), hi and lo
  __host__ __device__ static constexpr int group_bytes(bool has_delta, bool has_M) {
    return ((2 * doubles(has_delta, has_M) * 8 + (4 * N + 2 * M) * 4) + 15) / 16 * 16;
  }
};

// Edge pass.  FOREST: fold maxima per tree.
template <int N, int M, bool FOREST>
__global__ void __launch_bounds__(128) k_res_edge(ResidualArgs a, FFArgs f, NodeArgs na) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using EB = EdgeBuf<N, M>;
  constexpr int G = RG<N>::G, OPS = RG<N>::OPS, LDA = EB::LDA, LDB = EB::LDB;
  const bool hd = a.Delta != nullptr, hm = a.M != nullptr, ks = a.with_knorm;
  const int gl = threadIdx.x & (G - 1), gid = (threadIdx.x & 31) / G;
  const int nd = EB::doubles(hd, hm);
  unsigned char* gbase = smem_raw + (size_t)((threadIdx.x >> 5) * OPS + gid) * EB::group_bytes(hd, hm);
  double* buf0 = reinterpret_cast<double*>(gbase);
  float* vxh = reinterpret_cast<float*>(gbase + 2 * (size_t)nd * 8);
  float *vxl = vxh + N, *vyh = vxl + N, *vyl = vyh + N, *vuh = vyl + N, *vul = vuh + M;
  const size_t nn = (size_t)N * N, nm = (size_t)N * M;
  auto issue = [&](int j, double* b) {
    double* sA = b;
    double* sD = sA + N * LDA;
    double* sB = sD + (hd ? N * LDA : 0);
    double* sM = sB + N * LDB;
    double* sR = sM + (hm ? N * LDB : 0);
    if (a.parent[j] >= 0) {
      stage_async<N, N, LDA, G>(sA, a.A + (size_t)j * nn, gl);
      stage_async<N, M, LDB, G>(sB, a.B + (size_t)j * nm, gl);
      stage_async<M, M, LDB, G>(sR, a.R + (size_t)j * M * M, gl);
      if (hm) stage_async<N, M, LDB, G>(sM, a.M + (size_t)j * nm, gl);
    }
    if (hd) stage_async<N, N, LDA, G>(sD, a.Delta + (size_t)j * nn, gl);
  };
  const NodeRange nr = warp_nodes<OPS>(a.N);
  Maxima mx;
  TreeAcc acc;
  if (nr.begin < nr.end) issue(nr.begin + gid < nr.end ? nr.begin + gid : nr.end - 1, buf0);
  cp_async_commit();
  int t = 0;
  for (int base = nr.begin; base < nr.end; base += OPS, ++t) {
    const int j0 = base + gid;
    const bool valid = j0 < nr.end;
    const int j = valid ? j0 : nr.end - 1;
    double* cur = buf0 + (t & 1) * nd;
    if (base + OPS < nr.end) {                           // prefetch this group's next node
      const int jn = base + OPS + gid < nr.end ? base + OPS + gid : nr.end - 1;
      issue(jn, buf0 + ((t + 1) & 1) * nd);
    }
    cp_async_commit();
    cp_async_wait<1>();
    const int p = a.parent[j];
    const bool has_p = p >= 0;
    if (gl < N) {
      vyh[gl] = f.yh[(size_t)j * N + gl];
      vyl[gl] = f.yl[(size_t)j * N + gl];
      vxh[gl] = has_p ? f.xh[(size_t)p * N + gl] : 0.f;
      vxl[gl] = has_p ? f.xl[(size_t)p * N + gl] : 0.f;
    }
    if (gl < M) {
      vuh[gl] = f.uh[(size_t)j * M + gl];
      vul[gl] = f.ul[(size_t)j * M + gl];
    }
    __syncwarp();
    const double* sA = cur;
    const double* sD = sA + N * LDA;
    const double* sB = sD + (hd ? N * LDA : 0);
    const double* sM = sB + N * LDB;
    const double* sR = sM + (hm ? N * LDB : 0);
    const int r = gl < N ? gl : 0;
    unsigned long long row[4] = {0ull, 0ull, 0ull, 0ull};
    // constraint row r entering j
    {
      const size_t tr = (size_t)j * N + r;
      FF s{0.f, 0.f};
      ff_add(s, a.c[tr]);
      ff_add2(s, -f.xh[tr], -f.xl[tr]);
      float rs = 1.f;
      if (hd) rs += ff_dot<N, 1>(s, sD + r * LDA, vyh, vyl, -1.f);
      if (has_p) {
        rs += ff_dot<N, 1>(s, sA + r * LDA, vxh, vxl);
        rs += ff_dot<M, 1>(s, sB + r * LDB, vuh, vul);
      }
      const double out = ff_value(s);
      if (valid && gl < N) a.res_c[tr] = out;
      if (gl < N) {
        row[0] = abits(out);
        row[3] = ks ? abits(f2d_bits(rs)) : 0ull;
      }
    }
    // control rows of the edge into j: P = G / M lanes per row, each summing
    // every P-th term, then a float-float reduction over those P lanes
    {
      constexpr int P = G / M;
      static_assert(P * M == G, "M must divide the group size");
      const int ua = gl / P, part = gl - ua * P;
      FF s{0.f, 0.f};
      float rs = 0.f;
      if (has_p) {
#pragma unroll
        for (int k = 0; k < (N + P - 1) / P; ++k) {
          const int b = part + k * P;
          if (b < N) {
            if (hm) rs += ff_fma_d(s, sM[b * LDB + ua], vxh[b], vxl[b]);
            rs += ff_fma_d(s, sB[b * LDB + ua], vyh[b], vyl[b]);
          }
        }
#pragma unroll
        for (int k = 0; k < (M + P - 1) / P; ++k) {
          const int c = part + k * P;
          if (c < M) rs += ff_fma_d(s, sR[ua * LDB + c], vuh[c], vul[c]);
        }
        if (part == 0) ff_add(s, a.r[(size_t)j * M + ua]);
      }
#pragma unroll
      for (int off = P / 2; off; off >>= 1) {
        const float oh = __shfl_xor_sync(TLQR_FULL_MASK, s.h, off, P);
        const float ol = __shfl_xor_sync(TLQR_FULL_MASK, s.l, off, P);
        rs += __shfl_xor_sync(TLQR_FULL_MASK, rs, off, P);
        ff_add2(s, oh, ol);
      }
      if (part == 0) {
        const size_t tu = (size_t)j * M + ua;
        if (has_p) {
          const double out = ff_value(s);
          if (valid) a.res_u[tu] = out;
          const unsigned long long ob = abits(out), kb = ks ? abits(f2d_bits(rs)) : 0ull;
          row[0] = ob > row[0] ? ob : row[0];
          row[3] = kb > row[3] ? kb : row[3];
        } else if (valid) {
          a.res_u[tu] = 0.0;
        }
      }
    }
    // message w_j = A_j^T y_j + M_j u_j to the parent's stationarity rows
    if (has_p && gl < N) {
      FF wv{0.f, 0.f};
      float wk = ff_dot<N, LDA>(wv, sA + r, vyh, vyl);
      if (hm) wk += ff_dot<M, 1>(wv, sM + r * LDB, vuh, vul);
      if (valid) {
        na.wh[(size_t)j * N + r] = wv.h;
        na.wl[(size_t)j * N + r] = wv.l;
        if (ks) na.wk[(size_t)j * N + r] = wk;
      }
    }
    // ||z|| and ||b||: u_j, r_j (edge) and x_j, y_j, q_j, c_j (node) entries of this node
    {
      double zv = 0.0, bv = 0.0;
      if (gl < N) {
        const size_t tr = (size_t)j * N + gl;
        zv = amax(amax(0.0, a.x[tr]), a.y[tr]);
        bv = fmax(fabs(a.q[tr]), fabs(a.c[tr]));
      }
      if (has_p && gl < M) {
        zv = amax(zv, a.u[(size_t)j * M + gl]);
        bv = fmax(bv, fabs(a.r[(size_t)j * M + gl]));
      }
      row[1] = dbits_abs(zv);
      row[2] = dbits_abs(bv);
    }
    if constexpr (FOREST) {
      acc.add(a, ks ? 4 : 3, valid, valid ? a.tree[j] : -1, row);
    } else if (valid) {
      mx.take(row);
    }
    __syncwarp();                                        // buffer and vectors free for reuse
  }
  cp_async_wait<0>();
  if constexpr (FOREST) {
    acc.flush(a, ks ? 4 : 3);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < 3 || ks) block_maxbits_to(a.maxes + q, mx.v[q]);
  }
}

template <int N>
struct NodeBuf {
  static constexpr int LDQ = N + 1;
  static constexpr int doubles = N * LDQ;
  static constexpr int group_bytes = ((2 * doubles * 8 + 2 * N * 4) + 15) / 16 * 16;
};

// Node pass: stationarity rows Q_i x_i + q_i - y_i + sum_children w_j.
template <int N, bool FOREST>
__global__ void __launch_bounds__(128) k_res_node(ResidualArgs a, FFArgs f, NodeArgs na) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using NB = NodeBuf<N>;
  constexpr int G = RG<N>::G, OPS = RG<N>::OPS, LDQ = NB::LDQ;
  const int gl = threadIdx.x & (G - 1), gid = (threadIdx.x & 31) / G;
  unsigned char* gbase = smem_raw + (size_t)((threadIdx.x >> 5) * OPS + gid) * NB::group_bytes;
  double* buf0 = reinterpret_cast<double*>(gbase);
  float* vxh = reinterpret_cast<float*>(gbase + 2 * (size_t)NB::doubles * 8);
  float* vxl = vxh + N;
  const bool ks = a.with_knorm;
  const NodeRange nr = warp_nodes<OPS>(a.N);
  Maxima mx;
  TreeAcc acc;
  if (nr.begin < nr.end) {
    const int i0 = nr.begin + gid < nr.end ? nr.begin + gid : nr.end - 1;
    stage_async<N, N, LDQ, G>(buf0, a.Q + (size_t)i0 * N * N, gl);
  }
  cp_async_commit();
  int t = 0;
  for (int base = nr.begin; base < nr.end; base += OPS, ++t) {
    const int i0 = base + gid;
    const bool valid = i0 < nr.end;
    const int i = valid ? i0 : nr.end - 1;
    const double* sQ = buf0 + (t & 1) * NB::doubles;
    if (base + OPS < nr.end) {
      const int in = base + OPS + gid < nr.end ? base + OPS + gid : nr.end - 1;
      stage_async<N, N, LDQ, G>(buf0 + ((t + 1) & 1) * NB::doubles, a.Q + (size_t)in * N * N, gl);
    }
    cp_async_commit();
    cp_async_wait<1>();
    if (gl < N) {
      vxh[gl] = f.xh[(size_t)i * N + gl];
      vxl[gl] = f.xl[(size_t)i * N + gl];
    }
    __syncwarp();
    const int r = gl < N ? gl : 0;
    const size_t tr = (size_t)i * N + r;
    FF s{0.f, 0.f};
    ff_add(s, a.q[tr]);
    ff_add2(s, -f.yh[tr], -f.yl[tr]);
    float rs = 1.f + ff_dot<N, 1>(s, sQ + r * LDQ, vxh, vxl);
    for (int k = a.child_start[i]; k < a.child_start[i + 1]; ++k) {
      const int jc = a.child_list[k];
      ff_add2(s, na.wh[(size_t)jc * N + r], na.wl[(size_t)jc * N + r]);
      if (ks) rs += na.wk[(size_t)jc * N + r];
    }
    const double out = ff_value(s);
    if (valid && gl < N) a.res_x[tr] = out;
    unsigned long long row[4] = {0ull, 0ull, 0ull, 0ull};
    if (gl < N) {
      row[0] = abits(out);
      row[3] = ks ? abits(f2d_bits(rs)) : 0ull;
    }
    if constexpr (FOREST) {
      acc.add(a, ks ? 4 : 3, valid, valid ? a.tree[i] : -1, row);
    } else if (valid) {
      mx.take(row);
    }
    __syncwarp();
  }
  cp_async_wait<0>();
  if constexpr (FOREST) {
    acc.flush(a, ks ? 4 : 3);
  } else {
    block_maxbits_to(a.maxes + 0, mx.v[0]);
    if (ks) block_maxbits_to(a.maxes + 3, mx.v[3]);
  }
}

}  // namespace rn
}  // namespace tlqr
