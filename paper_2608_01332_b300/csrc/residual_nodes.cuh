// Float-float KKT residual of eq. (kkt), organised by node for compile-time
// (n, m): one group of G lanes per node, the node's FP64 blocks staged once
// into shared memory with coalesced loads and split into (hi, lo) FP32 pairs
// there, lane r owning row r.  Every FP64 matrix entry is read from HBM
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
  static constexpr int LDP = N + 1;           // padded row stride (conflict-free rows and columns)
};

// Stage an R x C FP64 block (row-major, contiguous) as (hi, lo) FP32 planes
// with row stride LDS; entries are read coalesced by the group.
template <int R, int C, int LDS, int G>
__device__ __forceinline__ void stage_split(float* h, float* l, const double* src, int gl) {
#pragma unroll 4
  for (int e = gl; e < R * C; e += G) {
    const int a = e / C, b = e - (e / C) * C;
    float hh, ll;
    dsplit(src[e], hh, ll);
    h[a * LDS + b] = hh;
    l[a * LDS + b] = ll;
  }
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

// Per-lane maxima: one tree (block fold at the end) or per tree (TreeAcc).
struct Maxima {
  unsigned long long v[4] = {0ull, 0ull, 0ull, 0ull};
  __device__ __forceinline__ void take(const unsigned long long (&r)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = r[q] > v[q] ? r[q] : v[q];
  }
};

template <int N, int M>
struct EdgeSmem {
  static constexpr int LDP = RG<N>::LDP, MLD = M + 1;
  // A (hi, lo), Delta (hi, lo): N x LDP; B (hi, lo): N x MLD; M (hi, lo): N x MLD; R (hi, lo): M x MLD;
  // vectors x_p, y_j (hi, lo): N; u_j (hi, lo): M
  static constexpr int floats = 4 * N * LDP + 4 * N * MLD + 2 * M * MLD + 4 * N + 2 * M;
  static constexpr int bytes = ((floats * 4 + 15) / 16) * 16;
};

// Edge pass.  FOREST: fold maxima per tree.
template <int N, int M, bool FOREST>
__global__ void __launch_bounds__(128) k_res_edge(ResidualArgs a, FFArgs f, NodeArgs na) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using R_ = RG<N>;
  constexpr int G = R_::G, OPS = R_::OPS, LDP = R_::LDP, MLD = M + 1;
  const int gl = threadIdx.x & (G - 1), gid = (threadIdx.x & 31) / G;
  float* sm = reinterpret_cast<float*>(smem_raw + ((threadIdx.x >> 5) * OPS + gid) * EdgeSmem<N, M>::bytes);
  float *sAh = sm, *sAl = sAh + N * LDP, *sDh = sAl + N * LDP, *sDl = sDh + N * LDP;
  float *sBh = sDl + N * LDP, *sBl = sBh + N * MLD, *sMh = sBl + N * MLD, *sMl = sMh + N * MLD;
  float *sRh = sMl + N * MLD, *sRl = sRh + M * MLD;
  float *vxh = sRl + M * MLD, *vxl = vxh + N, *vyh = vxl + N, *vyl = vyh + N, *vuh = vyl + N, *vul = vuh + M;
  const bool ks = a.with_knorm;
  const NodeRange nr = warp_nodes<OPS>(a.N);
  Maxima mx;
  TreeAcc acc;
  for (int base = nr.begin; base < nr.end; base += OPS) {
    const int j0 = base + gid;
    const bool valid = j0 < nr.end;
    const int j = valid ? j0 : nr.end - 1;
    const int p = a.parent[j];
    const bool has_p = p >= 0;
    const size_t nn = (size_t)N * N, nm = (size_t)N * M;
    // stage this node's blocks
    if (has_p) {
      stage_split<N, N, LDP, G>(sAh, sAl, a.A + (size_t)j * nn, gl);
      stage_split<N, M, MLD, G>(sBh, sBl, a.B + (size_t)j * nm, gl);
      stage_split<M, M, MLD, G>(sRh, sRl, a.R + (size_t)j * M * M, gl);
      if (a.M) stage_split<N, M, MLD, G>(sMh, sMl, a.M + (size_t)j * nm, gl);
    }
    if (a.Delta) stage_split<N, N, LDP, G>(sDh, sDl, a.Delta + (size_t)j * nn, gl);
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
    const int r = gl < N ? gl : 0;
    unsigned long long row[4] = {0ull, 0ull, 0ull, 0ull};
    // constraint row r entering j
    {
      const size_t t = (size_t)j * N + r;
      FF s{0.f, 0.f};
      ff_add(s, a.c[t]);
      ff_add2(s, -f.xh[t], -f.xl[t]);
      float rs = 1.f;
      if (a.Delta) {
#pragma unroll 8
        for (int b = 0; b < N; ++b) {
          ff_fma2(s, sDh[r * LDP + b], sDl[r * LDP + b], -vyh[b], -vyl[b]);
          rs += fabsf(sDh[r * LDP + b]);
        }
      }
      if (has_p) {
#pragma unroll 8
        for (int b = 0; b < N; ++b) {
          ff_fma2(s, sAh[r * LDP + b], sAl[r * LDP + b], vxh[b], vxl[b]);
          rs += fabsf(sAh[r * LDP + b]);
        }
#pragma unroll
        for (int c = 0; c < M; ++c) {
          ff_fma2(s, sBh[r * MLD + c], sBl[r * MLD + c], vuh[c], vul[c]);
          rs += fabsf(sBh[r * MLD + c]);
        }
      }
      const double out = ff_value(s);
      if (valid && gl < N) a.res_c[t] = out;
      if (gl < N) {
        row[0] = abits(out);
        row[3] = ks ? abits(f2d_bits(rs)) : 0ull;
      }
    }
    // control row gl of the edge into j (lanes gl < M), and the message w_j
    {
      unsigned long long ur = 0ull, uk = 0ull;
      if (has_p && gl < M) {
        const size_t tu = (size_t)j * M + gl;
        FF s{0.f, 0.f};
        ff_add(s, a.r[tu]);
        float rs = 0.f;
        if (a.M) {
#pragma unroll 8
          for (int b = 0; b < N; ++b) {
            ff_fma2(s, sMh[b * MLD + gl], sMl[b * MLD + gl], vxh[b], vxl[b]);
            rs += fabsf(sMh[b * MLD + gl]);
          }
        }
#pragma unroll
        for (int c = 0; c < M; ++c) {
          ff_fma2(s, sRh[gl * MLD + c], sRl[gl * MLD + c], vuh[c], vul[c]);
          rs += fabsf(sRh[gl * MLD + c]);
        }
#pragma unroll 8
        for (int b = 0; b < N; ++b) {
          ff_fma2(s, sBh[b * MLD + gl], sBl[b * MLD + gl], vyh[b], vyl[b]);
          rs += fabsf(sBh[b * MLD + gl]);
        }
        const double out = ff_value(s);
        if (valid) a.res_u[tu] = out;
        ur = abits(out);
        uk = ks ? abits(f2d_bits(rs)) : 0ull;
      } else if (!has_p && gl < M && valid) {
        a.res_u[(size_t)j * M + gl] = 0.0;
      }
      row[0] = ur > row[0] ? ur : row[0];
      row[3] = uk > row[3] ? uk : row[3];
      if (has_p && gl < N) {
        FF wv{0.f, 0.f};
        float wk = 0.f;
#pragma unroll 8
        for (int b = 0; b < N; ++b) {
          ff_fma2(wv, sAh[b * LDP + r], sAl[b * LDP + r], vyh[b], vyl[b]);
          wk += fabsf(sAh[b * LDP + r]);
        }
        if (a.M) {
#pragma unroll
          for (int c = 0; c < M; ++c) {
            ff_fma2(wv, sMh[r * MLD + c], sMl[r * MLD + c], vuh[c], vul[c]);
            wk += fabsf(sMh[r * MLD + c]);
          }
        }
        if (valid) {
          na.wh[(size_t)j * N + r] = wv.h;
          na.wl[(size_t)j * N + r] = wv.l;
          if (ks) na.wk[(size_t)j * N + r] = wk;
        }
      }
    }
    // ||z|| and ||b||: u_j, r_j (edge) and x_j, y_j, q_j, c_j (node) entries of this node
    {
      double zv = 0.0, bv = 0.0;
      if (gl < N) {
        const size_t t = (size_t)j * N + gl;
        zv = amax(amax(0.0, a.x[t]), a.y[t]);
        bv = fmax(fabs(a.q[t]), fabs(a.c[t]));
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
    __syncwarp();
  }
  if constexpr (FOREST) {
    acc.flush(a, ks ? 4 : 3);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < 3 || ks) block_maxbits_to(a.maxes + q, mx.v[q]);
  }
}

template <int N>
struct NodeSmem {
  static constexpr int LDP = RG<N>::LDP;
  static constexpr int floats = 2 * N * LDP + 2 * N;      // Q (hi, lo), x_i (hi, lo)
  static constexpr int bytes = ((floats * 4 + 15) / 16) * 16;
};

// Node pass: stationarity rows Q_i x_i + q_i - y_i + sum_children w_j.
template <int N, bool FOREST>
__global__ void __launch_bounds__(128) k_res_node(ResidualArgs a, FFArgs f, NodeArgs na) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using R_ = RG<N>;
  constexpr int G = R_::G, OPS = R_::OPS, LDP = R_::LDP;
  const int gl = threadIdx.x & (G - 1), gid = (threadIdx.x & 31) / G;
  float* sm = reinterpret_cast<float*>(smem_raw + ((threadIdx.x >> 5) * OPS + gid) * NodeSmem<N>::bytes);
  float *sQh = sm, *sQl = sQh + N * LDP, *vxh = sQl + N * LDP, *vxl = vxh + N;
  const bool ks = a.with_knorm;
  const NodeRange nr = warp_nodes<OPS>(a.N);
  Maxima mx;
  TreeAcc acc;
  for (int base = nr.begin; base < nr.end; base += OPS) {
    const int i0 = base + gid;
    const bool valid = i0 < nr.end;
    const int i = valid ? i0 : nr.end - 1;
    stage_split<N, N, LDP, G>(sQh, sQl, a.Q + (size_t)i * N * N, gl);
    if (gl < N) {
      vxh[gl] = f.xh[(size_t)i * N + gl];
      vxl[gl] = f.xl[(size_t)i * N + gl];
    }
    __syncwarp();
    const int r = gl < N ? gl : 0;
    const size_t t = (size_t)i * N + r;
    FF s{0.f, 0.f};
    ff_add(s, a.q[t]);
    ff_add2(s, -f.yh[t], -f.yl[t]);
    float rs = 1.f;
#pragma unroll 8
    for (int b = 0; b < N; ++b) {
      ff_fma2(s, sQh[r * LDP + b], sQl[r * LDP + b], vxh[b], vxl[b]);
      rs += fabsf(sQh[r * LDP + b]);
    }
    for (int k = a.child_start[i]; k < a.child_start[i + 1]; ++k) {
      const int jc = a.child_list[k];
      ff_add2(s, na.wh[(size_t)jc * N + r], na.wl[(size_t)jc * N + r]);
      if (ks) rs += na.wk[(size_t)jc * N + r];
    }
    const double out = ff_value(s);
    if (valid && gl < N) a.res_x[t] = out;
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
  if constexpr (FOREST) {
    acc.flush(a, ks ? 4 : 3);
  } else {
    block_maxbits_to(a.maxes + 0, mx.v[0]);
    if (ks) block_maxbits_to(a.maxes + 3, mx.v[3]);
  }
}

}  // namespace rn
}  // namespace tlqr
