// Float-float KKT residual of eq. (kkt), organised by node for compile-time
// (n, m): one group of G lanes per node, lane r owning row r.  Each node's
// FP64 blocks are moved into shared memory by the bulk-copy (TMA) engine: one
// lane per group issues one `cp.async.bulk` per block (contiguous, 16-byte
// aligned, a multiple of 16 bytes) that completes on an mbarrier, with two
// buffers per group so that the next node's blocks are in flight while the
// current node is computed.  Every FP64 matrix entry is read from HBM once per
// evaluation (the row-per-thread kernels of residual.cuh read A_j and B_j
// twice and walk Q by strided rows), and a node whose Delta_i is zero (the
// per-node flag the condensation records) has no Delta block copied at all.
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
//
// The node's FP64 vectors (x_j, x_parent, y_j, u_j, c_j, r_j, q_j) travel the
// same way, and each lane splits its entries into float-float pairs in shared
// memory, so no separate split pass over x, u, y is needed.
// Blocks sit in shared memory densely (a bulk copy cannot pad rows); a lane
// walks its row starting at column r and wrapping around, so that the lanes of
// a group read different banks.  Every wait on an mbarrier is bounded: a wait
// that runs out sets ST_TIMEOUT in the status word, the warp stops taking
// nodes, waits (again bounded) for the copies it has in flight and joins the
// block's final reduction.
#pragma once
#include "residual.cuh"

namespace tlqr {
namespace rn {

template <int N>
struct RG {
  static constexpr int G = N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32;
  static constexpr int OPS = 32 / G;          // nodes per warp
};

constexpr int kResStTimeout = 7;              // ST_TIMEOUT of the factor's status word

// ------------------------------------------------------------- bulk copies
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
// make initialised barriers visible to the bulk-copy engine
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// the one arrival of a phase, announcing `bytes` of copies that complete on it
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared bulk copy (dst, src 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait until the phase of parity `parity` has completed; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int limit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_test(bar, parity)) return true;
  return false;
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
// The same over a dense row, visiting columns c0, c0 + 1, ..., wrapping at K.
template <int K>
__device__ __forceinline__ float ff_dot_row(FF& s, const double* a, const float* xh, const float* xl, int c0,
                                            float sign = 1.f) {
  FF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  float rs = 0.f;
  int c = c0;
#pragma unroll
  for (int b = 0; b < K; ++b) {
    rs += ff_fma_d(acc[b & 3], a[c], sign * xh[c], sign * xl[c]);
    c = c + 1 == K ? 0 : c + 1;
  }
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
  float *wh, *wl;              // [N][n] float-float message w_j to the parent row
  float* wk;                   // [N][n] absolute column sums of [A_j^T | M_j] (when with_knorm)
  const unsigned char* dflag;  // per node: Delta_i has a nonzero entry (null: every Delta_i is read)
  int* status;                 // ST_TIMEOUT when a bounded wait ran out (null: not reported)
  int spin;                    // polls of one mbarrier wait before it gives up
  int withhold;                // testing failure detection: the first group of the grid
                               // announces its first node's bytes but copies nothing, so
                               // that wait runs out
};

struct Maxima {
  unsigned long long v[4] = {0ull, 0ull, 0ull, 0ull};
  __device__ __forceinline__ void take(const unsigned long long (&r)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = r[q] > v[q] ? r[q] : v[q];
  }
};

// Group of the edge pass in shared memory: two mbarriers (16 bytes), two
// buffers [A | Delta | B | M | R | x_j x_p y_j c_j q_j (N each) u_j r_j (M each)]
// of dense FP64 blocks and vectors, then the float-float vectors x_p, y_j (N
// each) and u_j (M), hi and lo.  With n and m even every block and vector is a
// multiple of 16 bytes, so each starts 16-byte aligned.
template <int N, int M>
struct EdgeBuf {
  static_assert(N % 2 == 0 && M % 2 == 0, "bulk copies need 16-byte multiples");
  __host__ __device__ static constexpr int mats(bool has_delta, bool has_M) {
    return N * N * (has_delta ? 2 : 1) + N * M * (has_M ? 2 : 1) + M * M;
  }
  __host__ __device__ static constexpr int doubles(bool has_delta, bool has_M) {
    return mats(has_delta, has_M) + 5 * N + 2 * M;
  }
  __host__ __device__ static constexpr int group_bytes(bool has_delta, bool has_M) {
    return 16 + 2 * doubles(has_delta, has_M) * 8 + ((4 * N + 2 * M) * 4 + 15) / 16 * 16;
  }
};

__device__ __forceinline__ void report_timeout(int* status) {
  if (status && (threadIdx.x & 31) == 0) atomicCAS(status, 0, kResStTimeout);
}

// Edge pass.  FOREST: fold maxima per tree.
template <int N, int M, bool FOREST>
__global__ void __launch_bounds__(128) k_res_edge(ResidualArgs a, FFArgs f, NodeArgs na) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using EB = EdgeBuf<N, M>;
  constexpr int G = RG<N>::G, OPS = RG<N>::OPS;
  constexpr unsigned kA = N * N * 8, kB = N * M * 8, kR = M * M * 8, kN = N * 8, kM = M * 8;
  const bool hd = a.Delta != nullptr, hm = a.M != nullptr, ks = a.with_knorm;
  const int gl = threadIdx.x & (G - 1), gid = (threadIdx.x & 31) / G;
  const int nd = EB::doubles(hd, hm), nmat = EB::mats(hd, hm);
  unsigned char* gbase = smem_raw + (size_t)((threadIdx.x >> 5) * OPS + gid) * EB::group_bytes(hd, hm);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(gbase);
  double* buf0 = reinterpret_cast<double*>(gbase + 16);
  float* vxh = reinterpret_cast<float*>(gbase + 16 + 2 * (size_t)nd * 8);
  float *vxl = vxh + N, *vyh = vxl + N, *vyl = vyh + N, *vuh = vyl + N, *vul = vuh + M;
  const size_t nn = (size_t)N * N, nm = (size_t)N * M;
  // block slots of buffer b: A, Delta, B, M, R
  auto slot = [&](int b, int which) -> double* {
    double* p = buf0 + (size_t)b * nd;
    if (which == 0) return p;
    p += N * N;
    if (which == 1) return p;
    if (hd) p += N * N;
    if (which == 2) return p;
    p += N * M;
    if (which == 3) return p;
    if (hm) p += N * M;
    return p;
  };
  auto has_delta = [&](int j) { return hd && (!na.dflag || na.dflag[j]); };
  // lane 0 of the group: the copies of node j's blocks into buffer b
  // vectors of buffer b: x_j, x_p, y_j, c_j, q_j (N each), u_j, r_j (M each)
  auto vslot = [&](int b) -> double* { return buf0 + (size_t)b * nd + nmat; };
  auto issue = [&](int j, int b, bool first) {
    if (gl != 0) return;
    const int p = a.parent[j];
    const bool hp = p >= 0, dz = has_delta(j);
    const unsigned bytes = (hp ? kA + kB + kR + (hm ? kB : 0u) + kN : 0u) + (dz ? kA : 0u) + 4 * kN + 2 * kM;
    mbar_expect(bar + b, bytes);
    if (na.withhold && blockIdx.x == 0 && threadIdx.x == 0 && first) return;
    if (hp) {
      bulk_load(slot(b, 0), a.A + (size_t)j * nn, kA, bar + b);
      bulk_load(slot(b, 2), a.B + (size_t)j * nm, kB, bar + b);
      bulk_load(slot(b, 4), a.R + (size_t)j * M * M, kR, bar + b);
      if (hm) bulk_load(slot(b, 3), a.M + (size_t)j * nm, kB, bar + b);
    }
    if (dz) bulk_load(slot(b, 1), a.Delta + (size_t)j * nn, kA, bar + b);
    double* v = vslot(b);
    bulk_load(v, a.x + (size_t)j * N, kN, bar + b);
    if (hp) bulk_load(v + N, a.x + (size_t)p * N, kN, bar + b);
    bulk_load(v + 2 * N, a.y + (size_t)j * N, kN, bar + b);
    bulk_load(v + 3 * N, a.c + (size_t)j * N, kN, bar + b);
    bulk_load(v + 4 * N, a.q + (size_t)j * N, kN, bar + b);
    bulk_load(v + 5 * N, a.u + (size_t)j * M, kM, bar + b);
    bulk_load(v + 5 * N + M, a.r + (size_t)j * M, kM, bar + b);
  };
  if (gl == 0) {
    mbar_init(bar);
    mbar_init(bar + 1);
    mbar_init_fence();
  }
  __syncwarp();
  const NodeRange nr = warp_nodes<OPS>(a.N);
  Maxima mx;
  TreeAcc acc;
  unsigned par = 0u;               // bit b: parity of buffer b's next phase to complete
  unsigned pend = 0u;              // bit b: copies into buffer b issued and not yet waited for
  bool timed_out = false;
  if (nr.begin < nr.end) {
    issue(nr.begin + gid < nr.end ? nr.begin + gid : nr.end - 1, 0, true);
    pend = 1u;
  }
  int t = 0;
  for (int base = nr.begin; base < nr.end; base += OPS, ++t) {
    const int cb = t & 1;
    const int j0 = base + gid;
    const bool valid = j0 < nr.end;
    const int j = valid ? j0 : nr.end - 1;
    if (base + OPS < nr.end) {                           // prefetch this group's next node
      issue(base + OPS + gid < nr.end ? base + OPS + gid : nr.end - 1, cb ^ 1, false);
      pend |= 2u >> cb;
    }
    const bool ok = mbar_wait(bar + cb, (par >> cb) & 1u, na.spin);
    if (__any_sync(TLQR_FULL_MASK, !ok)) {
      timed_out = true;
      break;
    }
    par ^= 1u << cb;
    pend &= ~(1u << cb);
    const int p = a.parent[j];
    const bool has_p = p >= 0, dz = has_delta(j);
    const double* V = vslot(cb);
    const double *vxj = V, *vxp = V + N, *vyj = V + 2 * N, *vcj = V + 3 * N, *vqj = V + 4 * N, *vuj = V + 5 * N,
                 *vrj = V + 5 * N + M;
    if (gl < N) {
      dsplit(vyj[gl], vyh[gl], vyl[gl]);
      if (has_p) {
        dsplit(vxp[gl], vxh[gl], vxl[gl]);
      } else {
        vxh[gl] = 0.f;
        vxl[gl] = 0.f;
      }
    }
    if (gl < M) dsplit(vuj[gl], vuh[gl], vul[gl]);
    __syncwarp();
    const double *sA = slot(cb, 0), *sD = slot(cb, 1), *sB = slot(cb, 2), *sM = slot(cb, 3), *sR = slot(cb, 4);
    const int r = gl < N ? gl : 0;
    unsigned long long row[4] = {0ull, 0ull, 0ull, 0ull};
    // constraint row r entering j
    {
      const size_t tr = (size_t)j * N + r;
      FF s{0.f, 0.f};
      ff_add(s, vcj[r]);
      float xh, xl;
      dsplit(vxj[r], xh, xl);
      ff_add2(s, -xh, -xl);
      float rs = 1.f;
      if (dz) rs += ff_dot_row<N>(s, sD + r * N, vyh, vyl, r, -1.f);
      if (has_p) {
        rs += ff_dot_row<N>(s, sA + r * N, vxh, vxl, r);
        rs += ff_dot<M, 1>(s, sB + r * M, vuh, vul);
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
            if (hm) rs += ff_fma_d(s, sM[b * M + ua], vxh[b], vxl[b]);
            rs += ff_fma_d(s, sB[b * M + ua], vyh[b], vyl[b]);
          }
        }
#pragma unroll
        for (int k = 0; k < (M + P - 1) / P; ++k) {
          const int c = part + k * P;
          if (c < M) rs += ff_fma_d(s, sR[ua * M + c], vuh[c], vul[c]);
        }
        if (part == 0) ff_add(s, vrj[ua]);
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
      float wk = ff_dot<N, N>(wv, sA + r, vyh, vyl);
      if (hm) wk += ff_dot<M, 1>(wv, sM + r * M, vuh, vul);
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
        zv = amax(amax(0.0, vxj[gl]), vyj[gl]);
        bv = fmax(fabs(vqj[gl]), fabs(vcj[gl]));
      }
      if (has_p && gl < M) {
        zv = amax(zv, vuj[gl]);
        bv = fmax(bv, fabs(vrj[gl]));
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
  if (timed_out) {
    report_timeout(na.status);
    // the shared memory of copies still in flight must outlive them
    for (int b = 0; b < 2; ++b)
      if ((pend >> b) & 1u) mbar_wait(bar + b, (par >> b) & 1u, na.spin);
  }
  if constexpr (FOREST) {
    acc.flush(a, ks ? 4 : 3);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < 3 || ks) block_maxbits_to(a.maxes + q, mx.v[q]);
  }
}

// Group of the node pass: two mbarriers, two buffers [Q | x_i q_i y_i] (FP64),
// x_i (hi, lo).
template <int N>
struct NodeBuf {
  static_assert(N % 2 == 0, "bulk copies need 16-byte multiples");
  static constexpr int doubles = N * N + 3 * N;
  static constexpr int group_bytes = 16 + 2 * doubles * 8 + (2 * N * 4 + 15) / 16 * 16;
};

// Node pass: stationarity rows Q_i x_i + q_i - y_i + sum_children w_j.
template <int N, bool FOREST>
__global__ void __launch_bounds__(128) k_res_node(ResidualArgs a, FFArgs f, NodeArgs na) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using NB = NodeBuf<N>;
  constexpr int G = RG<N>::G, OPS = RG<N>::OPS;
  constexpr unsigned kQ = N * N * 8, kN = N * 8;
  const int gl = threadIdx.x & (G - 1), gid = (threadIdx.x & 31) / G;
  unsigned char* gbase = smem_raw + (size_t)((threadIdx.x >> 5) * OPS + gid) * NB::group_bytes;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(gbase);
  double* buf0 = reinterpret_cast<double*>(gbase + 16);
  float* vxh = reinterpret_cast<float*>(gbase + 16 + 2 * (size_t)NB::doubles * 8);
  float* vxl = vxh + N;
  const bool ks = a.with_knorm;
  auto issue = [&](int i, int b, bool first) {
    if (gl != 0) return;
    mbar_expect(bar + b, kQ + 3 * kN);
    if (na.withhold && blockIdx.x == 0 && threadIdx.x == 0 && first) return;
    double* q = buf0 + (size_t)b * NB::doubles;
    bulk_load(q, a.Q + (size_t)i * N * N, kQ, bar + b);
    bulk_load(q + N * N, a.x + (size_t)i * N, kN, bar + b);
    bulk_load(q + N * N + N, a.q + (size_t)i * N, kN, bar + b);
    bulk_load(q + N * N + 2 * N, a.y + (size_t)i * N, kN, bar + b);
  };
  if (gl == 0) {
    mbar_init(bar);
    mbar_init(bar + 1);
    mbar_init_fence();
  }
  __syncwarp();
  const NodeRange nr = warp_nodes<OPS>(a.N);
  Maxima mx;
  TreeAcc acc;
  unsigned par = 0u, pend = 0u;
  bool timed_out = false;
  if (nr.begin < nr.end) {
    issue(nr.begin + gid < nr.end ? nr.begin + gid : nr.end - 1, 0, true);
    pend = 1u;
  }
  int t = 0;
  for (int base = nr.begin; base < nr.end; base += OPS, ++t) {
    const int cb = t & 1;
    const int i0 = base + gid;
    const bool valid = i0 < nr.end;
    const int i = valid ? i0 : nr.end - 1;
    if (base + OPS < nr.end) {
      issue(base + OPS + gid < nr.end ? base + OPS + gid : nr.end - 1, cb ^ 1, false);
      pend |= 2u >> cb;
    }
    const bool ok = mbar_wait(bar + cb, (par >> cb) & 1u, na.spin);
    if (__any_sync(TLQR_FULL_MASK, !ok)) {
      timed_out = true;
      break;
    }
    par ^= 1u << cb;
    pend &= ~(1u << cb);
    const double* sQ = buf0 + (size_t)cb * NB::doubles;
    const double *vxi = sQ + N * N, *vqi = vxi + N, *vyi = vqi + N;
    if (gl < N) dsplit(vxi[gl], vxh[gl], vxl[gl]);
    __syncwarp();
    const int r = gl < N ? gl : 0;
    const size_t tr = (size_t)i * N + r;
    FF s{0.f, 0.f};
    ff_add(s, vqi[r]);
    float yh, yl;
    dsplit(vyi[r], yh, yl);
    ff_add2(s, -yh, -yl);
    float rs = 1.f + ff_dot_row<N>(s, sQ + r * N, vxh, vxl, r);
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
  if (timed_out) {
    report_timeout(na.status);
    for (int b = 0; b < 2; ++b)
      if ((pend >> b) & 1u) mbar_wait(bar + b, (par >> b) & 1u, na.spin);
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
