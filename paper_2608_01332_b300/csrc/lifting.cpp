// Node-control lifting and projection (Prop. 2, Sec. III-B), host side.
//
// A node-control problem (one control v_i per nonterminal node, shared by all
// outgoing transitions, eq. (node-control)) becomes an edge-control problem with
// state s = (x, v) of size n + m:
//   * every node i keeps a predecision copy i- (same label i) carrying the state
//     cost diag(Q_i, 0), q = (q_i, 0), the constraint data c = (c_i, 0) and
//     Delta = diag(Delta_i, 0) of the transition entering it;
//   * every nonterminal i gets a decision copy i+ (labels N, N+1, ... in
//     increasing i), child of i-, reached through the decision edge
//     eq. (decision-edge): A = [[I,0],[0,0]], B = [[0],[I]], with the original
//     control cost M = [M_i; 0], R_i, r_i and zero node data;
//   * every uncertainty edge (i, j) becomes i+ -> j- eq. (uncertainty-edge):
//     A = [[A_ij, B_ij],[0,0]], B = 0 with a dummy control of cost R = I, r = 0.
#include <cstring>
#include <vector>

#include "../../include/tlqr.h"

extern "C" int tlqr_lift_node_controls(const int32_t* parent, int32_t N, int32_t n, int32_t m,
                                       const double* Q, const double* q, const double* Mv,
                                       const double* Rv, const double* rv, const double* Av,
                                       const double* Bv, const double* c, const double* Delta,
                                       int32_t* Nl, int32_t* lifted_parent, double* lQ, double* lq,
                                       double* lM, double* lR, double* lr, double* lA, double* lB,
                                       double* lc, double* lDelta, int32_t* map) {
  if (!parent || N < 1 || n < 1 || m < 1 || !Nl) return TLQR_ERR_ARG;
  int root = -1;
  std::vector<char> nonterm(N, 0);
  for (int j = 0; j < N; ++j) {
    const int p = parent[j];
    if (p == -1) {
      if (root >= 0) return TLQR_ERR_TOPOLOGY;
      root = j;
    } else if (p < 0 || p >= N || p == j) {
      return TLQR_ERR_TOPOLOGY;
    } else {
      nonterm[p] = 1;
    }
  }
  if (root < 0) return TLQR_ERR_TOPOLOGY;
  std::vector<int32_t> plus(N, -1);
  int L = N;
  for (int i = 0; i < N; ++i) if (nonterm[i]) plus[i] = L++;
  *Nl = L;
  if (!lifted_parent) return TLQR_OK;   // size query
  if (!Q || !q || !Mv || !Rv || !rv || !Av || !Bv || !c || !lQ || !lq || !lM || !lR || !lr || !lA ||
      !lB || !lc || !lDelta || !map)
    return TLQR_ERR_ARG;
  const size_t s = (size_t)n + m, ss = s * s, sm = s * m, nn = (size_t)n * n, nm = (size_t)n * m,
               mm = (size_t)m * m;
  std::memset(lQ, 0, sizeof(double) * L * ss);
  std::memset(lq, 0, sizeof(double) * L * s);
  std::memset(lM, 0, sizeof(double) * L * sm);
  std::memset(lR, 0, sizeof(double) * L * mm);
  std::memset(lr, 0, sizeof(double) * L * m);
  std::memset(lA, 0, sizeof(double) * L * ss);
  std::memset(lB, 0, sizeof(double) * L * sm);
  std::memset(lc, 0, sizeof(double) * L * s);
  std::memset(lDelta, 0, sizeof(double) * L * ss);
  for (int i = 0; i < N; ++i) {
    // predecision node i-: state cost, constraint entering it
    for (int a = 0; a < n; ++a) {
      for (int b = 0; b < n; ++b) {
        lQ[i * ss + a * s + b] = Q[i * nn + a * n + b];
        if (Delta) lDelta[i * ss + a * s + b] = Delta[i * nn + a * n + b];
      }
      lq[i * s + a] = q[i * n + a];
      lc[i * s + a] = c[i * n + a];
    }
    map[i] = i;
    map[N + i] = plus[i];
    if (parent[i] >= 0) {
      // uncertainty edge parent(i)+ -> i-, indexed by the child i-
      lifted_parent[i] = plus[parent[i]];
      for (int a = 0; a < n; ++a) {
        for (int b = 0; b < n; ++b) lA[i * ss + a * s + b] = Av[i * nn + a * n + b];
        for (int b = 0; b < m; ++b) lA[i * ss + a * s + n + b] = Bv[i * nm + a * m + b];
      }
      for (int a = 0; a < m; ++a) lR[i * mm + a * m + a] = 1.0;   // dummy control, B = 0
    } else {
      lifted_parent[i] = -1;
    }
    if (plus[i] >= 0) {
      // decision edge i- -> i+, indexed by the child i+
      const int d = plus[i];
      lifted_parent[d] = i;
      for (int a = 0; a < n; ++a) lA[d * ss + a * s + a] = 1.0;
      for (int a = 0; a < m; ++a) lB[d * sm + (n + a) * m + a] = 1.0;
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < m; ++b) lM[d * sm + a * m + b] = Mv[i * nm + a * m + b];
      for (int a = 0; a < mm; ++a) lR[d * mm + a] = Rv[i * mm + a];
      for (int a = 0; a < m; ++a) lr[d * m + a] = rv[i * m + a];
    }
  }
  return TLQR_OK;
}

extern "C" int tlqr_project_lifted(int32_t N, int32_t n, int32_t m, const int32_t* map, const double* lx,
                                   const double* lu, const double* ly, double* x, double* v, double* y) {
  if (N < 1 || n < 1 || m < 1 || !map || !lx || !lu || !ly || !x || !v || !y) return TLQR_ERR_ARG;
  const size_t s = (size_t)n + m;
  for (int i = 0; i < N; ++i) {
    const int im = map[i], ip = map[N + i];
    for (int a = 0; a < n; ++a) {
      x[(size_t)i * n + a] = lx[(size_t)im * s + a];
      y[(size_t)i * n + a] = ly[(size_t)im * s + a];
    }
    for (int a = 0; a < m; ++a) v[(size_t)i * m + a] = ip >= 0 ? lu[(size_t)ip * m + a] : 0.0;
  }
  return TLQR_OK;
}
