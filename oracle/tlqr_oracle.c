/*
 * ORACLE -- test infrastructure only.  Plain, slow, obviously correct FP64 CPU
 * reference for the branched dual-regularized LQR problem.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load this file.
 * It shares no code with the CUDA solver.
 *
 * Problem (Sec. III-A, eq. (1)-(2)): minimise over states x and edge controls u,
 * maximise over multipliers y, the saddle function of the edge-control normal
 * form.  Its unique solution (Prop. 1) satisfies the KKT system eq. (kkt):
 *   Q_i x_i + q_i - y_i + sum_{e=(i,j)} (M_e u_e + A_e^T y_j) = 0      (kkt-x)
 *   M_e^T x_i + R_e u_e + r_e + B_e^T y_j = 0                          (kkt-u)
 *   c_rho - x_rho - Delta_rho y_rho = 0                                (kkt-root)
 *   A_e x_i + B_e u_e + c_j - x_j = Delta_j y_j                        (kkt-dyn)
 *
 * Method: the sequential dual-regularized tree Riccati recursion (the
 * "CPU seq." baseline of Sec. XI-A).  It visits nodes children-before-parents
 * and uses, per edge e=(i,j), the local factor of Sec. V-C eq. (FW),
 * (factor-local), the Hessian accumulation derived in the proof of Lemma 5,
 * and the affine recursion eq. (affine-message); then the root equation
 * eq. (xroot) and the recovery eq. (recover) with the local affine solve
 * eq. (local-affine-solve), parents-before-children.
 *
 * Layout: row-major dense blocks; node arrays [N][..]; edge arrays indexed by
 * the child node [N][..] with the root slot ignored.  M and Delta may be NULL
 * (all zero).  parent[] may hold several roots: a forest is a batch of
 * independent problems, solved tree by tree.
 *
 * Factorisations: F = I + Delta P is nonsymmetric, so it is factored by LU with
 * partial pivoting; G = R + B^T W B is symmetric positive definite (Sec. V-C)
 * and is factored by Cholesky.
 *
 * Return codes: 0 ok, 1 bad topology, 2 G not positive definite,
 * 3 singular F, 4 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(r, c, ld) ((size_t)(r) * (size_t)(ld) + (size_t)(c))

/* ---------------- small dense helpers (row-major) ---------------- */

/* C[r x c] = A[r x k] * B[k x c] (+ C if acc) */
static void mm(int r, int k, int c, const double *A, const double *B, double *C, int acc) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) {
      double s = acc ? C[IDX(i, j, c)] : 0.0;
      for (int t = 0; t < k; ++t) s += A[IDX(i, t, k)] * B[IDX(t, j, c)];
      C[IDX(i, j, c)] = s;
    }
}

/* C[r x c] = A^T * B, A is [k x r], B is [k x c] */
static void mtm(int r, int k, int c, const double *A, const double *B, double *C, int acc) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) {
      double s = acc ? C[IDX(i, j, c)] : 0.0;
      for (int t = 0; t < k; ++t) s += A[IDX(t, i, r)] * B[IDX(t, j, c)];
      C[IDX(i, j, c)] = s;
    }
}

/* y[r] = A[r x c] x (+ y if acc) */
static void mv(int r, int c, const double *A, const double *x, double *y, int acc) {
  for (int i = 0; i < r; ++i) {
    double s = acc ? y[i] : 0.0;
    for (int t = 0; t < c; ++t) s += A[IDX(i, t, c)] * x[t];
    y[i] = s;
  }
}

/* y[c] = A^T x, A is [r x c] (+ y if acc) */
static void mtv(int r, int c, const double *A, const double *x, double *y, int acc) {
  for (int j = 0; j < c; ++j) {
    double s = acc ? y[j] : 0.0;
    for (int t = 0; t < r; ++t) s += A[IDX(t, j, c)] * x[t];
    y[j] = s;
  }
}

/* In-place LU with partial pivoting of an n x n matrix; piv[k] = row swapped with k. */
static int lu_factor(int n, double *a, int *piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[IDX(k, k, n)]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[IDX(i, k, n)]) > best) { best = fabs(a[IDX(i, k, n)]); p = i; }
    piv[k] = p;
    if (!(best > 0.0) || !isfinite(best)) return 3;
    if (p != k)
      for (int j = 0; j < n; ++j) { double t = a[IDX(k, j, n)]; a[IDX(k, j, n)] = a[IDX(p, j, n)]; a[IDX(p, j, n)] = t; }
    for (int i = k + 1; i < n; ++i) {
      double l = a[IDX(i, k, n)] / a[IDX(k, k, n)];
      a[IDX(i, k, n)] = l;
      for (int j = k + 1; j < n; ++j) a[IDX(i, j, n)] -= l * a[IDX(k, j, n)];
    }
  }
  return 0;
}

/* Solve (LU) X = B in place, B is [n x nrhs]. */
static void lu_solve(int n, const double *lu, const int *piv, double *b, int nrhs) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k)
      for (int j = 0; j < nrhs; ++j) { double t = b[IDX(k, j, nrhs)]; b[IDX(k, j, nrhs)] = b[IDX(piv[k], j, nrhs)]; b[IDX(piv[k], j, nrhs)] = t; }
  for (int i = 0; i < n; ++i)
    for (int t = 0; t < i; ++t)
      for (int j = 0; j < nrhs; ++j) b[IDX(i, j, nrhs)] -= lu[IDX(i, t, n)] * b[IDX(t, j, nrhs)];
  for (int i = n - 1; i >= 0; --i) {
    for (int t = i + 1; t < n; ++t)
      for (int j = 0; j < nrhs; ++j) b[IDX(i, j, nrhs)] -= lu[IDX(i, t, n)] * b[IDX(t, j, nrhs)];
    for (int j = 0; j < nrhs; ++j) b[IDX(i, j, nrhs)] /= lu[IDX(i, i, n)];
  }
}

/* Solve (LU)^T X = B in place: U^T L^T P X = B. */
static void lu_solve_t(int n, const double *lu, const int *piv, double *b, int nrhs) {
  for (int i = 0; i < n; ++i) {               /* U^T w = b (lower triangular) */
    for (int t = 0; t < i; ++t)
      for (int j = 0; j < nrhs; ++j) b[IDX(i, j, nrhs)] -= lu[IDX(t, i, n)] * b[IDX(t, j, nrhs)];
    for (int j = 0; j < nrhs; ++j) b[IDX(i, j, nrhs)] /= lu[IDX(i, i, n)];
  }
  for (int i = n - 1; i >= 0; --i)            /* L^T v = w (unit upper) */
    for (int t = i + 1; t < n; ++t)
      for (int j = 0; j < nrhs; ++j) b[IDX(i, j, nrhs)] -= lu[IDX(t, i, n)] * b[IDX(t, j, nrhs)];
  for (int k = n - 1; k >= 0; --k)            /* undo the row permutation */
    if (piv[k] != k)
      for (int j = 0; j < nrhs; ++j) { double t = b[IDX(k, j, nrhs)]; b[IDX(k, j, nrhs)] = b[IDX(piv[k], j, nrhs)]; b[IDX(piv[k], j, nrhs)] = t; }
}

/* In-place lower Cholesky G = L L^T (upper part left untouched). */
static int chol_factor(int m, double *g) {
  for (int j = 0; j < m; ++j) {
    double d = g[IDX(j, j, m)];
    for (int t = 0; t < j; ++t) d -= g[IDX(j, t, m)] * g[IDX(j, t, m)];
    if (!(d > 0.0) || !isfinite(d)) return 2;
    d = sqrt(d);
    g[IDX(j, j, m)] = d;
    for (int i = j + 1; i < m; ++i) {
      double s = g[IDX(i, j, m)];
      for (int t = 0; t < j; ++t) s -= g[IDX(i, t, m)] * g[IDX(j, t, m)];
      g[IDX(i, j, m)] = s / d;
    }
  }
  return 0;
}

/* Solve L L^T X = B in place, B is [m x nrhs]. */
static void chol_solve(int m, const double *l, double *b, int nrhs) {
  for (int i = 0; i < m; ++i) {
    for (int t = 0; t < i; ++t)
      for (int j = 0; j < nrhs; ++j) b[IDX(i, j, nrhs)] -= l[IDX(i, t, m)] * b[IDX(t, j, nrhs)];
    for (int j = 0; j < nrhs; ++j) b[IDX(i, j, nrhs)] /= l[IDX(i, i, m)];
  }
  for (int i = m - 1; i >= 0; --i) {
    for (int t = i + 1; t < m; ++t)
      for (int j = 0; j < nrhs; ++j) b[IDX(i, j, nrhs)] -= l[IDX(t, i, m)] * b[IDX(t, j, nrhs)];
    for (int j = 0; j < nrhs; ++j) b[IDX(i, j, nrhs)] /= l[IDX(i, i, m)];
  }
}

/* ---------------- topology ---------------- */

/* Breadth-first order from the roots (a forest is a batch of independent
 * trees; a single tree has one root), children visited in increasing index.
 * Returns the number of roots, or -1 when parent[] is not a forest. */
static int bfs_order(int N, const int32_t *parent, int *order, int *child_start, int *child_list) {
  int n_roots = 0;
  for (int i = 0; i < N; ++i) {
    if (parent[i] == -1) ++n_roots;
    else if (parent[i] < 0 || parent[i] >= N || parent[i] == i) return -1;
  }
  if (n_roots == 0) return -1;
  memset(child_start, 0, sizeof(int) * (N + 1));
  for (int i = 0; i < N; ++i) if (parent[i] >= 0) child_start[parent[i] + 1]++;
  for (int i = 0; i < N; ++i) child_start[i + 1] += child_start[i];
  int *fill = (int *)malloc(sizeof(int) * N);
  if (!fill) return -1;
  for (int i = 0; i < N; ++i) fill[i] = child_start[i];
  for (int j = 0; j < N; ++j) if (parent[j] >= 0) child_list[fill[parent[j]]++] = j;  /* increasing j */
  free(fill);
  int head = 0, tail = 0;
  for (int i = 0; i < N; ++i) if (parent[i] < 0) order[tail++] = i;
  while (head < tail) {
    int i = order[head++];
    for (int t = child_start[i]; t < child_start[i + 1]; ++t) order[tail++] = child_list[t];
  }
  return tail == N ? n_roots : -1;   /* a cycle leaves nodes unreached */
}

/* ---------------- the recursion ---------------- */

int oracle_tree_riccati(int32_t N, int32_t n, int32_t m, const int32_t *parent,
                        const double *Q, const double *q, const double *M, const double *R,
                        const double *r, const double *A, const double *B, const double *c,
                        const double *Delta,
                        double *x, double *u, double *y, double *P, double *K, double *p_out) {
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
  int *order = (int *)malloc(sizeof(int) * N);
  int *cs = (int *)malloc(sizeof(int) * (N + 1));
  int *cl = (int *)malloc(sizeof(int) * (N > 1 ? N : 1));
  double *Flu = (double *)malloc(sizeof(double) * nn * N);   /* LU of F_j */
  int *Fpiv = (int *)malloc(sizeof(int) * (size_t)n * N);
  double *W = (double *)malloc(sizeof(double) * nn * N);
  double *Gl = (double *)malloc(sizeof(double) * mm_ * N);   /* Cholesky of G_e */
  double *T = (double *)malloc(sizeof(double) * nn * N);
  double *p = (double *)malloc(sizeof(double) * (size_t)n * N);
  const size_t L = (size_t)(n > m ? n : m) * (size_t)(n > m ? n : m);
  double *tmp = (double *)malloc(sizeof(double) * (8 * L + 4 * (size_t)(n + m)));
  int rc = 0;
  if (!order || !cs || !cl || !Flu || !Fpiv || !W || !Gl || !T || !p || !tmp) { rc = 4; goto done; }

  if (bfs_order(N, parent, order, cs, cl) < 0) { rc = 1; goto done; }

  double *Acl = tmp, *H = Acl + L, *t1 = H + L, *t2 = t1 + L, *t3 = t2 + L, *Ft = t3 + L,
         *v1 = Ft + L, *v2 = v1 + (n + m), *v3 = v2 + (n + m), *w1 = v3 + (n + m);

  /* P_i <- Q_i, p_i <- q_i */
  memcpy(P, Q, sizeof(double) * nn * N);
  memcpy(p, q, sizeof(double) * (size_t)n * N);

  /* Backward pass: children before parents (reverse BFS order). */
  for (int oi = N - 1; oi >= 0; --oi) {
    int j = order[oi];
    const double *Pj = P + nn * j;
    double *Fj = Flu + nn * j, *Wj = W + nn * j;
    /* F_j = I + Delta_j P_j  (eq. FW) */
    if (Delta) mm(n, n, n, Delta + nn * j, Pj, Fj, 0); else memset(Fj, 0, sizeof(double) * nn);
    for (int d = 0; d < n; ++d) Fj[IDX(d, d, n)] += 1.0;
    if (lu_factor(n, Fj, Fpiv + (size_t)n * j)) { rc = 3; goto done; }
    /* W_j = P_j F_j^{-1}:  F_j^T W_j^T = P_j^T */
    for (int a = 0; a < n; ++a) for (int b = 0; b < n; ++b) Ft[IDX(a, b, n)] = Pj[IDX(b, a, n)];
    lu_solve_t(n, Fj, Fpiv + (size_t)n * j, Ft, n);
    for (int a = 0; a < n; ++a) for (int b = 0; b < n; ++b) Wj[IDX(a, b, n)] = Ft[IDX(b, a, n)];
    if (parent[j] < 0) continue;     /* a root: no entering edge */
    int i = parent[j];
    const double *Ae = A + nn * j, *Be = B + nm * j, *Re = R + mm_ * j;
    const double *Me = M ? M + nm * j : NULL;
    double *Ke = K + nm * j, *Te = T + nn * j, *Ge = Gl + mm_ * j;
    /* G_e = R_e + B^T W_j B (eq. factor-local) */
    mm(n, n, m, Wj, Be, t1, 0);              /* t1 = W B  [n x m] */
    memcpy(Ge, Re, sizeof(double) * mm_);
    mtm(m, n, m, Be, t1, Ge, 1);
    if (chol_factor(m, Ge)) { rc = 2; goto done; }
    /* H_e = B^T W_j A_e + M_e^T */
    mm(n, n, n, Wj, Ae, t2, 0);              /* t2 = W A  [n x n] */
    mtm(m, n, n, Be, t2, H, 0);
    if (Me) for (int a = 0; a < m; ++a) for (int b = 0; b < n; ++b) H[IDX(a, b, n)] += Me[IDX(b, a, m)];
    /* K_e = -G^{-1} H */
    for (size_t t = 0; t < nm; ++t) Ke[t] = -H[t];
    chol_solve(m, Ge, Ke, n);
    /* A_cl = A + B K */
    memcpy(Acl, Ae, sizeof(double) * nn);
    mm(n, m, n, Be, Ke, Acl, 1);
    /* T_e = F_j^{-1} A_cl */
    memcpy(Te, Acl, sizeof(double) * nn);
    lu_solve(n, Fj, Fpiv + (size_t)n * j, Te, n);
    /* P_i += M_e K_e + A_e^T W_j A_cl   (proof of Lemma 5) */
    double *Pi = P + nn * i;
    if (Me) mm(n, m, n, Me, Ke, Pi, 1);
    mm(n, n, n, Wj, Acl, t3, 0);
    mtm(n, n, n, Ae, t3, Pi, 1);
    /* p_i += T_e^T p_j + z_e,  z_e = K_e^T r_e + A_cl^T W_j c_j  (eq. affine-edge, affine-message) */
    double *pi = p + (size_t)n * i;
    mtv(n, n, Te, p + (size_t)n * j, pi, 1);
    mtv(m, n, Ke, r + (size_t)m * j, pi, 1);
    mv(n, n, Wj, c + (size_t)n * j, v1, 0);
    mtv(n, n, Acl, v1, pi, 1);
  }

  /* Roots: f = Delta p - c, x_rho = -F^{-1} f  (eq. xroot) */
  for (int root = 0; root < N; ++root) {
    if (parent[root] >= 0) continue;
    double *f = v1;
    if (Delta) mv(n, n, Delta + nn * root, p + (size_t)n * root, f, 0); else memset(f, 0, sizeof(double) * n);
    for (int a = 0; a < n; ++a) f[a] -= c[(size_t)n * root + a];
    lu_solve(n, Flu + nn * root, Fpiv + (size_t)n * root, f, 1);
    for (int a = 0; a < n; ++a) x[(size_t)n * root + a] = -f[a];
  }
  /* Forward pass: parents before children (BFS order). eq. (local-affine-solve), (recover) */
  for (int oi = 0; oi < N; ++oi) {
    int j = order[oi], i = parent[j];
    if (i < 0) continue;
    const double *pj = p + (size_t)n * j;
    double *f = v1, *g = v2, *bb = v3, *k = w1;
    if (Delta) mv(n, n, Delta + nn * j, pj, f, 0); else memset(f, 0, sizeof(double) * n);
    for (int a = 0; a < n; ++a) f[a] -= c[(size_t)n * j + a];
    mv(n, n, W + nn * j, f, g, 0);
    for (int a = 0; a < n; ++a) g[a] = pj[a] - g[a];
    /* k = -G^{-1}(r + B^T g) */
    for (int a = 0; a < m; ++a) k[a] = r[(size_t)m * j + a];
    mtv(n, m, B + nm * j, g, k, 1);
    chol_solve(m, Gl + mm_ * j, k, 1);
    for (int a = 0; a < m; ++a) k[a] = -k[a];
    /* b = F_j^{-1}(B k - f) */
    mv(n, m, B + nm * j, k, bb, 0);
    for (int a = 0; a < n; ++a) bb[a] -= f[a];
    lu_solve(n, Flu + nn * j, Fpiv + (size_t)n * j, bb, 1);
    /* x_j = T x_i + b, u_e = K x_i + k */
    mv(n, n, T + nn * j, x + (size_t)n * i, x + (size_t)n * j, 0);
    for (int a = 0; a < n; ++a) x[(size_t)n * j + a] += bb[a];
    mv(m, n, K + nm * j, x + (size_t)n * i, u + (size_t)m * j, 0);
    for (int a = 0; a < m; ++a) u[(size_t)m * j + a] += k[a];
  }
  for (int i = 0; i < N; ++i) {
    mv(n, n, P + nn * i, x + (size_t)n * i, y + (size_t)n * i, 0);
    for (int a = 0; a < n; ++a) y[(size_t)n * i + a] += p[(size_t)n * i + a];
  }
  for (int root = 0; root < N; ++root) {
    if (parent[root] >= 0) continue;
    memset(u + (size_t)m * root, 0, sizeof(double) * m);
    memset(K + nm * root, 0, sizeof(double) * nm);
  }
  if (p_out) memcpy(p_out, p, sizeof(double) * (size_t)n * N);

done:
  free(order); free(cs); free(cl); free(Flu); free(Fpiv); free(W); free(Gl); free(T); free(p); free(tmp);
  return rc;
}

/*
 * KKT residual blocks of eq. (kkt) and the normwise backward error
 *   eta = ||K z - b||_inf / (||K||_inf ||z||_inf + ||b||_inf),
 * where K is the KKT matrix, z = (x, u, y) and b = (q, r, c) (up to sign).
 * ||K||_inf is the largest absolute row sum, formed block row by block row.
 * res_x [N][n], res_u [N][m] (root row zero), res_c [N][n] (root row = kkt-root,
 * other rows = kkt-dyn).  stats[0] = ||res||_inf, stats[1] = eta,
 * stats[2] = ||K||_inf, stats[3] = ||z||_inf, stats[4] = ||b||_inf.
 */
int oracle_kkt_residual(int32_t N, int32_t n, int32_t m, const int32_t *parent,
                        const double *Q, const double *q, const double *M, const double *R,
                        const double *r, const double *A, const double *B, const double *c,
                        const double *Delta, const double *x, const double *u, const double *y,
                        double *res_x, double *res_u, double *res_c, double *stats) {
  const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
  double *rowsum_x = (double *)calloc((size_t)N * n, sizeof(double));
  if (!rowsum_x) return 4;
  double rmax = 0, Kmax = 0, zmax = 0, bmax = 0;
  int n_roots = 0;
  for (int i = 0; i < N; ++i) if (parent[i] < 0) ++n_roots;
  if (n_roots == 0) { free(rowsum_x); return 1; }
  /* node rows: Q x + q - y */
  for (int i = 0; i < N; ++i) {
    mv(n, n, Q + nn * i, x + (size_t)n * i, res_x + (size_t)n * i, 0);
    for (int a = 0; a < n; ++a) {
      res_x[(size_t)n * i + a] += q[(size_t)n * i + a] - y[(size_t)n * i + a];
      double s = 1.0;
      for (int b = 0; b < n; ++b) s += fabs(Q[nn * i + IDX(a, b, n)]);
      rowsum_x[(size_t)n * i + a] = s;
    }
  }
  for (int j = 0; j < N; ++j) {
    double *rc_ = res_c + (size_t)n * j;
    double *ru = res_u + (size_t)m * j;
    if (parent[j] < 0) {
      for (int a = 0; a < n; ++a) {
        double s = c[(size_t)n * j + a] - x[(size_t)n * j + a];
        double rs = 1.0;
        if (Delta) for (int b = 0; b < n; ++b) { s -= Delta[nn * j + IDX(a, b, n)] * y[(size_t)n * j + b]; rs += fabs(Delta[nn * j + IDX(a, b, n)]); }
        rc_[a] = s;
        if (rs > Kmax) Kmax = rs;
      }
      for (int a = 0; a < m; ++a) ru[a] = 0.0;
      continue;
    }
    int i = parent[j];
    const double *Ae = A + nn * j, *Be = B + nm * j, *Re = R + mm_ * j;
    const double *Me = M ? M + nm * j : NULL;
    const double *xi = x + (size_t)n * i, *xj = x + (size_t)n * j, *ue = u + (size_t)m * j, *yj = y + (size_t)n * j;
    /* parent row contributions: M u + A^T y_j */
    double *rxi = res_x + (size_t)n * i;
    if (Me) mv(n, m, Me, ue, rxi, 1);
    mtv(n, n, Ae, yj, rxi, 1);
    for (int a = 0; a < n; ++a) {
      double s = 0;
      if (Me) for (int b = 0; b < m; ++b) s += fabs(Me[IDX(a, b, m)]);
      for (int b = 0; b < n; ++b) s += fabs(Ae[IDX(b, a, n)]);
      rowsum_x[(size_t)n * i + a] += s;
    }
    /* control row: M^T x_i + R u + r + B^T y_j */
    for (int a = 0; a < m; ++a) {
      double s = r[(size_t)m * j + a], rs = 0;
      if (Me) for (int b = 0; b < n; ++b) { s += Me[IDX(b, a, m)] * xi[b]; rs += fabs(Me[IDX(b, a, m)]); }
      for (int b = 0; b < m; ++b) { s += Re[IDX(a, b, m)] * ue[b]; rs += fabs(Re[IDX(a, b, m)]); }
      for (int b = 0; b < n; ++b) { s += Be[IDX(b, a, m)] * yj[b]; rs += fabs(Be[IDX(b, a, m)]); }
      ru[a] = s;
      if (rs > Kmax) Kmax = rs;
    }
    /* dynamics row: A x_i + B u + c_j - x_j - Delta_j y_j */
    for (int a = 0; a < n; ++a) {
      double s = c[(size_t)n * j + a] - xj[a], rs = 1.0;
      for (int b = 0; b < n; ++b) { s += Ae[IDX(a, b, n)] * xi[b]; rs += fabs(Ae[IDX(a, b, n)]); }
      for (int b = 0; b < m; ++b) { s += Be[IDX(a, b, m)] * ue[b]; rs += fabs(Be[IDX(a, b, m)]); }
      if (Delta) for (int b = 0; b < n; ++b) { s -= Delta[nn * j + IDX(a, b, n)] * yj[b]; rs += fabs(Delta[nn * j + IDX(a, b, n)]); }
      rc_[a] = s;
      if (rs > Kmax) Kmax = rs;
    }
  }
  for (size_t t = 0; t < (size_t)N * n; ++t) {
    if (rowsum_x[t] > Kmax) Kmax = rowsum_x[t];
    if (fabs(res_x[t]) > rmax) rmax = fabs(res_x[t]);
    if (fabs(res_c[t]) > rmax) rmax = fabs(res_c[t]);
    if (fabs(x[t]) > zmax) zmax = fabs(x[t]);
    if (fabs(y[t]) > zmax) zmax = fabs(y[t]);
    if (fabs(q[t]) > bmax) bmax = fabs(q[t]);
    if (fabs(c[t]) > bmax) bmax = fabs(c[t]);
  }
  for (int j = 0; j < N; ++j) {
    if (parent[j] < 0) continue;
    for (int a = 0; a < m; ++a) {
      size_t t = (size_t)m * j + a;
      if (fabs(res_u[t]) > rmax) rmax = fabs(res_u[t]);
      if (fabs(u[t]) > zmax) zmax = fabs(u[t]);
      if (fabs(r[t]) > bmax) bmax = fabs(r[t]);
    }
  }
  free(rowsum_x);
  stats[0] = rmax;
  stats[1] = rmax / (Kmax * zmax + bmax);
  stats[2] = Kmax;
  stats[3] = zmax;
  stats[4] = bmax;
  return 0;
}
