"""ORACLE -- test infrastructure only.

Brute force: the KKT system eq. (kkt) of the edge-control problem (Sec. III-A)
assembled as one dense matrix and solved directly with LAPACK (numpy), with no
use of the tree structure.  By Prop. 1 the matrix is nonsingular under Def. 1,
so the solution is the unique saddle point.  Also the node-control problem of
eq. (node-lagrangian) (Sec. III-B) assembled the same way from its stationarity
conditions, for the lifting of Prop. 2.

Unknown ordering: x_0..x_{N-1} (n each), then u_j for every nonroot j in
increasing j (m each), then y_0..y_{N-1} (n each).
Row ordering: (kkt-x) for every node, (kkt-u) for every nonroot j, then for
every node i the constraint entering i: (kkt-root) at the root, (kkt-dyn)
elsewhere.  The system is written as  K z + b = 0  with b built from (q, r, c).
"""
from __future__ import annotations

import numpy as np


def assemble_kkt(parent, n: int, m: int, data: dict):
    parent = np.asarray(parent)
    N = len(parent)
    nonroot = [j for j in range(N) if parent[j] >= 0]
    upos = {j: k for k, j in enumerate(nonroot)}
    nx, nu = N * n, len(nonroot) * m
    dim = nx + nu + nx
    K = np.zeros((dim, dim))
    b = np.zeros(dim)
    Q, q, M, R, r = data["Q"], data["q"], data.get("M"), data["R"], data["r"]
    A, B, c, D = data["A"], data["B"], data["c"], data.get("Delta")
    X = lambda i: slice(i * n, (i + 1) * n)
    U = lambda j: slice(nx + upos[j] * m, nx + (upos[j] + 1) * m)
    Y = lambda i: slice(nx + nu + i * n, nx + nu + (i + 1) * n)
    I = np.eye(n)
    for i in range(N):
        # (kkt-x): Q_i x_i + q_i - y_i + sum_children (M_e u_e + A_e^T y_j) = 0
        K[X(i), X(i)] += Q[i]
        K[X(i), Y(i)] += -I
        b[X(i)] += q[i]
    for j in nonroot:
        i = parent[j]
        if M is not None:
            K[X(i), U(j)] += M[j]
        K[X(i), Y(j)] += A[j].T
        # (kkt-u): M^T x_i + R u + r + B^T y_j = 0
        if M is not None:
            K[U(j), X(i)] += M[j].T
        K[U(j), U(j)] += R[j]
        K[U(j), Y(j)] += B[j].T
        b[U(j)] += r[j]
        # (kkt-dyn): A x_i + B u + c_j - x_j - Delta_j y_j = 0
        K[Y(j), X(i)] += A[j]
        K[Y(j), U(j)] += B[j]
        K[Y(j), X(j)] += -I
        if D is not None:
            K[Y(j), Y(j)] += -D[j]
        b[Y(j)] += c[j]
    # (kkt-root): c_rho - x_rho - Delta_rho y_rho = 0, for every root (a forest is a batch)
    for root in np.nonzero(parent < 0)[0]:
        root = int(root)
        K[Y(root), X(root)] += -I
        if D is not None:
            K[Y(root), Y(root)] += -D[root]
        b[Y(root)] += c[root]
    return K, b, (X, U, Y, nonroot)


def dense_solve(parent, n: int, m: int, data: dict) -> dict:
    """Unique solution of eq. (kkt) by a dense LU solve (numpy.linalg.solve)."""
    K, b, (X, U, Y, nonroot) = assemble_kkt(parent, n, m, data)
    z = np.linalg.solve(K, -b)
    N = len(parent)
    x = np.stack([z[X(i)] for i in range(N)])
    y = np.stack([z[Y(i)] for i in range(N)])
    u = np.zeros((N, m))
    for j in nonroot:
        u[j] = z[U(j)]
    return dict(x=x, u=u, y=y, K=K, b=b)


def assemble_node_control(parent, n: int, m: int, nd: dict):
    """Stationarity system of the node-control saddle function eq. (node-lagrangian).

    nd holds Q (N,n,n), q (N,n), Mv (N,n,m), Rv (N,m,m), rv (N,m) for every
    node (used only at nonterminal nodes), Av (N,n,n), Bv (N,n,m) indexed by
    the child j of each uncertainty edge (i,j), c (N,n), Delta (N,n,n) or None.
    Unknowns: x_i (all nodes), v_i (nonterminal nodes, increasing i), y_i.
    """
    parent = np.asarray(parent)
    N = len(parent)
    has_child = np.zeros(N, dtype=bool)
    for j in range(N):
        if parent[j] >= 0:
            has_child[parent[j]] = True
    nonterm = [i for i in range(N) if has_child[i]]
    vpos = {i: k for k, i in enumerate(nonterm)}
    nx, nv = N * n, len(nonterm) * m
    dim = nx + nv + nx
    K = np.zeros((dim, dim))
    b = np.zeros(dim)
    X = lambda i: slice(i * n, (i + 1) * n)
    V = lambda i: slice(nx + vpos[i] * m, nx + (vpos[i] + 1) * m)
    Y = lambda i: slice(nx + nv + i * n, nx + nv + (i + 1) * n)
    I = np.eye(n)
    D = nd.get("Delta")
    for i in range(N):
        K[X(i), X(i)] += nd["Q"][i]
        K[X(i), Y(i)] += -I
        b[X(i)] += nd["q"][i]
        if has_child[i]:
            # d/dx_i of x_i^T M_i v_i ; d/dv_i of the control terms
            K[X(i), V(i)] += nd["Mv"][i]
            K[V(i), X(i)] += nd["Mv"][i].T
            K[V(i), V(i)] += nd["Rv"][i]
            b[V(i)] += nd["rv"][i]
    for j in range(N):
        i = parent[j]
        if i < 0:
            K[Y(j), X(j)] += -I
            if D is not None:
                K[Y(j), Y(j)] += -D[j]
            b[Y(j)] += nd["c"][j]
            continue
        Aij, Bij = nd["Av"][j], nd["Bv"][j]
        K[X(i), Y(j)] += Aij.T
        K[V(i), Y(j)] += Bij.T
        K[Y(j), X(i)] += Aij
        K[Y(j), V(i)] += Bij
        K[Y(j), X(j)] += -I
        if D is not None:
            K[Y(j), Y(j)] += -D[j]
        b[Y(j)] += nd["c"][j]
    return K, b, (X, V, Y, nonterm)


def dense_solve_node_control(parent, n: int, m: int, nd: dict) -> dict:
    K, b, (X, V, Y, nonterm) = assemble_node_control(parent, n, m, nd)
    z = np.linalg.solve(K, -b)
    N = len(parent)
    x = np.stack([z[X(i)] for i in range(N)])
    y = np.stack([z[Y(i)] for i in range(N)])
    v = np.zeros((N, m))
    for i in nonterm:
        v[i] = z[V(i)]
    return dict(x=x, v=v, y=y)
