"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own arithmetic: a dense direct
solve of the KKT system (Prop. 1 uniqueness), the textbook chain Riccati
recursion, a hand-derived two-node solution, invariants of Thm. 1 and Lemma 1,
and Schur complements of small saddle matrices for the per-operation formulas.
"""
import math

import numpy as np
import pytest

from oracle import dense, ops, riccati
from paper_2608_01332_b300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def small_instances():
    """The population of the paper's KKT-accuracy test (Sec. IX-A): chain, star
    and irregular trees with Delta = 0 and Delta >= 0, plus random trees with
    permuted labels; n in 1..4, m in 1..3.  M != 0 in half of them."""
    rng = inputs.rng_for(11)
    cases = []
    fixed = [("chain", inputs.chain(9)), ("star", inputs.star(8)),
             ("irregular", np.array([-1, 0, 1, 1, 2, 4, 4, 5], dtype=np.int32)),
             ("balanced", inputs.balanced(13)), ("chain2", inputs.chain(2))]
    k = 0
    for name, p in fixed:
        for delta in (None, "random"):
            n, m = 1 + k % 4, 1 + k % 3
            d = inputs.problem_data(p, n, m, rng, M_scale=0.3 if k % 2 else 0.0, delta=delta,
                                    delta_value=0.5)
            cases.append((f"{name}-{delta}-n{n}m{m}", p, n, m, d))
            k += 1
    for t in range(16):
        N = int(rng.integers(2, 31))
        p = inputs.random_recursive(N, rng)
        p, perm = inputs.permute_labels(p, rng)
        n, m = int(rng.integers(1, 5)), int(rng.integers(1, 4))
        d = inputs.problem_data(p, n, m, rng, M_scale=0.3 if t % 2 else 0.0,
                                delta=("random" if t % 3 else None), delta_value=0.3)
        cases.append((f"random{t}-N{N}-n{n}m{m}", p, n, m, d))
    return cases


CASES = small_instances()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_oracle_matches_dense_kkt(case):
    _, parent, n, m, data = case
    sol = riccati.tree_riccati(parent, n, m, data)
    ref = dense.dense_solve(parent, n, m, data)
    assert riccati.forward_error(sol, ref, parent) < 1e-11
    res = riccati.kkt_residual(parent, n, m, data, sol["x"], sol["u"], sol["y"])
    assert res["eta"] < 1e-14
    assert res["abs"] < 1e-11


@pytest.mark.parametrize("case", CASES[:12], ids=[c[0] for c in CASES[:12]])
def test_riccati_matrices_symmetric_psd(case):
    """Thm. 1: every P_i is the PSD Hessian of a subtree value function."""
    _, parent, n, m, data = case
    sol = riccati.tree_riccati(parent, n, m, data)
    for P in sol["P"]:
        scale = max(1.0, np.abs(P).max())
        assert np.abs(P - P.T).max() <= 1e-12 * scale
        assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() >= -1e-10 * scale


def test_residual_matches_dense_matrix():
    """The tree-structured residual equals K z + b of the dense KKT system for
    an arbitrary z, and ||K||_inf equals the dense max absolute row sum."""
    rng = inputs.rng_for(5)
    p = inputs.random_recursive(17, rng)
    p, _ = inputs.permute_labels(p, rng)
    n, m = 3, 2
    d = inputs.problem_data(p, n, m, rng, M_scale=0.4, delta="random", delta_value=0.2)
    N = len(p)
    x = rng.standard_normal((N, n)); y = rng.standard_normal((N, n)); u = rng.standard_normal((N, m))
    u[p < 0] = 0
    res = riccati.kkt_residual(p, n, m, d, x, u, y)
    K, b, (X, U, Y, nonroot) = dense.assemble_kkt(p, n, m, d)
    z = np.zeros(K.shape[0])
    for i in range(N):
        z[X(i)] = x[i]; z[Y(i)] = y[i]
    for j in nonroot:
        z[U(j)] = u[j]
    rz = K @ z + b
    for i in range(N):
        np.testing.assert_allclose(res["res_x"][i], rz[X(i)], atol=1e-12)
        np.testing.assert_allclose(res["res_c"][i], rz[Y(i)], atol=1e-12)
    for j in nonroot:
        np.testing.assert_allclose(res["res_u"][j], rz[U(j)], atol=1e-12)
    assert res["normK"] == pytest.approx(np.abs(K).sum(axis=1).max(), rel=1e-14)
    assert res["abs"] == pytest.approx(np.abs(rz).max(), rel=1e-12)


def test_chain_equals_textbook_riccati():
    """On a path tree with Delta = 0 the recursion is the classical discrete-time
    LQR Riccati recursion P = Q + A'PA - (A'PB + M)(R + B'PB)^{-1}(B'PA + M')."""
    rng = inputs.rng_for(7)
    N, n, m = 12, 4, 2
    p = inputs.chain(N)
    d = inputs.problem_data(p, n, m, rng, M_scale=0.3)
    sol = riccati.tree_riccati(p, n, m, d)
    Pn = d["Q"][N - 1].copy()
    np.testing.assert_allclose(sol["P"][N - 1], Pn, rtol=1e-13, atol=1e-13)
    for t in range(N - 2, -1, -1):
        A, B, R, M = d["A"][t + 1], d["B"][t + 1], d["R"][t + 1], d["M"][t + 1]
        S = A.T @ Pn @ B + M
        Pn = d["Q"][t] + A.T @ Pn @ A - S @ np.linalg.solve(R + B.T @ Pn @ B, S.T)
        np.testing.assert_allclose(sol["P"][t], Pn, rtol=1e-11, atol=1e-11)
        Kt = -np.linalg.solve(R + B.T @ sol["P"][t + 1] @ B, S.T)
        np.testing.assert_allclose(sol["K"][t + 1], Kt, rtol=1e-10, atol=1e-11)


def test_two_node_closed_form():
    """Root 0 with one child 1, Delta = 0, M = 0.  By hand: x_0 = c_0,
    u = -G^{-1}(r + B'Q_1(A c_0 + c_1) + B'q_1) with G = R + B'Q_1 B,
    x_1 = A x_0 + B u + c_1, y_1 = Q_1 x_1 + q_1, y_0 = Q_0 x_0 + q_0 + A'y_1."""
    rng = inputs.rng_for(8)
    n, m = 3, 2
    p = np.array([-1, 0], dtype=np.int32)
    d = inputs.problem_data(p, n, m, rng)
    A, B, R, r = d["A"][1], d["B"][1], d["R"][1], d["r"][1]
    Q0, Q1, q0, q1, c0, c1 = d["Q"][0], d["Q"][1], d["q"][0], d["q"][1], d["c"][0], d["c"][1]
    G = R + B.T @ Q1 @ B
    x0 = c0
    u = -np.linalg.solve(G, r + B.T @ Q1 @ (A @ c0 + c1) + B.T @ q1)
    x1 = A @ x0 + B @ u + c1
    y1 = Q1 @ x1 + q1
    y0 = Q0 @ x0 + q0 + A.T @ y1
    P0 = Q0 + A.T @ Q1 @ A - A.T @ Q1 @ B @ np.linalg.solve(G, B.T @ Q1 @ A)
    sol = riccati.tree_riccati(p, n, m, d)
    np.testing.assert_allclose(sol["x"][0], x0, atol=1e-13)
    np.testing.assert_allclose(sol["x"][1], x1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sol["u"][1], u, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sol["y"][1], y1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sol["y"][0], y0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sol["P"][1], Q1, rtol=0, atol=0)
    np.testing.assert_allclose(sol["P"][0], P0, rtol=1e-12, atol=1e-12)


def test_zero_regularization_paths_agree():
    """Delta = None and an explicit all-zero Delta give the same solution; a
    vanishing regularization eps*I converges to it (strictly convex data)."""
    rng = inputs.rng_for(9)
    p = inputs.random_recursive(25, rng)
    n, m = 4, 2
    d = inputs.problem_data(p, n, m, rng)
    s0 = riccati.tree_riccati(p, n, m, d)
    dz = dict(d, Delta=np.zeros((len(p), n, n)))
    s1 = riccati.tree_riccati(p, n, m, dz)
    assert riccati.forward_error(s1, s0, p) <= 1e-14
    prev = None
    for eps in (1e-2, 1e-4, 1e-6, 1e-8):
        de = dict(d, Delta=np.broadcast_to(eps * np.eye(n), (len(p), n, n)).copy())
        err = riccati.forward_error(riccati.tree_riccati(p, n, m, de), s0, p)
        if prev is not None:
            assert err < prev * 0.05 + 1e-13
        prev = err
    assert prev < 1e-6


def test_oracle_rejects_bad_topology():
    d = inputs.problem_data(inputs.chain(3), 2, 1, inputs.rng_for(1))
    with pytest.raises(RuntimeError):
        riccati.tree_riccati(np.array([-1, 2, 1], dtype=np.int32), 2, 1, d)   # cycle 1<->2
    with pytest.raises(RuntimeError):
        riccati.tree_riccati(np.array([1, 2, 0], dtype=np.int32), 2, 1, d)    # no root


def test_forest_is_a_batch_of_independent_trees():
    """A forest's KKT system is block diagonal: its solution is exactly the
    independent per-tree solutions (bitwise, same arithmetic per tree) and it
    matches the dense solve of the whole block system."""
    rng = inputs.rng_for(41)
    n, m = 3, 2
    trees = [inputs.random_recursive(int(rng.integers(2, 15)), rng) for _ in range(4)]
    datas = [inputs.problem_data(p, n, m, rng, M_scale=0.2, delta="random", delta_value=0.2) for p in trees]
    par, offs = inputs.forest(trees)
    data = inputs.concat_data(datas)
    sol = riccati.tree_riccati(par, n, m, data)
    for t, p in enumerate(trees):
        alone = riccati.tree_riccati(p, n, m, datas[t])
        sl = slice(offs[t], offs[t] + len(p))
        for k in ("x", "u", "y", "P", "K"):
            np.testing.assert_array_equal(sol[k][sl], alone[k])
    ref = dense.dense_solve(par, n, m, data)
    assert riccati.forward_error(sol, ref, par) < 1e-11
    assert riccati.kkt_residual(par, n, m, data, sol["x"], sol["u"], sol["y"])["eta"] < 1e-14


# ---------------------------------------------------------------- per-op pins

def _rand_psd(rng, n, rank=None, scale=1.0):
    G = rng.standard_normal((n, rank or n))
    return scale * G @ G.T


def _schur(H, keep, elim):
    """Schur complement of H[elim, elim] in H, as a quadratic form on ``keep``."""
    Hkk = H[np.ix_(keep, keep)]
    Hke = H[np.ix_(keep, elim)]
    Hee = H[np.ix_(elim, elim)]
    return Hkk - Hke @ np.linalg.solve(Hee, Hke.T)


@pytest.mark.parametrize("rank_C", [None, 1])
def test_fold_identity_by_saddle_elimination(rank_C):
    """eq. (fold-identity): eliminating (x_j, lambda) from
    1/2 x_i'P x_i + lambda'(A x_i - x_j) - 1/2 lambda'C lambda + 1/2 x_j'U x_j
    leaves 1/2 x_i' tau x_i.  Also holds for singular C (exact dynamics)."""
    rng = inputs.rng_for(21)
    n = 4
    A = rng.standard_normal((n, n)); C = _rand_psd(rng, n, rank_C); U = _rand_psd(rng, n)
    Pp = -_rand_psd(rng, n, 2, 0.1)
    # variables (x_i, x_j, lambda)
    Z = np.zeros((n, n)); I = np.eye(n)
    H = np.block([[Pp, Z, A.T], [Z, U, -I], [A, -I, -C]])
    S = _schur(H, list(range(n)), list(range(n, 3 * n)))
    np.testing.assert_allclose(ops.tau(A, C, Pp, U), S, rtol=1e-11, atol=1e-11)
    # PSD increment, eq. (elimination-psd)
    assert np.linalg.eigvalsh(0.5 * (S - Pp + (S - Pp).T)).min() > -1e-10


@pytest.mark.parametrize("rank_C", [None, 1])
def test_compose_identity_by_saddle_elimination(rank_C):
    """eq. (compose-identity): eliminating (x_j, lambda_l) from the two segment
    values plus 1/2 x_j'U x_j leaves the conditional quadratic of the composed
    triple, as a quadratic form in (x_i, x_k, lambda_r)."""
    rng = inputs.rng_for(22)
    n = 3
    Al, Ar = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    Cl, Cr = _rand_psd(rng, n, rank_C), _rand_psd(rng, n, rank_C)
    Pl, Pr = -_rand_psd(rng, n, 1, 0.1), -_rand_psd(rng, n, 1, 0.1)
    U = _rand_psd(rng, n) + 0.5 * np.eye(n)
    Z = np.zeros((n, n)); I = np.eye(n)
    # variables: x_i, x_k, lambda_r | x_j, lambda_l
    # 1/2 x_i'Pl x_i + lam_l'(Al x_i - x_j) - 1/2 lam_l'Cl lam_l + 1/2 x_j'(U + Pr) x_j
    #   + lam_r'(Ar x_j - x_k) - 1/2 lam_r'Cr lam_r
    H = np.block([
        [Pl, Z, Z, Z, Al.T],
        [Z, Z, -I, Z, Z],
        [Z, -I, -Cr, Ar, Z],
        [Z, Z, Ar.T, U + Pr, -I],
        [Al, Z, Z, -I, -Cl]])
    S = _schur(H, list(range(3 * n)), list(range(3 * n, 5 * n)))
    (A_new, C_new, P_new), tape = ops.compose((Ar, Cr, Pr), (Al, Cl, Pl), U)
    target = np.block([[P_new, Z, A_new.T], [Z, Z, -I], [A_new, -I, -C_new]])
    np.testing.assert_allclose(S, target, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(tape[2], Pr + U)
    assert np.linalg.eigvalsh(0.5 * (C_new + C_new.T)).min() > -1e-10
    assert np.linalg.eigvalsh(0.5 * (P_new - Pl + (P_new - Pl).T)).min() > -1e-10


def test_compose_associativity():
    """eq. (node-aware-associativity) on three consecutive edges."""
    rng = inputs.rng_for(23)
    n = 4
    tri = [(rng.standard_normal((n, n)), _rand_psd(rng, n), -_rand_psd(rng, n, 1, 0.05)) for _ in range(3)]
    U1, U2 = _rand_psd(rng, n) + np.eye(n), _rand_psd(rng, n) + np.eye(n)
    left, _ = ops.compose(tri[2], ops.compose(tri[1], tri[0], U1)[0], U2)
    right, _ = ops.compose(ops.compose(tri[2], tri[1], U2)[0], tri[0], U1)
    for a, b in zip(left, right):
        np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-10)


def test_condense_matches_control_elimination():
    """eq. (edge-components): eliminating u from
    x_i'M u + 1/2 u'R u + lambda'(A x_i + B u - x_j) - 1/2 lambda'Delta lambda
    leaves the triple (Abar, Cbar, Pbar) as a quadratic form in (x_i, x_j, lambda)."""
    rng = inputs.rng_for(24)
    n, m = 4, 2
    A = rng.standard_normal((n, n)); B = rng.standard_normal((n, m)); M = rng.standard_normal((n, m))
    R = _rand_psd(rng, m) + np.eye(m); D = _rand_psd(rng, n, 2, 0.1)
    Z = np.zeros((n, n)); I = np.eye(n); Znm = np.zeros((n, m))
    # variables x_i, x_j, lambda | u
    H = np.block([
        [Z, Z, A.T, M],
        [Z, Z, -I, Znm],
        [A, -I, -D, B],
        [M.T, Znm.T, B.T, R]])
    S = _schur(H, list(range(3 * n)), list(range(3 * n, 3 * n + m)))
    Ab, Cb, Pb = ops.condense(A, B, R, M, D)
    target = np.block([[Pb, Z, Ab.T], [Z, Z, -I], [Ab, -I, -Cb]])
    np.testing.assert_allclose(S, target, rtol=1e-11, atol=1e-11)


def test_local_factor_consistent_with_recursion():
    """Sec. V-C: K_e of eq. (factor-local) evaluated on the oracle's P_j equals the
    oracle's gain, and P_i = Q_i + sum (M K + A'W A_cl) over the children."""
    rng = inputs.rng_for(25)
    p = inputs.random_recursive(12, rng)
    n, m = 3, 2
    d = inputs.problem_data(p, n, m, rng, M_scale=0.2, delta="random", delta_value=0.3)
    sol = riccati.tree_riccati(p, n, m, d)
    Pacc = d["Q"].copy()
    for j in range(len(p)):
        if p[j] < 0:
            continue
        lf = ops.local_factor(sol["P"][j], d["A"][j], d["B"][j], d["R"][j], d["M"][j], d["Delta"][j])
        np.testing.assert_allclose(lf["K"], sol["K"][j], rtol=1e-11, atol=1e-12)
        Pacc[p[j]] += d["M"][j] @ lf["K"] + d["A"][j].T @ lf["W"] @ lf["Acl"]
    np.testing.assert_allclose(Pacc, sol["P"], rtol=1e-11, atol=1e-11)


# ------------------------------------------------------------------ brute-force subtree maps
# The value function of a subtree with its root state held fixed is quadratic
# in that state, and the subtree's optimal states are affine in it.  Both are
# obtained here by dense solves of the subtree's KKT system with the root's
# state moved to the right-hand side (no tree recursion involved); by the
# envelope theorem the gradient of the value at x_i is sum over the children j
# of (M_j u_j + A_j^T y_j).  These pin the oracle's affine maps (Sec. VI) and
# state maps (Sec. VII) at one operation.

def _subtree_nodes(parent, i):
    parent = np.asarray(parent)
    out, stack = [], [i]
    while stack:
        v = stack.pop()
        out.append(v)
        stack.extend(int(c) for c in np.nonzero(parent == v)[0][::-1])
    return [out[0]] + sorted(out[1:])


def _fixed_root(parent, n, m, d, i, xi):
    """Saddle point of the subtree of i with x_i = xi held fixed (root data of
    i excluded).  Returns (nodes, x, u, y, grad) in subtree order, grad = the
    gradient of the subtree's value at xi."""
    parent = np.asarray(parent)
    nodes = _subtree_nodes(parent, i)
    idx = {v: t for t, v in enumerate(nodes)}
    sp = np.array([-1] + [idx[int(parent[v])] for v in nodes[1:]], dtype=np.int32)
    sd = {k: (None if v is None else np.asarray(v)[nodes]) for k, v in d.items()}
    K, b, (X, U, Y, nonroot) = dense.assemble_kkt(sp, n, m, sd)
    dim = K.shape[0]
    drop = set(range(X(0).start, X(0).stop)) | set(range(Y(0).start, Y(0).stop))
    keep = [t for t in range(dim) if t not in drop]
    cols = list(range(X(0).start, X(0).stop))
    z = np.zeros(dim)
    z[cols] = xi
    z[keep] = np.linalg.solve(K[np.ix_(keep, keep)], -(b[keep] + K[np.ix_(keep, cols)] @ xi))
    Ns = len(nodes)
    x = np.stack([z[X(t)] for t in range(Ns)])
    y = np.stack([z[Y(t)] for t in range(Ns)])
    u = np.zeros((Ns, m))
    for j in nonroot:
        u[j] = z[U(j)]
    grad = np.zeros(n)
    for j in range(1, Ns):
        if sp[j] == 0:
            grad += (sd["M"][j] @ u[j] if sd.get("M") is not None else 0.0) + sd["A"][j].T @ y[j]
    return nodes, x, u, y, grad


def _affine_in_root(parent, n, m, d, i, what):
    """(Jacobian, value at 0) of an affine function of x_i computed by _fixed_root."""
    f0 = what(*_fixed_root(parent, n, m, d, i, np.zeros(n)))
    J = np.stack([what(*_fixed_root(parent, n, m, d, i, np.eye(n)[a])) - f0 for a in range(n)], axis=1)
    return J, f0


def _chain_case(seed, N, n, m, delta):
    rng = inputs.rng_for(seed)
    p = inputs.chain(N)
    d = inputs.problem_data(p, n, m, rng, M_scale=0.3, delta=delta, delta_value=0.4)
    return p, d


@pytest.mark.parametrize("delta", [None, "random"])
def test_expand_compress_gives_the_subtree_value_hessian(delta):
    """eq. (value-reconstruction): at a centre j compressed between the edges
    (i, j) and (j, k), expanding its tape with P_k gives P_j, the Hessian of the
    value of j's subtree (Thm. 1) -- here obtained by brute force."""
    n, m = 3, 2
    p, d = _chain_case(41, 4, n, m, delta)
    D = d.get("Delta")
    cond = lambda e: ops.condense(d["A"][e], d["B"][e], d["R"][e], d["M"][e], None if D is None else D[e])
    i, j, k = 1, 2, 3
    Pk = d["Q"][k]                                    # a leaf's value Hessian is its own Q
    _, tape = ops.compose(cond(k), cond(j), d["Q"][j])
    Pj = ops.expand_compress(tape, Pk)
    J, _ = _affine_in_root(p, n, m, d, j, lambda nodes, x, u, y, g: g)
    np.testing.assert_allclose(Pj, d["Q"][j] + J, rtol=1e-10, atol=1e-11)
    # Delta = 0, M != 0: also the textbook one-step Riccati update of P_k across edge (j, k)
    if D is None:
        A, B, M, R = d["A"][k], d["B"][k], d["M"][k], d["R"][k]
        H = A.T @ Pk @ B + M
        textbook = d["Q"][j] + A.T @ Pk @ A - H @ np.linalg.solve(R + B.T @ Pk @ B, H.T)
        np.testing.assert_allclose(Pj, textbook, rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("delta", [None, "random"])
def test_affine_edge_is_the_value_gradient_of_a_leaf_edge(delta):
    """eq. (affine-edge): for a leaf j under i, the message T_e^T p_j + z_e with
    p_j = q_j is the gradient of the leaf edge's value at x_i = 0, and T_e^T
    is its sensitivity to q_j (brute force on the two-node subtree)."""
    n, m = 3, 2
    p, d = _chain_case(42, 3, n, m, delta)
    D = d.get("Delta")
    i, j = 1, 2
    lf = ops.local_factor(d["Q"][j], d["A"][j], d["B"][j], d["R"][j], d["M"][j], None if D is None else D[j])
    Z, z = ops.affine_edge(lf["T"], lf["K"], lf["W"], lf["Acl"], d["r"][j], d["c"][j])
    grad0 = _fixed_root(p, n, m, d, i, np.zeros(n))[4]
    np.testing.assert_allclose(Z @ d["q"][j] + z, grad0, rtol=1e-10, atol=1e-11)
    sens = []
    for a in range(n):
        d2 = {k: (None if v is None else v.copy()) for k, v in d.items()}
        d2["q"][j] += np.eye(n)[a]
        sens.append(_fixed_root(p, n, m, d2, i, np.zeros(n))[4] - grad0)
    np.testing.assert_allclose(np.stack(sens, axis=1), Z, rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("delta", [None, "random"])
def test_affine_compose_is_the_value_gradient_across_a_compressed_node(delta):
    """eq. (affine-compose): composing the affine maps of the edges (i, j) and
    (j, k) through the centre's linear data h_j = q_j gives the message from
    k's subtree to i: Zhat p_k + zhat with p_k = q_k equals the gradient of the
    value of i's subtree at x_i = 0, and Zhat = Z_l Z_r is its sensitivity to
    q_k (brute force on a three-edge chain)."""
    n, m = 3, 2
    p, d = _chain_case(43, 4, n, m, delta)
    D = d.get("Delta")
    i, j, k = 1, 2, 3
    J, _ = _affine_in_root(p, n, m, d, j, lambda nodes, x, u, y, g: g)
    Pj = d["Q"][j] + J                                  # brute-force value Hessian at j

    def edge(e, Pe):
        lf = ops.local_factor(Pe, d["A"][e], d["B"][e], d["R"][e], d["M"][e], None if D is None else D[e])
        return ops.affine_edge(lf["T"], lf["K"], lf["W"], lf["Acl"], d["r"][e], d["c"][e])

    Zl, zl = edge(j, Pj)
    Zr, zr = edge(k, d["Q"][k])
    Zh, zh = ops.affine_compose(Zl, zl, Zr, zr, d["q"][j])
    grad0 = _fixed_root(p, n, m, d, i, np.zeros(n))[4]
    np.testing.assert_allclose(Zh @ d["q"][k] + zh, grad0, rtol=1e-10, atol=1e-11)
    sens = []
    for a in range(n):
        d2 = {kk: (None if v is None else v.copy()) for kk, v in d.items()}
        d2["q"][k] += np.eye(n)[a]
        sens.append(_fixed_root(p, n, m, d2, i, np.zeros(n))[4] - grad0)
    np.testing.assert_allclose(np.stack(sens, axis=1), Zh, rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("delta", [None, "random"])
def test_transition_compose_matches_the_brute_force_state_maps(delta):
    """eq. (transition-compose): the optimal x_j is affine in x_i (x_j = T_l x_i
    + b_l) and x_k in x_j (T_r, b_r); composing the two maps gives x_k as a
    function of x_i.  All three maps come from dense solves of the subtrees with
    their root state held fixed; T_l also equals the local factor's
    T = F^{-1} A_cl of eq. (FW)."""
    n, m = 3, 2
    p, d = _chain_case(44, 4, n, m, delta)
    D = d.get("Delta")
    i, j, k = 1, 2, 3
    Tl, bl = _affine_in_root(p, n, m, d, i, lambda nodes, x, u, y, g: x[nodes.index(j)])
    Tr, br = _affine_in_root(p, n, m, d, j, lambda nodes, x, u, y, g: x[nodes.index(k)])
    Tik, bik = _affine_in_root(p, n, m, d, i, lambda nodes, x, u, y, g: x[nodes.index(k)])
    T, b = ops.transition_compose(Tr, br, Tl, bl)
    np.testing.assert_allclose(T, Tik, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(b, bik, rtol=1e-10, atol=1e-11)
    J, _ = _affine_in_root(p, n, m, d, j, lambda nodes, x, u, y, g: g)
    lf = ops.local_factor(d["Q"][j] + J, d["A"][j], d["B"][j], d["R"][j], d["M"][j], None if D is None else D[j])
    np.testing.assert_allclose(lf["T"], Tl, rtol=1e-10, atol=1e-11)
