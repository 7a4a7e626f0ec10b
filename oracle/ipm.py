"""ORACLE -- test infrastructure only.

Box-constrained tree LQR: the problem of eq. (1)-(2) (Sec. III-A) with bounds
u_lo <= u_e <= u_hi on every control, the setting in which the paper's solver
is called by an interior-point method (Sec. IX-B, XI-B: each Newton step of a
primal-dual method is one tree-structured KKT solve).  This file solves it with
no tree structure at all:

  * ``dense_ipm``: a textbook primal-dual path-following method on the dense
    KKT matrix of ``dense.assemble_kkt``.  With slacks s_lo = u - u_lo,
    s_hi = u_hi - u and multipliers l_lo, l_hi >= 0, the Newton point for the
    barrier parameter mu solves the KKT system with R replaced by
    R + diag(l_lo / s_lo + l_hi / s_hi) and r by
    r - diag(l_lo / s_lo + l_hi / s_hi) u - mu / s_lo + mu / s_hi; the step
    length keeps slacks and multipliers positive (fraction to the boundary
    tau), and mu <- sigma * mean(l * s); it stops after a full step (alpha =
    1, so the linear rows hold to solve accuracy) once mean(l * s) <= tol.
  * ``active_set_bruteforce``: for tiny problems, every assignment of each
    bounded control component to {free, at lower, at upper}; the equality-
    constrained QP of each assignment is solved densely and the one whose
    multipliers and bounds satisfy the KKT sign conditions is the unique
    optimum (strict convexity).
  * ``kkt_violation``: stationarity, complementarity, feasibility and sign
    errors of a candidate point, written out from the optimality conditions.

Infinite bounds mark components without that bound; the root's control slot
carries no control.
"""
from __future__ import annotations

import itertools

import numpy as np

from oracle import dense


def _u_index(parent, m, U, nonroot):
    """Rows of the dense system holding each (edge, component) of u."""
    idx = []
    for j in nonroot:
        sl = U(j)
        idx.extend((j, a, sl.start + a) for a in range(m))
    return idx


def dense_ipm(parent, n: int, m: int, data: dict, u_lo, u_hi, tol: float = 1e-11, max_iter: int = 200,
              sigma: float = 0.1, tau: float = 0.995):
    K, b, (X, U, Y, nonroot) = dense.assemble_kkt(parent, n, m, data)
    N = len(parent)
    comps = _u_index(parent, m, U, nonroot)
    rows = np.array([r for _, _, r in comps], dtype=int)
    lo = np.array([u_lo[j][a] for j, a, _ in comps])
    hi = np.array([u_hi[j][a] for j, a, _ in comps])
    has_lo, has_hi = np.isfinite(lo), np.isfinite(hi)
    # interior start: the box midpoint, or one unit inside a one-sided bound
    u = np.where(has_lo & has_hi, 0.5 * (lo + hi), np.where(has_lo, lo + 1.0, np.where(has_hi, hi - 1.0, 0.0)))
    mu = 1.0
    s_lo = np.where(has_lo, u - lo, 1.0)
    s_hi = np.where(has_hi, hi - u, 1.0)
    l_lo = np.where(has_lo, mu / s_lo, 0.0)
    l_hi = np.where(has_hi, mu / s_hi, 0.0)
    z = np.zeros(K.shape[0])
    z[rows] = u
    n_ineq = int(has_lo.sum() + has_hi.sum())
    it = 0
    for it in range(1, max_iter + 1):
        sig = np.where(has_lo, l_lo / s_lo, 0.0) + np.where(has_hi, l_hi / s_hi, 0.0)
        Kt = K.copy()
        bt = b.copy()
        Kt[rows, rows] += sig
        bt[rows] += -sig * u - np.where(has_lo, mu / s_lo, 0.0) + np.where(has_hi, mu / s_hi, 0.0)
        zp = np.linalg.solve(Kt, -bt)
        du = zp[rows] - u
        dl_lo = np.where(has_lo, mu / s_lo - l_lo - (l_lo / s_lo) * du, 0.0)
        dl_hi = np.where(has_hi, mu / s_hi - l_hi + (l_hi / s_hi) * du, 0.0)
        alpha = 1.0
        for v, dv, act in ((s_lo, du, has_lo), (s_hi, -du, has_hi), (l_lo, dl_lo, has_lo), (l_hi, dl_hi, has_hi)):
            neg = act & (dv < 0)
            if neg.any():
                alpha = min(alpha, float(np.min(-tau * v[neg] / dv[neg])))
        z = z + alpha * (zp - z)
        u = z[rows]
        s_lo = np.where(has_lo, u - lo, 1.0)
        s_hi = np.where(has_hi, hi - u, 1.0)
        l_lo = l_lo + alpha * dl_lo
        l_hi = l_hi + alpha * dl_hi
        gap = float((np.where(has_lo, l_lo * s_lo, 0.0) + np.where(has_hi, l_hi * s_hi, 0.0)).sum())
        mean_gap = gap / max(1, n_ineq)
        # stop after a full Newton step: the linear KKT rows then hold to solve accuracy
        if mean_gap <= tol and alpha >= 1.0:
            break
        mu = sigma * mean_gap
    x = np.stack([z[X(i)] for i in range(N)])
    y = np.stack([z[Y(i)] for i in range(N)])
    uo = np.zeros((N, m))
    lam_lo, lam_hi = np.zeros((N, m)), np.zeros((N, m))
    for t, (j, a, _) in enumerate(comps):
        uo[j, a] = u[t]
        lam_lo[j, a] = l_lo[t]
        lam_hi[j, a] = l_hi[t]
    return dict(x=x, u=uo, y=y, lam_lo=lam_lo, lam_hi=lam_hi, iterations=it)


def active_set_bruteforce(parent, n: int, m: int, data: dict, u_lo, u_hi):
    """Exact optimum of a tiny box-constrained problem by enumeration."""
    K, b, (X, U, Y, nonroot) = dense.assemble_kkt(parent, n, m, data)
    N = len(parent)
    comps = _u_index(parent, m, U, nonroot)
    choices = []
    for j, a, _ in comps:
        opts = ["free"]
        if np.isfinite(u_lo[j][a]):
            opts.append("lo")
        if np.isfinite(u_hi[j][a]):
            opts.append("hi")
        choices.append(opts)
    found = None
    for pick in itertools.product(*choices):
        act = [(t, p) for t, p in enumerate(pick) if p != "free"]
        k = len(act)
        dim = K.shape[0]
        E = np.zeros((k, dim))
        e = np.zeros(k)
        for q, (t, p) in enumerate(act):
            j, a, r = comps[t]
            E[q, r] = 1.0
            e[q] = u_lo[j][a] if p == "lo" else u_hi[j][a]
        # stationarity K z + b + E^T nu = 0 with E z = e; nu = l_hi - l_lo at active rows
        big = np.block([[K, E.T], [E, np.zeros((k, k))]])
        sol = np.linalg.solve(big, np.concatenate([-b, e]))
        z, nu = sol[:dim], sol[dim:]
        ok = True
        for q, (t, p) in enumerate(act):
            if (p == "lo" and nu[q] > 1e-12) or (p == "hi" and nu[q] < -1e-12):
                ok = False
        for t, (j, a, r) in enumerate(comps):
            if z[r] < u_lo[j][a] - 1e-12 or z[r] > u_hi[j][a] + 1e-12:
                ok = False
        if ok:
            if found is not None:
                raise RuntimeError("two active sets satisfy the KKT conditions")
            x = np.stack([z[X(i)] for i in range(N)])
            y = np.stack([z[Y(i)] for i in range(N)])
            u = np.zeros((N, m))
            for t, (j, a, r) in enumerate(comps):
                u[j, a] = z[r]
            found = dict(x=x, u=u, y=y)
    if found is None:
        raise RuntimeError("no active set satisfies the KKT conditions")
    return found


def kkt_violation(parent, n: int, m: int, data: dict, u_lo, u_hi, x, u, y, lam_lo, lam_hi) -> dict:
    """Largest violation of each optimality condition of the box-constrained problem."""
    K, b, (X, U, Y, nonroot) = dense.assemble_kkt(parent, n, m, data)
    N = len(parent)
    z = np.zeros(K.shape[0])
    for i in range(N):
        z[X(i)] = x[i]
        z[Y(i)] = y[i]
    for j in nonroot:
        z[U(j)] = u[j]
    g = K @ z + b
    for j in nonroot:
        g[U(j)] += -lam_lo[j] + lam_hi[j]
    comp, feas, sign = 0.0, 0.0, 0.0
    for j in nonroot:
        for a in range(m):
            lo, hi = u_lo[j][a], u_hi[j][a]
            if np.isfinite(lo):
                comp = max(comp, abs(lam_lo[j, a] * (u[j, a] - lo)))
                feas = max(feas, lo - u[j, a])
            if np.isfinite(hi):
                comp = max(comp, abs(lam_hi[j, a] * (hi - u[j, a])))
                feas = max(feas, u[j, a] - hi)
            sign = max(sign, -lam_lo[j, a], -lam_hi[j, a])
    return dict(stationarity=float(np.abs(g).max()), complementarity=comp, feasibility=max(0.0, feas),
                sign=max(0.0, sign))
