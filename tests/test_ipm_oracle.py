"""Pins of the box-constrained oracle (oracle/ipm.py) against facts fixed by the
mathematics: a one-control closed form (a convex quadratic in one variable is
minimised over an interval by clipping its unconstrained minimiser), the
unconstrained KKT solve when no bound is active, exhaustive active-set
enumeration on tiny trees (strict convexity makes the optimum unique), and the
optimality conditions themselves."""
import numpy as np
import pytest

from oracle import dense, ipm
from paper_2608_01332_b300 import inputs


def _bounds(rng, N, m, width, parent):
    lo = -width * (0.2 + rng.random((N, m)))
    hi = width * (0.2 + rng.random((N, m)))
    root = np.asarray(parent) < 0
    lo[root], hi[root] = -np.inf, np.inf
    return lo, hi


@pytest.mark.parametrize("seed", range(6))
def test_single_control_is_clipped_minimiser(seed):
    rng = inputs.rng_for(1300 + seed)
    p = inputs.chain(2)
    d = inputs.problem_data(p, 1, 1, rng)
    Q1, q1, R, r = d["Q"][1, 0, 0], d["q"][1, 0], d["R"][1, 0, 0], d["r"][1, 0]
    A, B, c0, c1 = d["A"][1, 0, 0], d["B"][1, 0, 0], d["c"][0, 0], d["c"][1, 0]
    u_free = -(r + B * (Q1 * (A * c0 + c1) + q1)) / (R + Q1 * B * B)
    lo, hi = u_free + (-0.5 if seed % 3 == 0 else 0.3), u_free + (0.5 if seed % 3 != 2 else -0.2)
    lo, hi = min(lo, hi), max(lo, hi)
    want = min(max(u_free, lo), hi)
    u_lo = np.array([[-np.inf], [lo]])
    u_hi = np.array([[np.inf], [hi]])
    sol = ipm.dense_ipm(p, 1, 1, d, u_lo, u_hi)
    assert abs(sol["u"][1, 0] - want) <= 1e-8 * max(1.0, abs(want))
    bf = ipm.active_set_bruteforce(p, 1, 1, d, u_lo, u_hi)
    assert abs(bf["u"][1, 0] - want) <= 1e-12 * max(1.0, abs(want))


def test_inactive_bounds_give_the_unconstrained_solution():
    rng = inputs.rng_for(1310)
    p = inputs.random_recursive(20, rng)
    n, m = 3, 2
    d = inputs.problem_data(p, n, m, rng, M_scale=0.2, delta="subset", delta_value=0.1)
    free = dense.dense_solve(p, n, m, d)
    lo, hi = _bounds(rng, len(p), m, 1e6, p)
    sol = ipm.dense_ipm(p, n, m, d, lo, hi)
    for k in ("x", "u", "y"):
        assert np.abs(sol[k] - free[k]).max() <= 1e-7 * max(1.0, np.abs(free[k]).max())
    assert max(sol["lam_lo"].max(), sol["lam_hi"].max()) <= 1e-9


@pytest.mark.parametrize("seed", range(5))
def test_dense_ipm_equals_active_set_enumeration(seed):
    rng = inputs.rng_for(1320 + seed)
    p = inputs.random_recursive(4 + seed % 2, rng)
    n, m = 2, 1 + seed % 2
    d = inputs.problem_data(p, n, m, rng, M_scale=0.2, delta=("subset" if seed % 2 else None), delta_value=0.1)
    free = dense.dense_solve(p, n, m, d)
    width = 0.5 * np.abs(free["u"]).max()                   # tight enough that some bounds bind
    lo, hi = _bounds(rng, len(p), m, width, p)
    bf = ipm.active_set_bruteforce(p, n, m, d, lo, hi)
    sol = ipm.dense_ipm(p, n, m, d, lo, hi)
    for k in ("x", "u", "y"):
        assert np.abs(sol[k] - bf[k]).max() <= 1e-7 * max(1.0, np.abs(bf[k]).max())
    active = (np.abs(bf["u"] - lo) < 1e-9) | (np.abs(bf["u"] - hi) < 1e-9)
    assert active.any()
    v = ipm.kkt_violation(p, n, m, d, lo, hi, sol["x"], sol["u"], sol["y"], sol["lam_lo"], sol["lam_hi"])
    # at an active bound the last Newton matrix holds l / s ~ 1e10 on the diagonal, so the
    # control rows carry a rounding error of about eps * (l / s) * |u|
    s_min = max(1e-300, min(np.abs(sol["u"] - lo)[np.isfinite(lo)].min(), np.abs(hi - sol["u"])[np.isfinite(hi)].min()))
    lam = max(sol["lam_lo"].max(), sol["lam_hi"].max(), 1.0)
    assert v["stationarity"] <= 1e-9 + 64 * np.finfo(float).eps * lam / s_min * max(1.0, np.abs(sol["u"]).max())
    assert v["complementarity"] <= 1e-9
    assert v["feasibility"] == 0.0 and v["sign"] == 0.0
