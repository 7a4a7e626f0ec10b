"""The interior-point driver (tlqr_ipm_box) against the dense oracle.

Small trees: the GPU method's solution equals the dense primal-dual method's
(oracle/ipm.py, pinned by enumeration and closed forms) and satisfies the
optimality conditions of the box-constrained problem.  A driving-style tree of
a few thousand nodes: stationarity through the tree residual of eq. (kkt) with
r replaced by r - l_lo + l_hi, complementarity, feasibility and multiplier
signs."""
import numpy as np
import pytest

from oracle import dense, ipm, riccati
from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = tlqr.TLQR_PREC_FP64, tlqr.TLQR_PREC_MIXED


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _bounds(rng, parent, m, width):
    N = len(parent)
    lo = -width * (0.2 + rng.random((N, m)))
    hi = width * (0.2 + rng.random((N, m)))
    root = np.asarray(parent) < 0
    lo[root], hi[root] = -np.inf, np.inf
    return lo, hi


def run_gpu(p, n, m, d, lo, hi, precision, forest=False):
    N = len(p)
    s = tlqr.TreeLQR(p, n, m, precision, has_M=d.get("M") is not None, has_delta=d.get("Delta") is not None,
                     forest=forest)
    try:
        out = {k: torch.zeros(sh, dtype=torch.float64, device="cuda") for k, sh in
               (("x", (N, n)), ("u", (N, m)), ("y", (N, n)), ("lam_lo", (N, m)), ("lam_hi", (N, m)))}
        info = tlqr.tlqr_ipm_box(s.plan, s.f, {k: dev(v) for k, v in d.items()}, dev(lo), dev(hi), out["x"],
                                 out["u"], out["y"], out["lam_lo"], out["lam_hi"], tol=1e-10)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}, info
    finally:
        s.close()


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ipm_matches_dense_oracle(precision, seed):
    rng = inputs.rng_for(1400 + seed)
    p, _ = inputs.permute_labels(inputs.random_recursive(40, rng), rng)
    n, m = 3, 2
    d = inputs.problem_data(p, n, m, rng, M_scale=0.2, delta=("subset" if seed % 2 else None), delta_value=0.1)
    free = dense.dense_solve(p, n, m, d)
    lo, hi = _bounds(rng, p, m, 0.6 * np.abs(free["u"]).max())
    ref = ipm.dense_ipm(p, n, m, d, lo, hi, tol=1e-12)
    got, info = run_gpu(p, n, m, d, lo, hi, precision)
    tol = 1e-7 if precision == FP64 else 1e-6
    for k in ("x", "u", "y"):
        assert np.abs(got[k] - ref[k]).max() <= tol * max(1.0, np.abs(ref[k]).max()), k
    active = (np.abs(ref["u"] - lo) < 1e-8) | (np.abs(ref["u"] - hi) < 1e-8)
    assert active.sum() >= 3
    v = ipm.kkt_violation(p, n, m, d, lo, hi, got["x"], got["u"], got["y"], got["lam_lo"], got["lam_hi"])
    assert v["complementarity"] <= 1e-8 and v["feasibility"] == 0.0 and v["sign"] == 0.0
    assert info["iterations"] < 60


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_ipm_on_a_driving_tree(precision):
    rng = inputs.rng_for(1450)
    p = inputs.driving_tree(rng, 3000)
    n, m = 6, 2
    d = inputs.problem_data(p, n, m, rng)
    lo, hi = _bounds(rng, p, m, 0.8)
    got, info = run_gpu(p, n, m, d, lo, hi, precision)
    nonroot = np.asarray(p) >= 0
    assert np.all(got["u"][nonroot] >= lo[nonroot]) and np.all(got["u"][nonroot] <= hi[nonroot])
    assert np.all(got["lam_lo"] >= 0) and np.all(got["lam_hi"] >= 0)
    comp = np.maximum(np.abs(got["lam_lo"][nonroot] * (got["u"][nonroot] - lo[nonroot])).max(),
                      np.abs(got["lam_hi"][nonroot] * (hi[nonroot] - got["u"][nonroot])).max())
    assert comp <= 1e-8
    active = ((np.abs(got["u"] - lo) < 1e-6) | (np.abs(got["u"] - hi) < 1e-6))[nonroot]
    assert active.sum() > 10
    # stationarity: the tree KKT residual with the bound multipliers folded into r
    d2 = dict(d)
    d2["r"] = d["r"] - got["lam_lo"] + got["lam_hi"]
    d2["r"][~nonroot] = 0.0
    res = riccati.kkt_residual(p, n, m, d2, got["x"], got["u"], got["y"])
    # the multipliers are recovered from the control rows at convergence: stationarity
    # holds to rounding, complementarity at the gap's scale (checked above)
    assert res["eta"] <= 1e-12
    assert info["iterations"] < 60
