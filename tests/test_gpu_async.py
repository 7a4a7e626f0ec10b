"""GPU tests of the level-asynchronous factorisation tail (one persistent
launch over the dependency DAG of the late rounds, Sec. X-B).

* The same arithmetic runs whether the late rounds go round by round
  (async_ops < 0), level-asynchronously from the default round on, or
  level-asynchronously from the first round: P, K and the solution agree to
  rounding (the kernels are the same device functions), and all match the
  oracle.
* Failure detection without a GPU fault: with test_withhold the launch's first
  operation never publishes completion, so every wait on it runs out after
  spin_limit polls; the factorisation returns TLQR_ERR_TIMEOUT and the context
  stays usable (a normal factorisation right after it is correct).
"""
import numpy as np
import pytest

from oracle import riccati
from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = tlqr.TLQR_PREC_FP64, tlqr.TLQR_PREC_MIXED


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def solve(parent, n, m, data, precision, forest=False, **kw):
    N = len(parent)
    s = tlqr.TreeLQR(parent, n, m, precision, has_M=data.get("M") is not None,
                     has_delta=data.get("Delta") is not None, forest=forest, **kw)
    try:
        d = {k: dev(v) for k, v in data.items()}
        out = {k: torch.zeros(shape, dtype=torch.float64, device="cuda") for k, shape in
               (("x", (N, n)), ("u", (N, m)), ("y", (N, n)), ("P", (N, n, n)), ("K", (N, m, n)))}
        tlqr.tlqr_solve(s.f, d, out["x"], out["u"], out["y"], out["P"], out["K"])
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}, None
    finally:
        s.close()


def _cases():
    rng = inputs.rng_for(901)
    out = []
    for n, m in ((4, 2), (12, 4), (16, 4), (32, 8)):
        p = inputs.long_trunk_tree(rng, trunk=300, total=3000)
        d = inputs.problem_data(p, n, m, rng, M_scale=0.2, delta="subset", delta_value=0.05)
        out.append((f"longtrunk-n{n}", p, n, m, d, False))
    p, _ = inputs.permute_labels(inputs.random_recursive(2500, rng), rng)
    out.append(("recursive-n12", p, 12, 4, inputs.problem_data(p, 12, 4, rng), False))
    f, _ = inputs.forest([inputs.random_recursive(int(k), rng) for k in (64, 900, 3, 1500)])
    out.append(("forest-n16", f, 16, 4, inputs.problem_data(f, 16, 4, rng), True))
    out.append(("chain-n12", inputs.chain(700), 12, 4, inputs.problem_data(inputs.chain(700), 12, 4, rng), False))
    out.append(("star-n8", inputs.star(600), 8, 2, inputs.problem_data(inputs.star(600), 8, 2, rng), False))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_async_tail_matches_round_by_round(case, precision):
    name, p, n, m, d, forest = case
    if precision == FP64 and n == 32:
        pytest.skip("FP64 at n = 32 runs the run-time-n kernels, which have no asynchronous tail")
    res = {}
    for mode, ops in (("rounds", -1), ("default", 0), ("all", 1 << 30)):
        res[mode], _ = solve(p, n, m, d, precision, forest=forest, async_ops=ops)
    scale = {k: max(1.0, np.abs(res["rounds"][k]).max()) for k in res["rounds"]}
    tol = 1e-12 if precision == FP64 else 1e-9
    for mode in ("default", "all"):
        for k in ("P", "K", "x", "u", "y"):
            assert np.abs(res[mode][k] - res["rounds"][k]).max() <= tol * scale[k], (mode, k)
    ref = riccati.tree_riccati(p, n, m, d)
    fe = riccati.forward_error(res["all"], ref, p)
    eta = riccati.kkt_residual(p, n, m, d, res["all"]["x"], res["all"]["u"], res["all"]["y"])["eta"]
    assert eta <= (1e-10 if precision == FP64 else 1e-8)
    assert fe <= (1e-8 if precision == FP64 else 1e-6)


def test_async_tail_is_one_launch():
    """With every round asynchronous the contraction and expansion of the whole
    tree are one launch (kind TLQR_K_FACTOR_TAIL); no per-round rake, compress or
    expansion launch remains."""
    rng = inputs.rng_for(902)
    p = inputs.long_trunk_tree(rng, trunk=300, total=3000)
    n, m = 12, 4
    d = {k: dev(v) for k, v in inputs.problem_data(p, n, m, rng).items()}
    s = tlqr.TreeLQR(p, n, m, MIXED, async_ops=1 << 30, use_graphs=False)
    try:
        tlqr.tlqr_profile_read(s.f)
        tlqr.tlqr_factor(s.f, d)
        prof = tlqr.tlqr_profile_read(s.f)
    finally:
        s.close()
    assert prof["factor_tail"]["launches"] == 1
    assert prof["rake"]["launches"] == prof["compress"]["launches"] == prof["expand"]["launches"] == 0


@pytest.mark.parametrize("n,m", [(12, 4), (32, 8)])
def test_async_wait_that_runs_out_reports_timeout_and_context_survives(n, m):
    rng = inputs.rng_for(903)
    p = inputs.long_trunk_tree(rng, trunk=200, total=2000)
    data = inputs.problem_data(p, n, m, rng)
    d = {k: dev(v) for k, v in data.items()}
    s = tlqr.TreeLQR(p, n, m, MIXED, async_ops=1 << 30, spin_limit=2000, test_withhold=True)
    try:
        with pytest.raises(tlqr.TLQRError) as e:
            tlqr.tlqr_factor(s.f, d)
        assert e.value.code == 7                  # TLQR_ERR_TIMEOUT
    finally:
        s.close()
    torch.cuda.synchronize()                      # the context is still usable
    out, _ = solve(p, n, m, data, MIXED, async_ops=1 << 30)
    ref = riccati.tree_riccati(p, n, m, data)
    assert riccati.forward_error(out, ref, p) <= 1e-6


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_async_solve_passes_match_round_by_round(case, precision):
    """The affine and state passes of the right-hand side, each one
    level-asynchronous launch over every round, give the solution of the
    round-by-round passes (same per-operation arithmetic)."""
    name, p, n, m, d, forest = case
    if precision == FP64 and n == 32:
        pytest.skip("FP64 at n = 32 runs the run-time-n kernels")
    a, _ = solve(p, n, m, d, precision, forest=forest, async_ops=-1, async_solve=1)
    b, _ = solve(p, n, m, d, precision, forest=forest, async_ops=-1, async_solve=-1)
    tol = 1e-12 if precision == FP64 else 1e-9
    for k in ("x", "u", "y"):
        assert np.abs(a[k] - b[k]).max() <= tol * max(1.0, np.abs(b[k]).max()), k


def test_async_solve_is_two_launches_per_pass():
    rng = inputs.rng_for(904)
    p = inputs.long_trunk_tree(rng, trunk=300, total=3000)
    n, m = 12, 4
    d = {k: dev(v) for k, v in inputs.problem_data(p, n, m, rng).items()}
    N = len(p)
    s = tlqr.TreeLQR(p, n, m, MIXED, use_graphs=False, async_solve=1)
    try:
        tlqr.tlqr_factor(s.f, d)
        tlqr.tlqr_profile_read(s.f)
        out = [torch.zeros(sh, dtype=torch.float64, device="cuda") for sh in ((N, n), (N, m), (N, n))]
        tlqr.tlqr_solve_rhs(s.f, d["q"], d["r"], d["c"], *out)
        torch.cuda.synchronize()
        prof = tlqr.tlqr_profile_read(s.f)
    finally:
        s.close()
    assert prof["aff_tail"]["launches"] == 1 and prof["state_tail"]["launches"] == 1
    for k in ("aff_rake", "aff_absorb", "aff_compress", "aff_expand", "state_compress", "state_expand"):
        assert prof[k]["launches"] == 0, k
