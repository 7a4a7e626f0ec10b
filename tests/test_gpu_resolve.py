"""FP64 re-solves of ill-conditioned eliminations in mixed precision.

With Delta = 0, a control weight R of condition number 1e8 (spectrum
1 .. 1e8) and a state weight Q scaled by 1e6, the node data U and value
Hessians P reach ~1e7 while C = B R^{-1} B^T stays O(1), so the systems
S = I + C U and S = I + C P~ of the rake, compression and reconstruction
have pivots spanning ~1e6-1e7, far more than 1e4: the FP32 kernels re-solve
those in FP64 (eq. (terminal-fold), eq. (compress-intermediates)).  (A tiny
R instead would make C ~ 1e8 but also ruin the FP32 condensation itself,
which no re-solve of S can repair.)  The refined solution must match the
FP64 oracle and reach eta <= 1e-8; the factorisation must report the
re-solves it took, and none when they are off.
"""
import numpy as np
import pytest

from oracle import riccati
from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED = tlqr.TLQR_PREC_MIXED


def _ill_case(n, m, N, seed):
    rng = inputs.rng_for(seed)
    p, _ = inputs.permute_labels(inputs.random_recursive(N, rng), rng)
    d = inputs.problem_data(p, n, m, rng, kappa_R=1e8)
    d["Q"] = d["Q"] * 1e6
    return p, d


def _solve(p, n, m, d, **kw):
    N = len(p)
    s = tlqr.TreeLQR(p, n, m, MIXED, **kw)
    try:
        dd = {k: (None if v is None else torch.from_numpy(np.ascontiguousarray(v)).cuda()) for k, v in d.items()}
        x = torch.zeros((N, n), dtype=torch.float64, device="cuda")
        u = torch.zeros((N, m), dtype=torch.float64, device="cuda")
        y = torch.zeros((N, n), dtype=torch.float64, device="cuda")
        code = 0
        try:
            tlqr.tlqr_solve(s.f, dd, x, u, y)
        except tlqr.TLQRError as e:
            code = e.code
        info = tlqr.tlqr_last_info(s.f)
        return code, info, dict(x=x.cpu().numpy(), u=u.cpu().numpy(), y=y.cpu().numpy())
    finally:
        s.close()


@pytest.mark.parametrize("n,m", [(12, 4), (16, 4), (8, 2), (32, 8)])
def test_ill_conditioned_S_is_resolved_in_fp64(n, m):
    p, d = _ill_case(n, m, 1500 if n < 32 else 600, 1800 + n)
    code, info, out = _solve(p, n, m, d)
    assert code == 0, code
    assert 0 < info["fp64_resolves"] <= 4096
    assert info["eta"] <= 1e-8
    res = riccati.kkt_residual(p, n, m, d, out["x"], out["u"], out["y"])
    assert res["eta"] <= 1e-8 and abs(res["eta"] - info["eta"]) <= 1e-13
    ref = riccati.tree_riccati(p, n, m, d)
    assert riccati.forward_error(out, ref, p) <= 1e-6
    # switched off: no re-solves are taken (whatever the refinement then reaches)
    code_off, info_off, _ = _solve(p, n, m, d, fp64_resolve=-1)
    assert info_off["fp64_resolves"] == 0
    assert code_off in (0, tlqr.TLQR_ERR_NO_CONVERGENCE, 4, 5)


def test_well_conditioned_problem_takes_no_resolve():
    """The c1-like data (kappa(R) small, Delta on a subset): no pivot ratio
    exceeds the threshold, so the FP32 path stands everywhere."""
    rng = inputs.rng_for(1850)
    p = inputs.long_trunk_tree(rng, trunk=300, total=3000)
    d = inputs.problem_data(p, 12, 4, rng, delta="subset", delta_value=1e-6)
    code, info, _ = _solve(p, 12, 4, d, has_delta=True)
    assert code == 0 and info["fp64_resolves"] == 0 and info["eta"] <= 1e-8
