"""Several right-hand sides with one factorisation (tlqr_solve_rhs_panel):
each right-hand side of a panel gets the solution that tlqr_solve_rhs gives it
alone -- the panel kernels apply each factor block to all of them with the same
per-right-hand-side arithmetic -- and the FP64 panel solution matches the
oracle.  Panels of 1, 3, 8 and 11 (two chunks); n = 12, 16, 32 run the panel
kernels, n = 5 (run-time-n kernels) the one-by-one path."""
import numpy as np
import pytest

from oracle import riccati
from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = tlqr.TLQR_PREC_FP64, tlqr.TLQR_PREC_MIXED


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("n,m", [(12, 4), (16, 4), (32, 8), (5, 3)])
@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("nrhs", [1, 3, 8, 11])
def test_panel_equals_one_by_one(n, m, precision, nrhs):
    if precision == FP64 and n == 32:
        pytest.skip("FP64 at n = 32 runs the run-time-n kernels (covered by n = 5)")
    rng = inputs.rng_for(1500 + n + nrhs)
    p = inputs.long_trunk_tree(rng, trunk=200, total=1500)
    d = inputs.problem_data(p, n, m, rng, delta="subset", delta_value=0.05)
    N = len(p)
    s = tlqr.TreeLQR(p, n, m, precision, has_delta=True)
    try:
        dd = {k: dev(v) for k, v in d.items()}
        tlqr.tlqr_factor(s.f, dd)
        rh = [inputs.rhs_data(p, n, m, rng) for _ in range(nrhs)]
        Q = dev(np.stack([r["q"] for r in rh])); Rr = dev(np.stack([r["r"] for r in rh]))
        C = dev(np.stack([r["c"] for r in rh]))
        X = torch.zeros((nrhs, N, n), dtype=torch.float64, device="cuda")
        U = torch.zeros((nrhs, N, m), dtype=torch.float64, device="cuda")
        Y = torch.zeros((nrhs, N, n), dtype=torch.float64, device="cuda")
        tlqr.tlqr_solve_rhs_panel(s.f, Q, Rr, C, X, U, Y)
        torch.cuda.synchronize()
        for k in range(nrhs):
            x = torch.zeros((N, n), dtype=torch.float64, device="cuda")
            u = torch.zeros((N, m), dtype=torch.float64, device="cuda")
            y = torch.zeros((N, n), dtype=torch.float64, device="cuda")
            tlqr.tlqr_solve_rhs(s.f, Q[k], Rr[k], C[k], x, u, y)
            torch.cuda.synchronize()
            for a, b in ((X[k], x), (U[k], u), (Y[k], y)):
                a, b = a.cpu().numpy(), b.cpu().numpy()
                assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max())
        if precision == FP64:
            dk = dict(d)
            dk.update(q=rh[-1]["q"], r=rh[-1]["r"], c=rh[-1]["c"])
            ref = riccati.tree_riccati(p, n, m, dk)
            out = dict(x=X[-1].cpu().numpy(), u=U[-1].cpu().numpy(), y=Y[-1].cpu().numpy())
            assert riccati.forward_error(out, ref, p) <= 1e-9
    finally:
        s.close()
