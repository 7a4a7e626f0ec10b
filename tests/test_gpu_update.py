"""tlqr_update_solve: in-place diagonal and right-hand-side updates of the
resident problem, then factor + solve, equal to solving the updated problem
from scratch (bitwise: the same kernels on the same data) and to the oracle."""
import numpy as np
import pytest

from oracle import riccati
from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = tlqr.TLQR_PREC_FP64, tlqr.TLQR_PREC_MIXED


def _host_solve(f, d, N, n, m):
    x, u, y = np.zeros((N, n)), np.zeros((N, m)), np.zeros((N, n))
    tlqr.tlqr_solve(f, d, x, u, y)
    return x, u, y


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("n,m", [(12, 4), (5, 3), (2, 5)])
def test_update_equals_fresh_solve(precision, n, m):
    rng = inputs.rng_for(1700 + n + 10 * m)
    p = inputs.random_recursive(1500, rng)
    N = len(p)
    d = inputs.problem_data(p, n, m, rng, delta="subset", delta_value=0.05)
    d = {k: (None if v is None else np.ascontiguousarray(v)) for k, v in d.items()}
    s = tlqr.TreeLQR(p, n, m, precision, has_delta=True)
    t = tlqr.TreeLQR(p, n, m, precision, has_delta=True)
    try:
        _host_solve(s.f, d, N, n, m)
        d2 = dict(d)
        for it in range(3):                      # an interior-point-like sequence of diagonal changes
            dq = np.abs(rng.standard_normal((N, n))) * 0.1
            dr = np.abs(rng.standard_normal((N, m))) * 0.1
            q, r, c = rng.standard_normal((N, n)), rng.standard_normal((N, m)), rng.standard_normal((N, n))
            x, u, y = np.zeros((N, n)), np.zeros((N, m)), np.zeros((N, n))
            tlqr.tlqr_update_solve(s.f, x, u, y, dq=dq, dr=dr, q=q, r=r, c=c)
            Q2, R2 = d2["Q"].copy(), d2["R"].copy()
            Q2[:, np.arange(n), np.arange(n)] += dq
            R2[:, np.arange(m), np.arange(m)] += dr
            d2 = dict(d2, Q=Q2, R=R2, q=q, r=r, c=c)
            xf, uf, yf = _host_solve(t.f, d2, N, n, m)
            for a, b in ((x, xf), (u, uf), (y, yf)):
                np.testing.assert_array_equal(a, b)
        ref = riccati.tree_riccati(p, n, m, d2)
        fe = riccati.forward_error(dict(x=x, u=u, y=y), ref, p)
        assert fe <= (1e-8 if precision == FP64 else 1e-6)
    finally:
        s.close()
        t.close()


def test_update_device_arrays_in_place_and_partial():
    """Device problems: the caller's Q and R receive the increments; arguments
    left out keep their values (here: only dr and c change)."""
    n, m = 6, 2
    rng = inputs.rng_for(1750)
    p = inputs.random_recursive(800, rng)
    N = len(p)
    d = inputs.problem_data(p, n, m, rng)
    dd = {k: (None if v is None else torch.from_numpy(np.ascontiguousarray(v)).cuda()) for k, v in d.items()}
    s = tlqr.TreeLQR(p, n, m, FP64)
    try:
        x = torch.zeros((N, n), dtype=torch.float64, device="cuda")
        u = torch.zeros((N, m), dtype=torch.float64, device="cuda")
        y = torch.zeros((N, n), dtype=torch.float64, device="cuda")
        tlqr.tlqr_solve(s.f, dd, x, u, y)
        dr = torch.from_numpy(np.full((N, m), 0.25)).cuda()
        c = torch.from_numpy(rng.standard_normal((N, n))).cuda()
        tlqr.tlqr_update_solve(s.f, x, u, y, dr=dr, c=c)
        torch.cuda.synchronize()
        R2 = d["R"].copy()
        R2[:, np.arange(m), np.arange(m)] += 0.25
        np.testing.assert_array_equal(dd["R"].cpu().numpy(), R2)
        np.testing.assert_array_equal(dd["Q"].cpu().numpy(), d["Q"])
        d2 = dict(d, R=R2, c=c.cpu().numpy())
        ref = riccati.tree_riccati(p, n, m, d2)
        out = dict(x=x.cpu().numpy(), u=u.cpu().numpy(), y=y.cpu().numpy())
        assert riccati.forward_error(out, ref, p) <= 1e-8
    finally:
        s.close()


def test_update_before_any_factorisation_is_refused():
    p = inputs.chain(10)
    s = tlqr.TreeLQR(p, 3, 2, FP64)
    try:
        x, u, y = np.zeros((10, 3)), np.zeros((10, 2)), np.zeros((10, 3))
        with pytest.raises(tlqr.TLQRError) as e:
            tlqr.tlqr_update_solve(s.f, x, u, y, dq=np.ones((10, 3)))
        assert e.value.code == 10                # TLQR_ERR_STATE
    finally:
        s.close()
