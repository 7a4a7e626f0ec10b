"""The node-organised float-float residual of eq. (kkt) -- each node's FP64
blocks staged in shared memory by bulk copies (TMA) that complete on
mbarriers -- against the oracle's FP64 residual and against the
row-per-thread kernels, at every compile-time (n, m), for one tree and for a
forest; the refinement's use of it (zero Delta blocks not copied); the
fallback to the row kernels for unaligned arrays; and its bounded waits.

Tolerances: the float-float residual keeps ~47 significant bits and rounds
each residual entry to FP32, so ||K z - b|| and eta agree with the FP64
oracle to a few FP32 ulps (rel 1e-6); the two kernel organisations agree with
each other to the same bound.
"""
import numpy as np
import pytest

from oracle import riccati
from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED = tlqr.TLQR_PREC_MIXED
PAIRS = [(4, 2), (6, 2), (8, 2), (12, 4), (16, 4), (32, 8)]


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _case(n, m, forest, seed, N=1300):
    rng = inputs.rng_for(seed)
    if forest:
        trees = [inputs.random_recursive(int(rng.integers(1, 400)), rng) for _ in range(7)] + [inputs.chain(150)]
        datas = [inputs.problem_data(p, n, m, rng, delta="subset", delta_value=0.05, delta_fraction=0.3,
                                     M_scale=0.2) for p in trees]
        par, offs = inputs.forest(trees)
        return par, inputs.concat_data(datas), rng, (trees, offs, datas)
    p, _ = inputs.permute_labels(inputs.random_recursive(N, rng), rng)
    d = inputs.problem_data(p, n, m, rng, delta="subset", delta_value=0.05, delta_fraction=0.3, M_scale=0.2)
    return p, d, rng, None


def _residual(p, n, m, d, x, u, y, kind, forest):
    s = tlqr.TreeLQR(p, n, m, MIXED, has_M=True, has_delta=True, residual=kind, forest=forest)
    try:
        st = tlqr.tlqr_kkt_residual(s.f, {k: dev(v) for k, v in d.items()}, dev(x), dev(u), dev(y))
        per_tree = tlqr.tlqr_tree_residuals(s.f, s.stats()["n_trees"]) if forest else None
    finally:
        s.close()
    return st, per_tree


@pytest.mark.parametrize("n,m", PAIRS)
@pytest.mark.parametrize("forest", [False, True])
def test_node_residual_matches_oracle_and_row_kernels(n, m, forest):
    p, d, rng, parts = _case(n, m, forest, 1300 + 10 * n + forest)
    N = len(p)
    x, u, y = rng.standard_normal((N, n)), rng.standard_normal((N, m)), rng.standard_normal((N, n))
    u[np.asarray(p) < 0] = 0
    st_rows, pt_rows = _residual(p, n, m, d, x, u, y, 1, forest)
    st_nodes, pt_nodes = _residual(p, n, m, d, x, u, y, 2, forest)
    if not forest:
        ref = riccati.kkt_residual(p, n, m, d, x, u, y)
        for st in (st_rows, st_nodes):
            assert st["abs"] == pytest.approx(ref["abs"], rel=1e-6)
            assert st["eta"] == pytest.approx(ref["eta"], rel=1e-6)
    else:
        trees, offs, datas = parts
        for t, pt in enumerate(trees):
            sl = slice(offs[t], offs[t] + len(pt))
            ref = riccati.kkt_residual(pt, n, m, datas[t], x[sl], u[sl], y[sl])
            for absr, eta in (pt_rows, pt_nodes):
                assert absr[t] == pytest.approx(ref["abs"], rel=1e-6)
                assert eta[t] == pytest.approx(ref["eta"], rel=1e-6)
    assert st_nodes["abs"] == pytest.approx(st_rows["abs"], rel=1e-6)
    assert st_nodes["eta"] == pytest.approx(st_rows["eta"], rel=1e-6)


@pytest.mark.parametrize("n,m", [(12, 4), (16, 4), (32, 8)])
def test_refinement_through_node_residual(n, m):
    """Refined mixed solves with the node residual (which skips the zero Delta
    blocks the condensation flagged) reach the oracle's solution; the eta the
    refinement reports is the oracle's eta of the returned solution."""
    p, d, _, _ = _case(n, m, False, 1400 + n, N=2000)
    N = len(p)
    ref = riccati.tree_riccati(p, n, m, d)
    for kind in (1, 2):
        s = tlqr.TreeLQR(p, n, m, MIXED, has_M=True, has_delta=True, residual=kind)
        try:
            x = torch.zeros((N, n), dtype=torch.float64, device="cuda")
            u = torch.zeros((N, m), dtype=torch.float64, device="cuda")
            y = torch.zeros((N, n), dtype=torch.float64, device="cuda")
            tlqr.tlqr_solve(s.f, {k: dev(v) for k, v in d.items()}, x, u, y)
            info = tlqr.tlqr_last_info(s.f)
        finally:
            s.close()
        out = dict(x=x.cpu().numpy(), u=u.cpu().numpy(), y=y.cpu().numpy())
        res = riccati.kkt_residual(p, n, m, d, out["x"], out["u"], out["y"])
        assert info["eta"] <= 1e-8 and res["eta"] <= 1e-8
        assert abs(info["eta"] - res["eta"]) <= 1e-13
        assert riccati.forward_error(out, ref, p) <= 1e-6


def test_unaligned_arrays_fall_back_to_row_kernels():
    """Matrix arrays that do not start on a 16-byte boundary cannot be bulk
    copied: the call takes the row kernels and gives the same residual."""
    n, m = 12, 4
    p, d, rng, _ = _case(n, m, False, 1500, N=600)
    N = len(p)
    x, u, y = rng.standard_normal((N, n)), rng.standard_normal((N, m)), rng.standard_normal((N, n))
    u[np.asarray(p) < 0] = 0

    def shifted(a):                              # same values, address 8 bytes past a 16-byte boundary
        flat = np.ascontiguousarray(a, dtype=np.float64).ravel()
        buf = torch.zeros(flat.size + 1, dtype=torch.float64, device="cuda")
        buf[1:] = torch.from_numpy(flat).cuda()
        v = buf[1:].view(a.shape)
        assert v.data_ptr() % 16 == 8
        return v

    s = tlqr.TreeLQR(p, n, m, MIXED, has_M=True, has_delta=True, residual=2)
    try:
        dd = {k: (shifted(v) if k in ("Q", "A", "B", "R", "M", "Delta") else dev(v)) for k, v in d.items()}
        st = tlqr.tlqr_kkt_residual(s.f, dd, dev(x), dev(u), dev(y))
    finally:
        s.close()
    ref = riccati.kkt_residual(p, n, m, d, x, u, y)
    assert st["abs"] == pytest.approx(ref["abs"], rel=1e-6)
    assert st["eta"] == pytest.approx(ref["eta"], rel=1e-6)


def test_withheld_bulk_copy_times_out_and_context_survives():
    """A bulk copy that is announced to the mbarrier but never issued (host
    switch for testing) makes that bounded wait run out: the solve returns
    TLQR_ERR_TIMEOUT, and the next solve on the device succeeds."""
    n, m = 12, 4
    p, d, _, _ = _case(n, m, False, 1600, N=800)
    N = len(p)
    dd = {k: dev(v) for k, v in d.items()}
    s = tlqr.TreeLQR(p, n, m, MIXED, has_M=True, has_delta=True, residual=2, test_withhold=2, spin_limit=2000)
    try:
        x = torch.zeros((N, n), dtype=torch.float64, device="cuda")
        u = torch.zeros((N, m), dtype=torch.float64, device="cuda")
        y = torch.zeros((N, n), dtype=torch.float64, device="cuda")
        with pytest.raises(tlqr.TLQRError) as e:
            tlqr.tlqr_solve(s.f, dd, x, u, y)
        assert e.value.code == tlqr.TLQR_ERR_TIMEOUT
    finally:
        s.close()
    s = tlqr.TreeLQR(p, n, m, MIXED, has_M=True, has_delta=True, residual=2)
    try:
        tlqr.tlqr_solve(s.f, dd, x, u, y)
        assert tlqr.tlqr_last_info(s.f)["eta"] <= 1e-8
    finally:
        s.close()
