"""Adjoint solve through the right-hand side (tlqr_solve_adjoint) against the
brute-force dense KKT system: for z = -K^{-1} b (eq. (kkt), b = (q, r, c) in
its row blocks) the gradient of L = <zbar, z> with respect to b is
-K^{-1} zbar, computed here by a dense LAPACK solve of the assembled matrix;
also a finite-difference check of one directional derivative."""
import numpy as np
import pytest

from oracle import dense
from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = tlqr.TLQR_PREC_FP64, tlqr.TLQR_PREC_MIXED


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def dense_grad(parent, n, m, data, xbar, ubar, ybar):
    K, b, (X, U, Y, nonroot) = dense.assemble_kkt(parent, n, m, data)
    zbar = np.zeros(K.shape[0])
    N = len(parent)
    for i in range(N):
        zbar[X(i)] = xbar[i]
        zbar[Y(i)] = ybar[i]
    for j in nonroot:
        zbar[U(j)] = ubar[j]
    g = -np.linalg.solve(K, zbar)
    qb = np.stack([g[X(i)] for i in range(N)])
    cb = np.stack([g[Y(i)] for i in range(N)])
    rb = np.zeros((N, m))
    for j in nonroot:
        rb[j] = g[U(j)]
    return qb, rb, cb


@pytest.mark.parametrize("n,m", [(3, 2), (12, 4), (16, 4)])
@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("host", [False, True])
def test_adjoint_equals_dense_gradient(n, m, precision, host):
    rng = inputs.rng_for(1100 + n)
    p, _ = inputs.permute_labels(inputs.random_recursive(60, rng), rng)
    d = inputs.problem_data(p, n, m, rng, M_scale=0.2, delta="subset", delta_value=0.1, delta_fraction=0.3)
    N = len(p)
    xbar, ubar, ybar = rng.standard_normal((N, n)), rng.standard_normal((N, m)), rng.standard_normal((N, n))
    root = int(np.nonzero(p < 0)[0][0])
    ubar[root] = 0.0
    qb_ref, rb_ref, cb_ref = dense_grad(p, n, m, d, xbar, ubar, ybar)
    s = tlqr.TreeLQR(p, n, m, precision, has_M=True, has_delta=True)
    try:
        dd = {k: dev(v) for k, v in d.items()}
        tlqr.tlqr_factor(s.f, dd)
        if host:
            qb, rb, cb = np.zeros((N, n)), np.zeros((N, m)), np.zeros((N, n))
            tlqr.tlqr_solve_adjoint(s.f, xbar, ubar, ybar, qb, rb, cb)
        else:
            out = [torch.zeros(sh, dtype=torch.float64, device="cuda") for sh in ((N, n), (N, m), (N, n))]
            tlqr.tlqr_solve_adjoint(s.f, dev(xbar), dev(ubar), dev(ybar), *out)
            torch.cuda.synchronize()
            qb, rb, cb = (o.cpu().numpy() for o in out)
    finally:
        s.close()
    tol = 1e-10 if precision == FP64 else 1e-6
    scale = max(np.abs(qb_ref).max(), np.abs(rb_ref).max(), np.abs(cb_ref).max())
    for got, want in ((qb, qb_ref), (rb, rb_ref), (cb, cb_ref)):
        assert np.abs(got - want).max() <= tol * scale
    assert np.all(rb[root] == 0.0)


def test_adjoint_matches_finite_differences():
    """<zbar, z(b + h e)> - <zbar, z(b)> = h <bbar, e> exactly for this linear
    map; checked in FP64 with the solver itself."""
    rng = inputs.rng_for(1200)
    p = inputs.long_trunk_tree(rng, trunk=60, total=400)
    n, m = 4, 2
    d = inputs.problem_data(p, n, m, rng)
    N = len(p)
    s = tlqr.TreeLQR(p, n, m, FP64)
    try:
        dd = {k: dev(v) for k, v in d.items()}
        tlqr.tlqr_factor(s.f, dd)
        zb = [rng.standard_normal(sh) for sh in ((N, n), (N, m), (N, n))]
        zb[1][0] = 0.0
        bb = [torch.zeros(sh, dtype=torch.float64, device="cuda") for sh in ((N, n), (N, m), (N, n))]
        tlqr.tlqr_solve_adjoint(s.f, *[dev(a) for a in zb], *bb)
        e = [rng.standard_normal(sh) for sh in ((N, n), (N, m), (N, n))]
        e[1][0] = 0.0

        def objective(q, r, c):
            out = [torch.zeros(sh, dtype=torch.float64, device="cuda") for sh in ((N, n), (N, m), (N, n))]
            tlqr.tlqr_solve_rhs(s.f, dev(q), dev(r), dev(c), *out)
            torch.cuda.synchronize()
            return sum(float((o.cpu().numpy() * z).sum()) for o, z in zip(out, zb))

        h = 1e-3
        base = objective(d["q"], d["r"], d["c"])
        pert = objective(d["q"] + h * e[0], d["r"] + h * e[1], d["c"] + h * e[2])
        directional = sum(float((b.cpu().numpy() * ee).sum()) for b, ee in zip(bb, e))
        assert abs((pert - base) / h - directional) <= 1e-8 * max(1.0, abs(directional))
    finally:
        s.close()
