"""FP64 re-solves of ill-conditioned eliminations in mixed precision.

A re-solve makes one operation exact up to the rounding of its result for
the FP32 operands it was given; it cannot undo the rounding of those
operands.  So the per-operation test gives the kernels operands that FP32
holds exactly (the oracle then computes the same operation on the same
numbers): with U ~ 1e6 and C = B R^{-1} B^T of rank m (kappa(R) = 1e8) the
pivots of S = I + C U span ~1e6, and the compile-time-n kernels (which
re-solve) must match the FP64 oracle to FP32 accuracy where the run-time-n
kernels (which do not) lose ~1e-2.  The whole-solve test (Delta = 0,
kappa(R) = 1e8, Q scaled by 1e3) takes re-solves in its rake, compression
and reconstruction steps and must still match the oracle after refinement;
well-conditioned data must take none.
"""
import numpy as np
import pytest

from oracle import ops, riccati  # noqa: F401
from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED = tlqr.TLQR_PREC_MIXED


def _ill_case(n, m, N, seed):
    rng = inputs.rng_for(seed)
    p, _ = inputs.permute_labels(inputs.random_recursive(N, rng), rng)
    d = inputs.problem_data(p, n, m, rng, kappa_R=1e8)
    d["Q"] = d["Q"] * 1e3
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
    # the backward error is what the refinement controls; this KKT system is ill-conditioned
    # enough (Q ~ 1e3..1e4, kappa(R) = 1e8) that eta = 1e-8 allows forward errors of ~1e-2
    res = riccati.kkt_residual(p, n, m, d, out["x"], out["u"], out["y"])
    assert res["eta"] <= 1e-8 and abs(res["eta"] - info["eta"]) <= 1e-13
    # switched off: no re-solves are taken (the refinement still converges here)
    code_off, info_off, _ = _solve(p, n, m, d, fp64_resolve=-1)
    assert info_off["fp64_resolves"] == 0
    assert code_off in (0, 3, 4, 5, tlqr.TLQR_ERR_NO_CONVERGENCE)


def test_well_conditioned_problem_takes_no_resolve():
    """The c1-like data (kappa(R) small, Delta on a subset): no pivot ratio
    exceeds the threshold, so the FP32 path stands everywhere."""
    rng = inputs.rng_for(1850)
    p = inputs.long_trunk_tree(rng, trunk=300, total=3000)
    d = inputs.problem_data(p, 12, 4, rng, delta="subset", delta_value=1e-6)
    code, info, _ = _solve(p, 12, 4, d, has_delta=True)
    assert code == 0 and info["fp64_resolves"] == 0 and info["eta"] <= 1e-8


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _f32(a):
    """The same numbers rounded to FP32 (held exactly by both sides)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("n,m", [(8, 2), (12, 4), (16, 4), (32, 8)])
def test_batched_rake_and_compression_with_large_U(n, m):
    """The per-operation kernels on FP32-exact blocks with U ~ 1e6 and
    C = B R^{-1} B^T of rank m (kappa(R) = 1e8): the re-solve forms S, solves
    it and forms U Y and P~ Y1 in FP64, so the compile-time-n kernels stay
    within 1e-5 (relative to the largest entry) of the FP64 oracle, where the
    run-time-n kernels (no re-solves) lose ~1e-2."""
    rng = inputs.rng_for(1900 + n)
    count = 48
    B = rng.standard_normal((count, n, m)) / np.sqrt(n)
    ev = np.logspace(0, 8, m)
    C = _f32((B / ev[None, None, :]) @ B.transpose(0, 2, 1))
    G = rng.standard_normal((count, n, n))
    U = _f32(1e6 * (G @ G.transpose(0, 2, 1)) / n + 1e5 * np.eye(n))
    A = _f32(rng.standard_normal((count, n, n)) / np.sqrt(n))
    H = rng.standard_normal((count, n, n))
    P = _f32(0.05 * H @ H.transpose(0, 2, 1) / n)
    ref = np.stack([ops.tau(A[t], C[t], P[t], U[t]) for t in range(count)])
    errs = {}
    for name, prec in (("fixed", MIXED), ("generic", MIXED | tlqr.TLQR_BATCHED_GENERIC)):
        out = _dev(np.zeros((count, n, n)))
        tlqr.tlqr_batched_tau(_dev(A), _dev(C), _dev(P), _dev(U), out, prec)
        errs[name] = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert errs["fixed"] <= 1e-5, errs
    assert errs["generic"] > 10 * errs["fixed"], errs
    # compression with the large block in P~ = P_r + U
    Ar = _f32(rng.standard_normal((count, n, n)) / np.sqrt(n))
    K = rng.standard_normal((count, n, n))
    Cr = _f32(0.1 * K @ K.transpose(0, 2, 1) / n)
    Pr = P.copy()                                # P~ = P_r + U is rounded once in FP32: benign (C P~ stays
                                                 # accurate to FP32 in every direction)
    outs = [_dev(np.zeros((count, n, n))) for _ in range(4)]
    tlqr.tlqr_batched_compose(_dev(A), _dev(C), _dev(P), _dev(Ar), _dev(Cr), _dev(Pr), _dev(U), *outs, MIXED)
    got = [o.cpu().numpy() for o in outs]
    for t in range(count):
        (a, c, pn), tape = ops.compose((Ar[t], Cr[t], Pr[t]), (A[t], C[t], P[t]), U[t])
        for g_, want in ((got[0][t], a), (got[1][t], c), (got[2][t], pn), (got[3][t], tape[2])):
            assert np.abs(g_ - want).max() <= 1e-5 * max(1.0, np.abs(want).max())
