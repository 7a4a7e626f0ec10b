"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (derived from the arithmetic; the accuracy targets are stated as
backward errors):
  * FP64 path: eta <= 1e-10 (normwise backward error of eq. (kkt)); elementwise
    |z - z_oracle| <= 1e-8 max|z_oracle| for z = (x, u, y), and P, K within
    1e-8 of the oracle relative to their largest entry.  Both sides are
    backward stable FP64 methods on well-conditioned data, so their difference
    is a few hundred ulps times the condition number.
  * MIXED path (FP32 factors + FP64 refinement): eta <= 1e-8 after
    refinement; forward error vs the oracle <= 1e-6.
  * Batched primitives: FP64 within 1e-10 relative; FP32 within 2e-4 relative
    (n <= 16, a few FP32 roundings amplified by the local condition number).
"""
import numpy as np
import pytest

from oracle import ops, riccati
from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = tlqr.TLQR_PREC_FP64, tlqr.TLQR_PREC_MIXED


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def gpu_solve(parent, n, m, data, precision=FP64, host=False, want_PK=True, **kw):
    N = len(parent)
    s = tlqr.TreeLQR(parent, n, m, precision, has_M=data.get("M") is not None,
                     has_delta=data.get("Delta") is not None, **kw)
    try:
        if host:
            d = {k: (None if v is None else np.ascontiguousarray(v)) for k, v in data.items()}
            x, u, y = np.zeros((N, n)), np.zeros((N, m)), np.zeros((N, n))
            P, K = (np.zeros((N, n, n)), np.zeros((N, m, n))) if want_PK else (None, None)
            tlqr.tlqr_solve(s.f, d, x, u, y, P, K)
            out = dict(x=x, u=u, y=y, P=P, K=K)
        else:
            d = {k: dev(v) for k, v in data.items()}
            x = torch.zeros((N, n), dtype=torch.float64, device="cuda")
            u = torch.zeros((N, m), dtype=torch.float64, device="cuda")
            y = torch.zeros((N, n), dtype=torch.float64, device="cuda")
            P = torch.zeros((N, n, n), dtype=torch.float64, device="cuda") if want_PK else None
            K = torch.zeros((N, m, n), dtype=torch.float64, device="cuda") if want_PK else None
            tlqr.tlqr_solve(s.f, d, x, u, y, P, K)
            torch.cuda.synchronize()
            out = dict(x=x.cpu().numpy(), u=u.cpu().numpy(), y=y.cpu().numpy(),
                       P=None if P is None else P.cpu().numpy(), K=None if K is None else K.cpu().numpy())
        out["info"] = tlqr.tlqr_last_info(s.f)
        if kw.get("forest"):
            out["tree_eta"] = tlqr.tlqr_tree_residuals(s.f, s.stats()["n_trees"])[1]
        return out
    finally:
        s.close()


def check_against_oracle(parent, n, m, data, out, fwd_tol, eta_tol, pk_tol=None):
    ref = riccati.tree_riccati(parent, n, m, data)
    fe = riccati.forward_error(out, ref, parent)
    res = riccati.kkt_residual(parent, n, m, data, out["x"], out["u"], out["y"])
    assert res["eta"] <= eta_tol, res["eta"]
    assert fe <= fwd_tol, fe
    if pk_tol is not None and out.get("P") is not None:
        nonroot = np.asarray(parent) >= 0
        assert np.abs(out["P"] - ref["P"]).max() <= pk_tol * np.abs(ref["P"]).max()
        if nonroot.any():
            assert np.abs(out["K"][nonroot] - ref["K"][nonroot]).max() <= pk_tol * max(1.0, np.abs(ref["K"]).max())
        np.testing.assert_array_equal(out["K"][~nonroot], 0.0)
    return fe, res["eta"]


# -------------------------------------------------------------------- batched primitives

@pytest.mark.parametrize("n", [1, 3, 4, 12, 16, 32])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_batched_tau_and_compose(n, precision):
    rng = inputs.rng_for(200 + n)
    count = 37                                   # several blocks of 8 warps plus a ragged tail
    def psd(k=None, s=1.0):
        G = rng.standard_normal((count, n, k or n))
        return s * G @ G.transpose(0, 2, 1) / n
    A = rng.standard_normal((count, n, n)) / np.sqrt(n)
    C, U, P = psd(), psd() + 0.5 * np.eye(n), -psd(1, 0.05)
    out = dev(np.zeros((count, n, n)))
    tlqr.tlqr_batched_tau(dev(A), dev(C), dev(P), dev(U), out, precision)
    ref = np.stack([ops.tau(A[t], C[t], P[t], U[t]) for t in range(count)])
    tol = 1e-10 if precision == FP64 else 2e-4
    assert np.abs(out.cpu().numpy() - ref).max() <= tol * np.abs(ref).max()
    Ar = rng.standard_normal((count, n, n)) / np.sqrt(n)
    Cr, Pr = psd(), -psd(1, 0.05)
    An, Cn, Pn, Pt = (dev(np.zeros((count, n, n))) for _ in range(4))
    tlqr.tlqr_batched_compose(dev(A), dev(C), dev(P), dev(Ar), dev(Cr), dev(Pr), dev(U), An, Cn, Pn, Pt,
                              precision)
    for t in range(count):
        (a, c, p), tape = ops.compose((Ar[t], Cr[t], Pr[t]), (A[t], C[t], P[t]), U[t])
        for got, want in ((An, a), (Cn, c), (Pn, p), (Pt, tape[2])):
            g = got.cpu().numpy()[t]
            assert np.abs(g - want).max() <= tol * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("n,m", [(1, 1), (4, 2), (12, 4), (16, 4), (32, 8), (6, 9)])
@pytest.mark.parametrize("withM", [False, True])
def test_batched_condense(n, m, withM):
    rng = inputs.rng_for(300 + n * m)
    count = 19
    A = rng.standard_normal((count, n, n)); B = rng.standard_normal((count, n, m))
    H = rng.standard_normal((count, m, m)); R = np.eye(m) + H @ H.transpose(0, 2, 1)
    M = 0.3 * rng.standard_normal((count, n, m)) if withM else None
    Dg = rng.standard_normal((count, n, n)); D = 0.1 * Dg @ Dg.transpose(0, 2, 1)
    outs = [dev(np.zeros((count, n, n))) for _ in range(3)]
    tlqr.tlqr_batched_condense(dev(A), dev(B), dev(R), dev(M), dev(D), *outs, FP64)
    for t in range(count):
        want = ops.condense(A[t], B[t], R[t], None if M is None else M[t], D[t])
        for g, w in zip(outs, want):
            assert np.abs(g.cpu().numpy()[t] - w).max() <= 1e-10 * max(1.0, np.abs(w).max())


@pytest.mark.parametrize("n,m", [(4, 2), (12, 4), (16, 4), (32, 8), (5, 3)])
@pytest.mark.parametrize("precision", [MIXED, MIXED | tlqr.TLQR_BATCHED_GENERIC])
def test_batched_condense_mixed(n, m, precision):
    """The condensation in FP32, through the compile-time-(n, m) kernel the
    solver runs for these sizes and through the run-time-n kernel."""
    rng = inputs.rng_for(310 + n * m)
    count = 45
    A = rng.standard_normal((count, n, n)); B = rng.standard_normal((count, n, m)) / np.sqrt(n)
    H = rng.standard_normal((count, m, m)); R = np.eye(m) + H @ H.transpose(0, 2, 1) / m
    M = 0.3 * rng.standard_normal((count, n, m))
    Dg = rng.standard_normal((count, n, n)); D = 0.1 * Dg @ Dg.transpose(0, 2, 1) / n
    outs = [dev(np.zeros((count, n, n))) for _ in range(3)]
    tlqr.tlqr_batched_condense(dev(A), dev(B), dev(R), dev(M), dev(D), *outs, precision)
    for t in range(count):
        want = ops.condense(A[t], B[t], R[t], M[t], D[t])
        for g, w in zip(outs, want):
            assert np.abs(g.cpu().numpy()[t] - w).max() <= 2e-5 * max(1.0, np.abs(w).max())


def _psd(rng, count, n, k=None, s=1.0):
    G = rng.standard_normal((count, n, k or n))
    return s * G @ G.transpose(0, 2, 1) / n


@pytest.mark.parametrize("n", [1, 3, 4, 12, 16, 32])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_batched_expand(n, precision):
    """eq. (value-reconstruction) through the expansion kernel against the oracle."""
    rng = inputs.rng_for(500 + n)
    count = 37
    Ar = rng.standard_normal((count, n, n)) / np.sqrt(n)
    Cr = _psd(rng, count, n)
    Pt = _psd(rng, count, n) + 0.5 * np.eye(n)
    Pk = _psd(rng, count, n) + 0.2 * np.eye(n)
    Pj = dev(np.zeros((count, n, n)))
    tlqr.tlqr_batched_expand(dev(Ar), dev(Cr), dev(Pt), dev(Pk), Pj, precision)
    ref = np.stack([ops.expand_compress((Ar[t], Cr[t], Pt[t]), Pk[t]) for t in range(count)])
    tol = 1e-10 if precision == FP64 else 2e-4
    assert np.abs(Pj.cpu().numpy() - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("n,m", [(1, 1), (4, 2), (6, 2), (12, 4), (16, 4), (32, 8), (5, 3)])
@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("extras", ["none", "M_Delta"])
def test_batched_local_factor(n, m, precision, extras):
    """eq. (FW), (factor-local): K and T = F^{-1} A_cl against the oracle, with
    and without M and Delta (the F = I + Delta P solve)."""
    rng = inputs.rng_for(600 + 7 * n + m)
    count = 41
    P = _psd(rng, count, n) + np.eye(n)
    A = 0.95 * rng.standard_normal((count, n, n)) / np.sqrt(n)
    B = rng.standard_normal((count, n, m)) / np.sqrt(n)
    H = rng.standard_normal((count, m, m)); R = np.eye(m) + H @ H.transpose(0, 2, 1) / m
    M = 0.3 * rng.standard_normal((count, n, m)) if extras == "M_Delta" else None
    D = _psd(rng, count, n, 2, 0.3) if extras == "M_Delta" else None
    K, T = dev(np.zeros((count, m, n))), dev(np.zeros((count, n, n)))
    tlqr.tlqr_batched_local_factor(dev(P), dev(A), dev(B), dev(R), dev(M), dev(D), K, T, precision)
    tol = 1e-10 if precision == FP64 else 2e-4
    Kg, Tg = K.cpu().numpy(), T.cpu().numpy()
    for t in range(count):
        lf = ops.local_factor(P[t], A[t], B[t], R[t], None if M is None else M[t], None if D is None else D[t])
        assert np.abs(Kg[t] - lf["K"]).max() <= tol * max(1.0, np.abs(lf["K"]).max())
        assert np.abs(Tg[t] - lf["T"]).max() <= tol * max(1.0, np.abs(lf["T"]).max())


@pytest.mark.parametrize("n", [1, 4, 12, 16, 32])
@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_batched_compose_T(n, precision):
    """eq. (transition-compose): T_k T_j by the composite-transition kernel."""
    rng = inputs.rng_for(700 + n)
    count = 37
    Tk = rng.standard_normal((count, n, n)) / np.sqrt(n)
    Tj = rng.standard_normal((count, n, n)) / np.sqrt(n)
    out = dev(np.zeros((count, n, n)))
    tlqr.tlqr_batched_compose_T(dev(Tk), dev(Tj), out, precision)
    ref = np.stack([ops.transition_compose(Tk[t], np.zeros(n), Tj[t], np.zeros(n))[0] for t in range(count)])
    tol = 1e-12 if precision == FP64 else 1e-5
    assert np.abs(out.cpu().numpy() - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("n", [4, 12, 16, 32])
def test_batched_fixed_and_generic_kernels_agree(n):
    """The compile-time-n group kernels (Gauss-Jordan solves, tensor-core
    products at n = 32) and the run-time-n warp kernels (LU) give the same rake
    fold and compression in FP32 up to rounding."""
    rng = inputs.rng_for(800 + n)
    count = 29
    A = rng.standard_normal((count, n, n)) / np.sqrt(n)
    C, U, P = _psd(rng, count, n), _psd(rng, count, n) + 0.5 * np.eye(n), -_psd(rng, count, n, 1, 0.05)
    outs = []
    for prec in (MIXED, MIXED | tlqr.TLQR_BATCHED_GENERIC):
        o = dev(np.zeros((count, n, n)))
        tlqr.tlqr_batched_tau(dev(A), dev(C), dev(P), dev(U), o, prec)
        outs.append(o.cpu().numpy())
    assert np.abs(outs[0] - outs[1]).max() <= 2e-4 * np.abs(outs[1]).max()


def test_batched_compose_associativity():
    """eq. (node-aware-associativity) evaluated by the GPU compress kernel."""
    rng = inputs.rng_for(401)
    n, count = 8, 11
    def tri():
        G = rng.standard_normal((count, n, n))
        return (rng.standard_normal((count, n, n)) / np.sqrt(n), G @ G.transpose(0, 2, 1) / n,
                np.zeros((count, n, n)))
    e1, e2, e3 = tri(), tri(), tri()
    U1 = np.eye(n) + 0.3 * np.stack([np.diag(rng.random(n)) for _ in range(count)])
    U2 = np.eye(n) + 0.3 * np.stack([np.diag(rng.random(n)) for _ in range(count)])
    def comp(r, l, U):
        An, Cn, Pn, Pt = (dev(np.zeros((count, n, n))) for _ in range(4))
        tlqr.tlqr_batched_compose(dev(l[0]), dev(l[1]), dev(l[2]), dev(r[0]), dev(r[1]), dev(r[2]), dev(U),
                                  An, Cn, Pn, Pt, FP64)
        return tuple(t.cpu().numpy() for t in (An, Cn, Pn))
    left = comp(e3, comp(e2, e1, U1), U2)
    right = comp(comp(e3, e2, U2), e1, U1)
    for a, b in zip(left, right):
        assert np.abs(a - b).max() <= 1e-10 * max(1.0, np.abs(a).max())


# -------------------------------------------------------------------- end to end, FP64

def e1_population():
    rng = inputs.rng_for(12)
    cases = []
    fixed = [("chain", inputs.chain(9)), ("star", inputs.star(8)),
             ("irregular", np.array([-1, 0, 1, 1, 2, 4, 4, 5], dtype=np.int32)),
             ("balanced", inputs.balanced(13)), ("single", np.array([-1], dtype=np.int32))]
    k = 0
    for name, p in fixed:
        for delta in (None, "random"):
            n, m = 1 + k % 4, 1 + k % 3
            cases.append((f"{name}-{delta}-n{n}m{m}", p, n, m,
                          inputs.problem_data(p, n, m, rng, M_scale=0.3 if k % 2 else 0.0, delta=delta,
                                              delta_value=0.5)))
            k += 1
    for t in range(16):
        N = int(rng.integers(2, 31))
        p, _ = inputs.permute_labels(inputs.random_recursive(N, rng), rng)
        n, m = int(rng.integers(1, 5)), int(rng.integers(1, 4))
        cases.append((f"random{t}-N{N}-n{n}m{m}", p, n, m,
                      inputs.problem_data(p, n, m, rng, M_scale=0.3 if t % 2 else 0.0,
                                          delta=("random" if t % 3 else None), delta_value=0.3)))
    return cases


E1 = e1_population()


@pytest.mark.parametrize("case", E1, ids=[c[0] for c in E1])
def test_fp64_small_population(case):
    _, p, n, m, d = case
    out = gpu_solve(p, n, m, d)
    check_against_oracle(p, n, m, d, out, fwd_tol=1e-10, eta_tol=1e-13, pk_tol=1e-10)


TOPOLOGIES = [("chain", inputs.chain(1000)), ("star", inputs.star(1000)), ("balanced", inputs.balanced(1023)),
              ("comb", inputs.comb(1001)), ("tight", inputs.tightness_tree(64))]


@pytest.mark.parametrize("topo", TOPOLOGIES, ids=lambda t: t[0])
@pytest.mark.parametrize("n,m", [(4, 2), (12, 4)])
def test_fp64_topologies(topo, n, m):
    _, p = topo
    rng = inputs.rng_for(500 + n)
    d = inputs.problem_data(p, n, m, rng, delta="subset", delta_value=0.1, delta_fraction=0.3, M_scale=0.2)
    out = gpu_solve(p, n, m, d)
    check_against_oracle(p, n, m, d, out, fwd_tol=1e-8, eta_tol=1e-10, pk_tol=1e-8)


def test_fp64_binary_depth6():
    w = inputs.binary_depth6()
    out = gpu_solve(w.parent, w.n, w.m, w.data)
    fe, eta = check_against_oracle(w.parent, w.n, w.m, w.data, out, fwd_tol=1e-10, eta_tol=1e-12, pk_tol=1e-10)


def test_fp64_long_trunk_full_size():
    """The benchmark workload at full size (N = 65,536, n = 12, m = 4)."""
    w = inputs.long_trunk()
    out = gpu_solve(w.parent, w.n, w.m, w.data)
    check_against_oracle(w.parent, w.n, w.m, w.data, out, fwd_tol=1e-8, eta_tol=1e-10, pk_tol=1e-8)


def test_fp64_dimensions_32_8():
    rng = inputs.rng_for(77)
    p, _ = inputs.permute_labels(inputs.random_recursive(300, rng), rng)
    d = inputs.problem_data(p, 32, 8, rng, kappa_R=1e4)
    out = gpu_solve(p, 32, 8, d)
    check_against_oracle(p, 32, 8, d, out, fwd_tol=1e-8, eta_tol=1e-10, pk_tol=1e-8)


def test_host_and_device_memory_agree():
    rng = inputs.rng_for(78)
    p = inputs.random_recursive(500, rng)
    d = inputs.problem_data(p, 6, 2, rng, delta="subset", delta_value=0.2)
    a = gpu_solve(p, 6, 2, d, host=False)
    b = gpu_solve(p, 6, 2, d, host=True)
    for k in ("x", "u", "y", "P", "K"):
        np.testing.assert_array_equal(a[k], b[k])


def test_zero_delta_paths_agree():
    """Delta = NULL and an explicit all-zero Delta give the same result."""
    rng = inputs.rng_for(79)
    p = inputs.random_recursive(400, rng)
    d = inputs.problem_data(p, 5, 2, rng)
    a = gpu_solve(p, 5, 2, d)
    b = gpu_solve(p, 5, 2, dict(d, Delta=np.zeros((len(p), 5, 5))))
    for k in ("x", "u", "y", "P", "K"):
        assert np.abs(a[k] - b[k]).max() <= 1e-12 * max(1.0, np.abs(a[k]).max())


def test_factor_reuse_multiple_rhs():
    """Sec. V: one factorisation serves several right-hand sides (Alg. 1 steps 4-6)."""
    rng = inputs.rng_for(80)
    p = inputs.random_recursive(700, rng)
    n, m = 6, 3
    d = inputs.problem_data(p, n, m, rng, delta="subset", delta_value=0.3, M_scale=0.2)
    s = tlqr.TreeLQR(p, n, m, FP64, has_M=True, has_delta=True)
    try:
        tlqr.tlqr_factor(s.f, {k: dev(v) for k, v in d.items()})
        for t in range(3):
            rhs = inputs.rhs_data(p, n, m, rng)
            dd = dict(d, **rhs)
            x = torch.zeros((len(p), n), dtype=torch.float64, device="cuda")
            u = torch.zeros((len(p), m), dtype=torch.float64, device="cuda")
            y = torch.zeros((len(p), n), dtype=torch.float64, device="cuda")
            tlqr.tlqr_solve_rhs(s.f, dev(rhs["q"]), dev(rhs["r"]), dev(rhs["c"]), x, u, y)
            torch.cuda.synchronize()
            out = dict(x=x.cpu().numpy(), u=u.cpu().numpy(), y=y.cpu().numpy())
            check_against_oracle(p, n, m, dd, out, fwd_tol=1e-9, eta_tol=1e-12)
    finally:
        s.close()


def test_lifted_node_controls_on_gpu():
    """Prop. 2 end to end: host lifting -> GPU edge-form solve -> projection,
    against the dense node-control KKT solution."""
    from oracle import dense
    from tests.test_boundary_cpu import node_control_instance
    rng = inputs.rng_for(81)
    p, _ = inputs.permute_labels(inputs.random_recursive(60, rng), rng)
    n, m = 4, 2
    nd = node_control_instance(rng, p, n, m, True)
    L = tlqr.tlqr_lift_node_controls(p, n, m, nd)
    data = {k: L[k] for k in ("Q", "q", "M", "R", "r", "A", "B", "c", "Delta")}
    out = gpu_solve(L["parent"], n + m, m, data, want_PK=False)
    x, v, y = tlqr.tlqr_project_lifted(len(p), n, m, L["map"], out["x"], out["u"], out["y"])
    ref = dense.dense_solve_node_control(p, n, m, nd)
    scale = max(np.abs(ref["x"]).max(), np.abs(ref["v"]).max(), np.abs(ref["y"]).max())
    for a, b in ((x, ref["x"]), (v, ref["v"]), (y, ref["y"])):
        assert np.abs(a - b).max() <= 1e-10 * scale


@pytest.mark.parametrize("with_delta", [False, True])
def test_lifted_node_controls_on_device(with_delta):
    """Prop. 2 with the data on the GPU: device lifting equals the host lifting
    entry for entry (pure copies), and device lifting -> GPU edge-form solve ->
    device projection equals the dense node-control KKT solution."""
    from oracle import dense
    from tests.test_boundary_cpu import node_control_instance
    rng = inputs.rng_for(83)
    p, _ = inputs.permute_labels(inputs.random_recursive(80, rng), rng)
    n, m = 3, 2
    nd = node_control_instance(rng, p, n, m, with_delta)
    host = tlqr.tlqr_lift_node_controls(p, n, m, nd)
    devnd = {k: (None if v is None else dev(v)) for k, v in nd.items()}
    L = tlqr.tlqr_lift_node_controls_device(p, n, m, devnd)
    np.testing.assert_array_equal(L["parent"], host["parent"])
    np.testing.assert_array_equal(L["map"], host["map"])
    for k in ("Q", "q", "M", "R", "r", "A", "B", "c", "Delta"):
        np.testing.assert_array_equal(L[k].cpu().numpy(), host[k])
    Nl, s = len(L["parent"]), n + m
    S = tlqr.TreeLQR(L["parent"], s, m, FP64, has_M=True, has_delta=True)
    try:
        x = torch.zeros((Nl, s), dtype=torch.float64, device="cuda")
        u = torch.zeros((Nl, m), dtype=torch.float64, device="cuda")
        y = torch.zeros((Nl, s), dtype=torch.float64, device="cuda")
        tlqr.tlqr_solve(S.f, {k: L[k] for k in ("Q", "q", "M", "R", "r", "A", "B", "c", "Delta")}, x, u, y)
    finally:
        S.close()
    xv, vv, yv = tlqr.tlqr_project_lifted_device(len(p), n, m, L["map"], x, u, y)
    ref = dense.dense_solve_node_control(p, n, m, nd)
    scale = max(np.abs(ref["x"]).max(), np.abs(ref["v"]).max(), np.abs(ref["y"]).max())
    for a, b in ((xv, ref["x"]), (vv, ref["v"]), (yv, ref["y"])):
        assert np.abs(a.cpu().numpy() - b).max() <= 1e-10 * scale


def test_gpu_residual_matches_oracle_residual():
    rng = inputs.rng_for(82)
    p = inputs.random_recursive(300, rng)
    n, m = 5, 3
    d = inputs.problem_data(p, n, m, rng, delta="random", delta_value=0.2, M_scale=0.3)
    x, u, y = rng.standard_normal((300, n)), rng.standard_normal((300, m)), rng.standard_normal((300, n))
    u[p < 0] = 0
    s = tlqr.TreeLQR(p, n, m, FP64, has_M=True, has_delta=True)
    try:
        st = tlqr.tlqr_kkt_residual(s.f, {k: dev(v) for k, v in d.items()}, dev(x), dev(u), dev(y))
    finally:
        s.close()
    ref = riccati.kkt_residual(p, n, m, d, x, u, y)
    assert st["abs"] == pytest.approx(ref["abs"], rel=1e-12)
    assert st["eta"] == pytest.approx(ref["eta"], rel=1e-12)


# -------------------------------------------------------------------- mixed precision

@pytest.mark.parametrize("name", ["binary", "long_trunk"])
def test_mixed_refined(name):
    w = inputs.binary_depth6() if name == "binary" else inputs.long_trunk()
    out = gpu_solve(w.parent, w.n, w.m, w.data, precision=MIXED, want_PK=False)
    assert out["info"]["eta"] <= 1e-8
    fe, eta = check_against_oracle(w.parent, w.n, w.m, w.data, out, fwd_tol=1e-6, eta_tol=1e-8)
    # the refinement's residual runs in float-float on the FP32 pipe; its eta for the returned
    # solution must agree with the oracle's FP64 eta to ~1e-14 of the residual's scale
    assert abs(out["info"]["eta"] - eta) <= 1e-13


# -------------------------------------------------------------------- errors

def test_indefinite_R_reports_not_pd():
    p = inputs.chain(20)
    d = inputs.problem_data(p, 3, 2, inputs.rng_for(83))
    d["R"][7] = -np.eye(2)
    with pytest.raises(tlqr.TLQRError) as e:
        gpu_solve(p, 3, 2, d)
    assert e.value.code == 3


def test_nan_data_is_reported():
    p = inputs.chain(20)
    d = inputs.problem_data(p, 3, 2, inputs.rng_for(84))
    d["Q"][5, 0, 0] = np.nan
    with pytest.raises(tlqr.TLQRError) as e:
        gpu_solve(p, 3, 2, d)
    assert e.value.code in (3, 4, 5)


# -------------------------------------------------------------------- graphs

@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_graph_replay_equals_direct_launches(precision):
    """The CUDA-graph launch path replays exactly the direct launch sequence:
    bitwise equal results, also after a recapture for new buffers."""
    rng = inputs.rng_for(90)
    p = inputs.random_recursive(3000, rng)
    n, m = 6, 2
    d = inputs.problem_data(p, n, m, rng, delta="subset", delta_value=1e-3)
    a = gpu_solve(p, n, m, d, precision=precision, use_graphs=False)
    s = tlqr.TreeLQR(p, n, m, precision, has_delta=True, use_graphs=True)
    try:
        outs = []
        for rep in range(3):               # capture, replay, recapture (fresh tensors)
            dd = {k: dev(v) for k, v in d.items()}
            x = torch.zeros((len(p), n), dtype=torch.float64, device="cuda")
            u = torch.zeros((len(p), m), dtype=torch.float64, device="cuda")
            y = torch.zeros((len(p), n), dtype=torch.float64, device="cuda")
            tlqr.tlqr_solve(s.f, dd, x, u, y)
            if rep == 1:
                tlqr.tlqr_solve(s.f, dd, x, u, y)
            torch.cuda.synchronize()
            outs.append((x.cpu().numpy(), u.cpu().numpy(), y.cpu().numpy()))
        prof = tlqr.tlqr_profile_read(s.f)
    finally:
        s.close()
    for o in outs:
        np.testing.assert_array_equal(o[0], a["x"])
        np.testing.assert_array_equal(o[1], a["u"])
        np.testing.assert_array_equal(o[2], a["y"])
    assert prof["compress"]["launches"] > 0 and prof["recover"]["launches"] >= 4


def test_profiler_times_kernels_inside_graphs():
    rng = inputs.rng_for(91)
    p = inputs.random_recursive(2000, rng)
    d = inputs.problem_data(p, 4, 2, rng)
    s = tlqr.TreeLQR(p, 4, 2, FP64, use_graphs=True)
    try:
        dd = {k: dev(v) for k, v in d.items()}
        x = torch.zeros((len(p), 4), dtype=torch.float64, device="cuda")
        u = torch.zeros((len(p), 2), dtype=torch.float64, device="cuda")
        y = torch.zeros((len(p), 4), dtype=torch.float64, device="cuda")
        tlqr.tlqr_profile_mask(s.f, ["compress", "expand"])
        for _ in range(3):
            tlqr.tlqr_solve(s.f, dd, x, u, y)
        prof = tlqr.tlqr_profile_read(s.f)
    finally:
        s.close()
    assert prof["compress"]["timed"] == prof["compress"]["launches"] > 0
    assert prof["compress"]["ms"] > 0 and prof["expand"]["ms"] > 0
    assert prof["local_factor"]["timed"] == 0 and prof["local_factor"]["launches"] > 0


# -------------------------------------------------------------------- kernel families

@pytest.mark.parametrize("n,m", [(4, 2), (6, 2), (8, 3), (12, 4), (16, 4)])
@pytest.mark.parametrize("generic", [False, True])
def test_fixed_and_runtime_dimension_kernels(n, m, generic):
    """The compile-time-n kernels (n = 4, 6, 8, 12, 16) and the run-time-n kernels
    both match the oracle, in FP64 and in refined mixed precision."""
    rng = inputs.rng_for(600 + n)
    p, _ = inputs.permute_labels(inputs.random_recursive(1500, rng), rng)
    d = inputs.problem_data(p, n, m, rng, delta="subset", delta_value=0.05, delta_fraction=0.3, M_scale=0.2)
    out = gpu_solve(p, n, m, d, generic_kernels=generic)
    check_against_oracle(p, n, m, d, out, fwd_tol=1e-8, eta_tol=1e-10, pk_tol=1e-8)
    outm = gpu_solve(p, n, m, d, precision=MIXED, want_PK=False, generic_kernels=generic)
    assert outm["info"]["eta"] <= 1e-8
    _, eta = check_against_oracle(p, n, m, d, outm, fwd_tol=1e-6, eta_tol=1e-8)
    # the refinement's own float-float residual (row- or node-organised) gives the oracle's eta
    assert abs(outm["info"]["eta"] - eta) <= 1e-13


# -------------------------------------------------------------------- batches (forests)

@pytest.mark.parametrize("n,m", [(4, 2), (12, 4), (16, 4), (5, 3)])
def test_forest_batch_equals_trees_alone(n, m):
    """A batch of independent trees solved as one forest: in FP64 every tree's
    x, u, y, P, K are bitwise those of the tree solved alone (same schedule, same
    per-operation arithmetic); all match the oracle.  In mixed precision each
    tree meets eta <= 1e-8 (the batch may take an extra refinement step)."""
    rng = inputs.rng_for(700 + n)
    trees = [inputs.random_recursive(int(rng.integers(1, 900)), rng) for _ in range(9)] + [inputs.chain(700)]
    datas = [inputs.problem_data(p, n, m, rng, delta="subset", delta_value=0.05, delta_fraction=0.3) for p in trees]
    par, offs = inputs.forest(trees)
    data = inputs.concat_data(datas)
    batch = gpu_solve(par, n, m, data, forest=True)
    check_against_oracle(par, n, m, data, batch, fwd_tol=1e-8, eta_tol=1e-10, pk_tol=1e-8)
    for t, p in enumerate(trees):
        alone = gpu_solve(p, n, m, datas[t])
        sl = slice(offs[t], offs[t] + len(p))
        for k in ("x", "u", "y", "P", "K"):
            np.testing.assert_array_equal(batch[k][sl], alone[k])
    mixed = gpu_solve(par, n, m, data, precision=MIXED, want_PK=False, forest=True)
    assert len(mixed["tree_eta"]) == len(trees)
    for t, p in enumerate(trees):
        sl = slice(offs[t], offs[t] + len(p))
        sub = {k: mixed[k][sl] for k in ("x", "u", "y")}
        res = riccati.kkt_residual(p, n, m, datas[t], sub["x"], sub["u"], sub["y"])
        assert res["eta"] <= 1e-8
        # the refinement's own per-tree eta (float-float residual, FP32 row sums of |K|)
        assert abs(mixed["tree_eta"][t] - res["eta"]) <= 1e-3 * res["eta"] + 1e-15
    assert mixed["info"]["eta"] == mixed["tree_eta"].max()


@pytest.mark.parametrize("permute", [False, True])
def test_forest_residual_is_per_tree(permute):
    """tlqr_kkt_residual on a forest: per-tree ||K z - b|| and eta equal the
    oracle's residual of each tree on its own (FP64 kernel), also when the
    forest's labels are permuted so that trees interleave in memory."""
    n, m = 5, 2
    rng = inputs.rng_for(720 + permute)
    trees = [inputs.random_recursive(int(rng.integers(1, 400)), rng) for _ in range(12)]
    datas = [inputs.problem_data(p, n, m, rng, delta="subset", delta_value=0.05) for p in trees]
    par, offs = inputs.forest(trees)
    data = inputs.concat_data(datas)
    # a perturbed solution so that the residual is well above rounding
    x = rng.standard_normal((len(par), n)); u = rng.standard_normal((len(par), m)); y = rng.standard_normal((len(par), n))
    owner = np.concatenate([np.full(len(p), t) for t, p in enumerate(trees)])
    if permute:
        par2, perm = inputs.permute_labels(par, rng)
        data = inputs.permute_data(data, perm)
        inv = np.argsort(perm)
        x, u, y, owner = x[inv], u[inv], y[inv], owner[inv]
        par = par2
    s = tlqr.TreeLQR(par, n, m, FP64, has_delta=True, forest=True)
    try:
        stats = tlqr.tlqr_kkt_residual(s.f, {k: dev(v) for k, v in data.items()}, dev(x), dev(u), dev(y))
        absr, eta = tlqr.tlqr_tree_residuals(s.f, len(trees))
    finally:
        s.close()
    roots = np.nonzero(np.asarray(par) < 0)[0]          # tree ordinals follow increasing root label
    for t, rt in enumerate(roots):
        sel = np.nonzero(owner == owner[rt])[0]
        pos = np.full(len(par), -1)
        pos[sel] = np.arange(len(sel))
        sub = np.where(par[sel] < 0, -1, pos[par[sel]]).astype(np.int32)
        d_t = {k: (None if v is None else v[sel]) for k, v in data.items()}
        ref = riccati.kkt_residual(sub, n, m, d_t, x[sel], u[sel], y[sel])
        assert abs(absr[t] - ref["abs"]) <= 1e-12 * ref["abs"]
        assert abs(eta[t] - ref["eta"]) <= 1e-12 * ref["eta"]
    assert stats["eta"] == eta.max()


def test_speculative_refinement_equals_checked_refinement():
    """A MIXED factor whose last solve needed a refinement step enqueues the
    next solve's first step without waiting (residual, device gate,
    correction, residual).  The result must not depend on it: solving B after
    A on one factor object equals solving B on a fresh one, bitwise -- for a B
    that needs a step, and for one whose first residual already meets the
    tolerance (the gate zeroes the correction's right-hand side)."""
    rng = inputs.rng_for(96)
    p = inputs.long_trunk_tree(rng, trunk=200, total=2000)
    n, m = 12, 4
    A = inputs.problem_data(p, n, m, rng)
    B = inputs.problem_data(p, n, m, rng)
    Z = dict(B)
    Z.update(q=np.zeros_like(B["q"]), r=np.zeros_like(B["r"]), c=np.zeros_like(B["c"]))
    N = len(p)

    def run(seq):
        s = tlqr.TreeLQR(p, n, m, MIXED)
        outs = []
        try:
            for data in seq:
                x = torch.zeros((N, n), dtype=torch.float64, device="cuda")
                u = torch.zeros((N, m), dtype=torch.float64, device="cuda")
                y = torch.zeros((N, n), dtype=torch.float64, device="cuda")
                tlqr.tlqr_solve(s.f, {k: dev(v) for k, v in data.items()}, x, u, y)
                torch.cuda.synchronize()
                outs.append((x.cpu().numpy(), u.cpu().numpy(), y.cpu().numpy(), tlqr.tlqr_last_info(s.f)))
        finally:
            s.close()
        return outs

    seq = run([A, B, Z, B])
    assert seq[0][3]["refine_steps"] >= 1                  # A needs a step: B's solve speculates
    alone_B = run([B])[0]
    alone_Z = run([Z])[0]
    for got, ref in ((seq[1], alone_B), (seq[3], alone_B), (seq[2], alone_Z)):
        for a, b in zip(got[:3], ref[:3]):
            np.testing.assert_array_equal(a, b)
        assert got[3]["refine_steps"] == ref[3]["refine_steps"]
    assert seq[2][3]["refine_steps"] == 0 and np.all(seq[2][0] == 0.0)
