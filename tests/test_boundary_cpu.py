"""CPU tests of the C ABI: the library loads and exports every declared symbol,
the host planner equals the literal schedule oracle, and the host lifting of
Prop. 2 is exact (checked through the FP64 oracle, no GPU needed)."""
import re

import numpy as np
import pytest

from oracle import dense, plan as oplan, riccati
from paper_2608_01332_b300 import inputs, tlqr
from tests.conftest import ROOT

OPCODE = {"-": tlqr.TLQR_OP_ROOT, "R": tlqr.TLQR_OP_RAKE, "C": tlqr.TLQR_OP_COMPRESS}


def declared_functions():
    src = open(f"{ROOT}/include/tlqr.h").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(tlqr_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 18
    L = tlqr.lib()
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(tlqr.EXPORTS)


def test_status_strings():
    for code in range(11):
        assert tlqr.tlqr_status_string(code)


def _trees():
    rng = inputs.rng_for(31)
    out = [("single", np.array([-1], dtype=np.int32)), ("pair", inputs.chain(2)),
           ("chain", inputs.chain(257)), ("star", inputs.star(300)), ("balanced", inputs.balanced(255)),
           ("comb", inputs.comb(301)), ("tight", inputs.tightness_tree(32)),
           ("longtrunk", inputs.long_trunk_tree(rng, trunk=300, total=3000)),
           ("driving", inputs.driving_tree(rng, 2000))]
    for t in range(40):
        N = int(rng.integers(2, 500))
        p = inputs.random_recursive(N, rng)
        p, _ = inputs.permute_labels(p, rng)
        out.append((f"rr{t}", p))
    return out


@pytest.mark.parametrize("tree", _trees(), ids=lambda t: t[0])
def test_planner_equals_schedule_oracle(tree):
    """Bit-exact: every node's (round, operation) and the plan statistics."""
    _, parent = tree
    N = len(parent)
    h = tlqr.tlqr_plan_create(parent)
    try:
        rnd, op = tlqr.tlqr_plan_schedule(h, N)
        ops = oplan.node_ops(parent)
        assert [int(r) for r in rnd] == [ops[i][0] for i in range(N)]
        assert [int(o) for o in op] == [OPCODE[ops[i][1]] for i in range(N)]
        st = tlqr.tlqr_plan_stats(h)
        assert st["n_rake"] + st["n_compress"] == N - 1
        if N > 1:
            lv = oplan.dependency_levels(parent)
            for k in ("levels", "rounds", "n_rake", "n_compress", "n_combine", "n_absorb"):
                assert st[k] == lv[k], k
    finally:
        tlqr.tlqr_plan_destroy(h)


def test_planner_star_column_of_table1():
    got = []
    for N in (16, 64, 256, 1024, 4096):
        h = tlqr.tlqr_plan_create(inputs.star(N))
        got.append(tlqr.tlqr_plan_stats(h)["levels"])
        tlqr.tlqr_plan_destroy(h)
    assert got == [6, 8, 10, 12, 14]


@pytest.mark.parametrize("bad", [[0, 0], [-1, -1, 0], [-1, 2, 1], [-1, 5], [-1, 1], []])
def test_planner_rejects_non_trees(bad):
    with pytest.raises(tlqr.TLQRError) as e:
        tlqr.tlqr_plan_create(np.array(bad, dtype=np.int32))
    assert e.value.code in (1, 2)


def node_control_instance(rng, parent, n, m, delta=True):
    """Random node-control data satisfying the sufficient conditions of Prop. 2."""
    N = len(parent)
    Q = np.zeros((N, n, n)); Mv = np.zeros((N, n, m)); Rv = np.zeros((N, m, m))
    for i in range(N):
        G = rng.standard_normal((n, n)); H = rng.standard_normal((m, m))
        Rv[i] = np.eye(m) + H @ H.T
        Mv[i] = 0.3 * rng.standard_normal((n, m))
        Q[i] = G @ G.T + 0.1 * np.eye(n) + Mv[i] @ Mv[i].T       # R >= I keeps Q - M R^-1 M' >= 0
    Av = 0.95 * inputs.haar_orthogonal(rng, N, n)
    Bv = rng.standard_normal((N, n, m)) / np.sqrt(n)
    D = None
    if delta:
        Dg = rng.standard_normal((N, n, n))
        D = 0.2 * Dg @ Dg.transpose(0, 2, 1) / n
    return dict(Q=Q, q=rng.standard_normal((N, n)), Mv=Mv, Rv=Rv, rv=rng.standard_normal((N, m)),
                Av=Av, Bv=Bv, c=np.sqrt(0.1) * rng.standard_normal((N, n)), Delta=D)


@pytest.mark.parametrize("seed,delta", [(1, False), (2, True), (3, True)])
def test_lifting_is_exact_through_the_oracle(seed, delta):
    """Prop. 2: lift (library, host) -> edge-form oracle solve -> project (library)
    equals the dense solution of the node-control KKT system; dummy controls are
    zero; the lifted tree has |V| + |V \\ leaves| nodes."""
    rng = inputs.rng_for(100 + seed)
    p = inputs.random_recursive(int(rng.integers(5, 25)), rng)
    p, _ = inputs.permute_labels(p, rng)
    n, m = 3, 2
    nd = node_control_instance(rng, p, n, m, delta)
    L = tlqr.tlqr_lift_node_controls(p, n, m, nd)
    n_nonterm = len(set(int(v) for v in p if v >= 0))
    assert len(L["parent"]) == len(p) + n_nonterm
    data = dict(Q=L["Q"], q=L["q"], M=L["M"], R=L["R"], r=L["r"], A=L["A"], B=L["B"], c=L["c"],
                Delta=L["Delta"])
    sol = riccati.tree_riccati(L["parent"], n + m, m, data)
    x, v, y = tlqr.tlqr_project_lifted(len(p), n, m, L["map"], sol["x"], sol["u"], sol["y"])
    ref = dense.dense_solve_node_control(p, n, m, nd)
    scale = max(np.abs(ref["x"]).max(), np.abs(ref["v"]).max(), np.abs(ref["y"]).max())
    for a, b in ((x, ref["x"]), (v, ref["v"]), (y, ref["y"])):
        assert np.abs(a - b).max() <= 1e-11 * scale
    # dummy controls of the uncertainty edges (children that are predecision nodes) are zero
    dummies = [j for j in range(len(p)) if p[j] >= 0]
    assert np.abs(sol["u"][dummies]).max() <= 1e-12 * scale


def test_forest_planner_equals_schedule_oracle():
    rng = inputs.rng_for(43)
    trees = [inputs.random_recursive(int(rng.integers(1, 300)), rng) for _ in range(8)]
    par, _ = inputs.forest(trees)
    par, _ = inputs.permute_labels(par, rng)      # relabelling handles several roots
    h = tlqr.tlqr_plan_create_forest(par)
    try:
        rnd, op = tlqr.tlqr_plan_schedule(h, len(par))
        ops = oplan.node_ops(par)
        assert [int(r) for r in rnd] == [ops[i][0] for i in range(len(par))]
        assert [int(o) for o in op] == [OPCODE[ops[i][1]] for i in range(len(par))]
        st = tlqr.tlqr_plan_stats(h)
        assert st["n_trees"] == len(trees)
        assert st["n_rake"] + st["n_compress"] == len(par) - len(trees)
    finally:
        tlqr.tlqr_plan_destroy(h)
    with pytest.raises(tlqr.TLQRError):
        tlqr.tlqr_plan_create(par)          # the single-tree entry point refuses several roots


def test_noalloc_residual_refuses_host_arrays():
    """The allocation-free residual takes device arrays only: host arrays are
    refused with TLQR_ERR_ARG by the binding, and by the C entry point itself
    when a caller flags host pointers as device memory (it asks CUDA what each
    pointer is before any launch)."""
    import ctypes
    p = inputs.chain(16)
    n, m = 3, 2
    d = inputs.problem_data(p, n, m, inputs.rng_for(5))
    x, u, y = np.zeros((16, n)), np.zeros((16, m)), np.zeros((16, n))
    plan = tlqr.tlqr_plan_create(p)
    try:
        with pytest.raises(tlqr.TLQRError) as e:
            tlqr.tlqr_kkt_residual_noalloc(plan, n, m, d, x, u, y)
        assert e.value.code == tlqr.TLQR_ERR_ARG
        prob = tlqr.make_problem(d)
        prob.mem = tlqr.TLQR_MEM_DEVICE           # a false claim: these are host arrays
        stats = np.zeros(2)
        rc = tlqr.lib().tlqr_kkt_residual_noalloc(plan, n, m, ctypes.byref(prob), tlqr._ptr(x), tlqr._ptr(u),
                                                  tlqr._ptr(y), tlqr._ptr(stats), None)
        assert rc == tlqr.TLQR_ERR_ARG
    finally:
        tlqr.tlqr_plan_destroy(plan)


def test_factor_options_are_validated_before_any_device_work():
    """Out-of-range options are refused with TLQR_ERR_ARG before the call
    touches the device (so this holds on a host without a GPU)."""
    import ctypes
    plan = tlqr.tlqr_plan_create(inputs.chain(8))
    try:
        for kw in (dict(residual=3), dict(residual=-1), dict(precision=7)):
            base = dict(n=4, m=2, precision=tlqr.TLQR_PREC_MIXED)
            base.update(kw)
            o = tlqr.make_options(base.pop("n"), base.pop("m"), base.pop("precision"), **base)
            h = ctypes.c_void_p()
            assert tlqr.lib().tlqr_factor_create(plan, ctypes.byref(o), ctypes.byref(h)) == tlqr.TLQR_ERR_ARG
            assert not h.value
        o = tlqr.make_options(tlqr.TLQR_MAX_DIM + 1, 2, tlqr.TLQR_PREC_FP64)
        h = ctypes.c_void_p()
        assert tlqr.lib().tlqr_factor_create(plan, ctypes.byref(o), ctypes.byref(h)) == tlqr.TLQR_ERR_ARG
    finally:
        tlqr.tlqr_plan_destroy(plan)


def test_update_solve_refuses_bad_arguments_without_a_device():
    """tlqr_update_solve checks its arguments first: no factor, or a memory
    kind that is neither host nor device, is TLQR_ERR_ARG."""
    import ctypes
    x, u, y = np.zeros((4, 3)), np.zeros((4, 2)), np.zeros((4, 3))
    sol = tlqr.make_solution(x, u, y, None, None)
    rc = tlqr.lib().tlqr_update_solve(None, tlqr.TLQR_MEM_HOST, None, None, None, None, None, ctypes.byref(sol), None)
    assert rc == tlqr.TLQR_ERR_ARG
