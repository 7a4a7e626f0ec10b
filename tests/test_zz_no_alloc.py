"""The allocation-free residual entry point against the regular one.

tlqr_kkt_residual_noalloc serves callers that may not allocate device memory
while running (a control loop with a hard deadline, or memory owned by another
framework's allocator).  It must report the same residual and backward error as
tlqr_kkt_residual, call after call, although every call reuses one fixed
scratch array; for a batch of trees both report the largest per-tree values;
trees too large for that array are refused, and so are host arrays.

This file is named so that pytest collects it after every other test file.
"""
import numpy as np
import pytest

from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _perturbed_solution(s, dd, N, n, m, roots):
    x = torch.zeros((N, n), dtype=torch.float64, device="cuda")
    u = torch.zeros((N, m), dtype=torch.float64, device="cuda")
    y = torch.zeros((N, n), dtype=torch.float64, device="cuda")
    tlqr.tlqr_solve(s.f, dd, x, u, y)
    # a perturbed point, so that the residual is far from zero
    g = torch.Generator(device="cuda")
    g.manual_seed(17)
    x += 1e-3 * torch.randn(x.shape, generator=g, dtype=x.dtype, device="cuda")
    u += 1e-3 * torch.randn(u.shape, generator=g, dtype=u.dtype, device="cuda")
    u[torch.as_tensor(roots, device="cuda")] = 0.0
    torch.cuda.synchronize()
    return x, u, y


def _check_twice(s, dd, n, m, x, u, y, stream=None):
    ref = tlqr.tlqr_kkt_residual(s.f, dd, x, u, y)
    free0 = None
    for k in range(3):
        got = tlqr.tlqr_kkt_residual_noalloc(s.plan, n, m, dd, x, u, y, stream=stream)
        assert got["abs"] == pytest.approx(ref["abs"], rel=1e-12)
        assert got["eta"] == pytest.approx(ref["eta"], rel=1e-12)
        assert got["abs"] > 1e-6
        if k == 0:
            # after the first call (which may load the library's code onto the device),
            # later calls must not change the device's free memory
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_residual_matches_regular_entry_point_twice():
    rng = inputs.rng_for(4242)
    p, _ = inputs.permute_labels(inputs.random_recursive(3000, rng), rng)
    n, m = 5, 3
    d = inputs.problem_data(p, n, m, rng, M_scale=0.3, delta="subset", delta_value=0.1)
    dd = {k: _dev(v) for k, v in d.items()}
    N = len(p)
    s = tlqr.TreeLQR(p, n, m, tlqr.TLQR_PREC_FP64, has_M=True, has_delta=True)
    try:
        x, u, y = _perturbed_solution(s, dd, N, n, m, np.nonzero(p < 0)[0])
        _check_twice(s, dd, n, m, x, u, y)
    finally:
        s.close()


def test_noalloc_residual_without_M_and_Delta_on_a_side_stream():
    rng = inputs.rng_for(4243)
    p = inputs.long_trunk_tree(rng, trunk=256, total=4000)
    n, m = 12, 4
    d = inputs.problem_data(p, n, m, rng)
    assert d["M"] is None and d["Delta"] is None
    dd = {k: _dev(v) for k, v in d.items()}
    s = tlqr.TreeLQR(p, n, m, tlqr.TLQR_PREC_FP64)
    try:
        x, u, y = _perturbed_solution(s, dd, len(p), n, m, np.nonzero(p < 0)[0])
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        _check_twice(s, dd, n, m, x, u, y, stream=side)
    finally:
        s.close()


def test_noalloc_residual_forest_reports_the_largest_per_tree_eta():
    rng = inputs.rng_for(4244)
    trees = [inputs.random_recursive(int(k), rng) for k in (40, 700, 3, 1500, 90)]
    p, offs = inputs.forest(trees)
    n, m = 4, 2
    d = inputs.problem_data(p, n, m, rng, M_scale=0.3)
    dd = {k: _dev(v) for k, v in d.items()}
    s = tlqr.TreeLQR(p, n, m, tlqr.TLQR_PREC_FP64, has_M=True, forest=True)
    try:
        x, u, y = _perturbed_solution(s, dd, len(p), n, m, np.nonzero(p < 0)[0])
        # move one tree's point far off its solution so that the trees' etas differ widely
        b, e = int(offs[3]), int(offs[3]) + len(trees[3])
        x[b:e] += 0.5
        torch.cuda.synchronize()
        _check_twice(s, dd, n, m, x, u, y)
        _, per_tree = tlqr.tlqr_tree_residuals(s.f, len(trees))
        got = tlqr.tlqr_kkt_residual_noalloc(s.plan, n, m, dd, x, u, y)
        assert got["eta"] == pytest.approx(per_tree.max(), rel=1e-12)
        assert per_tree.min() < 0.5 * per_tree.max()
    finally:
        s.close()


def test_noalloc_residual_just_below_its_scratch_limit():
    n, m = 12, 4
    N = 70000                     # about 16.5 MB of scratch: just inside the 16 MiB array
    p = inputs.chain(N)
    d = inputs.problem_data_device(p, n, m, 99, "cuda")
    s = tlqr.TreeLQR(p, n, m, tlqr.TLQR_PREC_FP64)
    try:
        x, u, y = _perturbed_solution(s, d, N, n, m, [0])
        _check_twice(s, d, n, m, x, u, y)
    finally:
        s.close()


def test_noalloc_residual_refuses_trees_beyond_its_scratch():
    n, m = 12, 4
    N = 80000                     # needs about 19 MB of scratch, more than the 16 MiB array
    p = inputs.chain(N)
    plan = tlqr.tlqr_plan_create(p)
    try:
        z = torch.zeros(1, dtype=torch.float64, device="cuda")
        dd = dict(Q=z, q=z, M=None, R=z, r=z, A=z, B=z, c=z, Delta=None)
        with pytest.raises(tlqr.TLQRError) as e:
            tlqr.tlqr_kkt_residual_noalloc(plan, n, m, dd, z, z, z)
        assert e.value.code == 1
    finally:
        tlqr.tlqr_plan_destroy(plan)
