"""The allocation-free residual entry point against the regular one.

tlqr_kkt_residual_noalloc serves callers that may not allocate device memory
while running (a control loop with a hard deadline, or memory owned by another
framework's allocator).  It must report the same residual and backward error as
tlqr_kkt_residual, call after call, although every call reuses one fixed
scratch array; trees too large for that array are refused.

This file is named so that pytest collects it after every other test file.
"""
import numpy as np
import pytest

from paper_2608_01332_b300 import inputs, tlqr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_residual_matches_regular_entry_point_twice():
    rng = inputs.rng_for(4242)
    p, _ = inputs.permute_labels(inputs.random_recursive(3000, rng), rng)
    n, m = 5, 3
    d = inputs.problem_data(p, n, m, rng, M_scale=0.3, delta="subset", delta_value=0.1)
    dd = {k: _dev(v) for k, v in d.items()}
    N = len(p)
    s = tlqr.TreeLQR(p, n, m, tlqr.TLQR_PREC_FP64, has_M=True, has_delta=True)
    try:
        x = torch.zeros((N, n), dtype=torch.float64, device="cuda")
        u = torch.zeros((N, m), dtype=torch.float64, device="cuda")
        y = torch.zeros((N, n), dtype=torch.float64, device="cuda")
        tlqr.tlqr_solve(s.f, dd, x, u, y)
        # a perturbed point, so that the residual is far from zero
        x += 1e-3 * torch.randn_like(x)
        u[:, :] += 1e-3 * torch.randn_like(u)
        u[int(np.nonzero(p < 0)[0][0])] = 0.0
        torch.cuda.synchronize()
        ref = tlqr.tlqr_kkt_residual(s.f, dd, x, u, y)
        for _ in range(2):
            got = tlqr.tlqr_kkt_residual_noalloc(s.plan, n, m, dd, x, u, y)
            assert got["abs"] == pytest.approx(ref["abs"], rel=1e-12)
            assert got["eta"] == pytest.approx(ref["eta"], rel=1e-12)
            assert got["abs"] > 1e-6
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
