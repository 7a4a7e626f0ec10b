"""GPU test of the serving loop: requests that run concurrently (overlapping
on the device, admitted while others are in flight, factors reused across
requests) give exactly the results they give alone."""
import numpy as np
import pytest

from paper_2608_01332_b300 import serve, tlqr
from tests.conftest import ROOT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import sys  # noqa: E402
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("precision", [tlqr.TLQR_PREC_MIXED, tlqr.TLQR_PREC_FP64])
@pytest.mark.parametrize("mode", ["perturb", "ipm"])
def test_alone_equals_in_the_mix(precision, mode):
    """Every request of a concurrent mix equals the same request run alone,
    bitwise: perturbed-data re-solves, and interior-point requests (whose
    Newton systems the driver forms on the device)."""
    dev = torch.device("cuda", 0)
    traffic = bench.ServeTraffic(dev, topologies=5, iterations=4 if mode == "perturb" else 12, lo=300, hi=6000,
                                 ipm=mode == "ipm")
    topo = [k % 5 for k in range(14)]
    srv = serve.Server(slots=4)
    mix = [srv.submit(traffic.request(k, precision, t=topo[k])) for k in range(14)]
    srv.drain()
    assert all(r.error is None for r in mix), [repr(r.error) for r in mix if r.error]
    assert srv.stats["factor_reuse"] > 0 and srv.stats["plan_hits"] > 0
    srv.close()
    for k, r in enumerate(mix):
        alone_srv = serve.Server(slots=1)
        a = alone_srv.submit(traffic.request(k, precision, t=topo[k]))
        alone_srv.drain()
        alone_srv.close()
        assert a.error is None
        for name in ("x", "u", "y"):
            assert torch.equal(getattr(r, name), getattr(a, name)), (k, name)
        if mode == "ipm":
            assert r.infos == a.infos
        elif precision == tlqr.TLQR_PREC_MIXED:
            assert max(i["eta"] for i in r.infos) <= 1e-8
            assert [i["refine_steps"] for i in r.infos] == [i["refine_steps"] for i in a.infos]
