"""CPU tests of the serving loop's scheduling (admission by device memory,
FIFO order, plan cache, factor reuse, eviction only while idle), with a fake
backend standing in for the C ABI."""
import threading
import time

import numpy as np
import pytest

from paper_2608_01332_b300 import inputs, serve


class FakeBackend:
    WORDS_PER_NODE = 1000

    def __init__(self):
        self.lock = threading.Lock()
        self.live = 0
        self.max_live = 0
        self.plans_made = 0
        self.factors_made = 0
        self.running = 0
        self.freed_while_running = 0
        self.server = None

    def plan(self, parent):
        with self.lock:
            self.plans_made += 1
        return ("plan", len(parent))

    def destroy_plan(self, plan):
        pass

    def options(self, req):
        return (req.n, req.m, req.precision)

    def workspace_bytes(self, plan, opts):
        return self.WORDS_PER_NODE * plan[1]

    def create_factor(self, plan, opts):
        with self.lock:
            self.factors_made += 1
            self.live += self.WORDS_PER_NODE * plan[1]
            self.max_live = max(self.max_live, self.live)
        return {"bytes": self.WORDS_PER_NODE * plan[1]}

    def destroy_factor(self, f):
        with self.lock:
            self.live -= f["bytes"]
            if self.server is not None and self.server.running:
                self.freed_while_running += 1

    def stream(self):
        return None

    def outputs(self, req):
        return np.zeros((req.N, req.n)), np.zeros((req.N, req.m)), np.zeros((req.N, req.n))

    def solve(self, f, data, x, u, y, stream):
        time.sleep(0.002)
        x[:] = data
        return {"refine_steps": 0}

    def synchronize(self, stream):
        pass


def make_req(parent, tag, iters=3):
    return serve.Request(parent=parent, n=2, m=1, iterations=iters, data=lambda it, s, t=tag: float(t * 100 + it),
                         tag=tag)


def test_admission_fifo_and_budget():
    rng = inputs.rng_for(11)
    be = FakeBackend()
    trees = [inputs.random_recursive(int(rng.integers(50, 400)), rng) for _ in range(6)]
    budget = 2200 * 1000 + 10 ** 6
    srv = serve.Server(slots=3, memory_budget=budget, backend=be)
    be.server = srv
    reqs = [srv.submit(make_req(trees[k % 6], k)) for k in range(30)]
    srv.drain()
    srv.close()
    assert all(r.error is None for r in reqs)
    adm = [r.admitted for r in reqs]
    assert adm == sorted(adm)                       # FIFO admission
    assert srv.peak <= budget and be.max_live <= budget
    assert be.plans_made == 6                       # one plan per distinct topology
    assert srv.stats["plan_misses"] == 6 and srv.stats["plan_hits"] == 24
    assert srv.stats["factor_reuse"] + srv.stats["factor_new"] == 30
    assert be.freed_while_running == 0              # evictions only while no slot runs
    for r in reqs:
        assert r.x[0, 0] == r.tag * 100 + r.iterations - 1 and len(r.infos) == r.iterations


def test_factor_reuse_and_eviction():
    be = FakeBackend()
    a, b = inputs.chain(1000), inputs.star(1000)
    srv = serve.Server(slots=1, memory_budget=2 * 10 ** 6, backend=be)
    be.server = srv
    r1 = srv.submit(make_req(a, 1))
    r1.done.wait()
    r2 = srv.submit(make_req(a, 2))                 # same topology: the idle factor is reused
    r2.done.wait()
    assert r2.reused_factor and be.factors_made == 1
    r3 = srv.submit(make_req(b, 3))                 # does not fit beside the idle factor: evict it
    r3.done.wait()
    srv.close()
    assert r3.error is None and srv.stats["evictions"] == 1 and be.factors_made == 2
    assert be.freed_while_running == 0 and be.live == 0


def test_request_larger_than_budget_fails_alone():
    be = FakeBackend()
    srv = serve.Server(slots=2, memory_budget=10 ** 6, backend=be)
    big = srv.submit(make_req(inputs.chain(5000), 1))
    small = srv.submit(make_req(inputs.chain(50), 2))
    srv.drain()
    srv.close()
    assert isinstance(big.error, MemoryError) and small.error is None


def test_bad_topology_fails_the_request_only():
    be = FakeBackend()

    def bad_plan(parent):
        if (np.asarray(parent) < 0).sum() != 1:
            raise ValueError("not a tree")
        return ("plan", len(parent))
    be.plan = bad_plan
    srv = serve.Server(slots=2, memory_budget=10 ** 9, backend=be)
    bad = srv.submit(make_req(np.array([-1, -1], dtype=np.int32), 1))
    good = srv.submit(make_req(inputs.chain(10), 2))
    srv.drain()
    srv.close()
    assert isinstance(bad.error, ValueError) and good.error is None


def test_latency_summary():
    reqs = []
    for k in range(10):
        r = serve.Request(parent=inputs.chain(3), n=1, m=1, iterations=1, data=None)
        r.arrival, r.admitted, r.finished = 0.0, 0.001 * k, 0.01 * (k + 1)
        reqs.append(r)
    s = serve.latency_summary(reqs)
    assert s["completed"] == 10 and s["p50_ms"] == pytest.approx(55.0) and s["p99_ms"] > 99.0
