"""Serving loop: continuous batching of tree-LQR solves on one GPU.

A request is one controller's work on one scenario-tree topology: a short
sequence of solves with fresh problem data (the Newton systems of an
interior-point method, or successive receding-horizon re-solves), each released
only after the previous one has finished (Sec. V: the factorisation is redone
for every new data set; the topology and therefore the plan stay fixed).

The server runs `slots` requests at a time.  Every slot owns a host thread and
a CUDA stream; its request's solves are issued back to back on that stream, so
the kernels of all admitted requests overlap on the device, and a request that
arrives while others are running is admitted as soon as a slot is free and its
device memory fits the budget (continuous batching: admission at request
granularity, no waiting for a batch to drain).

  * Plans are cached per topology (keyed by the parent array's bytes): the
    host planner runs once per distinct tree.
  * Factor objects (the device workspace of one solve, one allocation each)
    stay resident for the whole request and are kept in an idle pool
    afterwards; a later request on the same topology and dimensions reuses
    them without allocating.
  * Admission by device memory: a request needs its factor's workspace
    (tlqr_factor_workspace_bytes) unless an idle one can be reused, plus its
    solution and problem buffers.  Idle factors are evicted (least recently
    used) only while no slot is running, so no device memory is freed while
    another thread may be capturing a CUDA graph.
  * Each request's arithmetic is exactly that of the same solve run alone
    (same kernels, same launch shapes, deterministic reductions): results do
    not depend on what else is in flight.

The device-side work goes through the C ABI only (`tlqr.py`); the backend
object is replaceable so that the scheduling logic can be tested on a CPU.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field
from typing import Callable

import numpy as np

from . import tlqr


def topology_key(parent) -> bytes:
    return np.ascontiguousarray(parent, dtype=np.int32).tobytes()


def problem_bytes(N: int, n: int, m: int, has_delta: bool) -> int:
    """FP64 bytes of one problem data set (Q, q, R, r, A, B, c, Delta)."""
    per = n * n + n + m * m + m + n * n + n * m + n + (n * n if has_delta else 0)
    return 8 * N * per


def ipm_bytes(N: int, n: int, m: int) -> int:
    """Device bytes of an interior-point request beyond its problem and solution:
    bounds and multipliers ([N][m] each) and the driver's workspace (Newton
    system R~, r~, the Newton point and the step directions)."""
    return 8 * N * (4 * m + m * m + 5 * m + 2 * n) + N


def solution_bytes(N: int, n: int, m: int) -> int:
    return 8 * N * (2 * n + m)


@dataclass
class Request:
    """parent: topology; data(it, stream) -> problem dict of device tensors
    for solve `it` (0 <= it < iterations), created on `stream`.

    With bounds(stream) -> (u_lo, u_hi) set, the request is one box-constrained
    problem solved by the interior-point driver (tlqr_ipm_box) with a budget of
    `iterations` Newton solves; data(0, stream) gives its data and each Newton
    system is formed on the device by the driver itself."""
    parent: np.ndarray
    n: int
    m: int
    iterations: int
    data: Callable
    precision: int = tlqr.TLQR_PREC_MIXED
    has_delta: bool = False
    tag: object = None
    bounds: Callable | None = None
    # filled by the server
    arrival: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0
    infos: list = field(default_factory=list)
    x: object = None
    u: object = None
    y: object = None
    error: BaseException | None = None
    reused_factor: bool = False
    done: threading.Event = field(default_factory=threading.Event)
    _prep: object = None

    @property
    def N(self) -> int:
        return len(self.parent)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class TlqrBackend:
    """The GPU path: C-ABI plans and factors, torch for buffers and streams."""

    def __init__(self, device=None, **option_overrides):
        import torch
        self.torch = torch
        self.option_overrides = option_overrides    # extra tlqr options for every factor (make_options keywords)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)

    def plan(self, parent):
        return tlqr.tlqr_plan_create(np.ascontiguousarray(parent, dtype=np.int32))

    def destroy_plan(self, plan):
        tlqr.tlqr_plan_destroy(plan)

    def options(self, req: Request):
        return tlqr.make_options(req.n, req.m, req.precision, has_delta=req.has_delta, **self.option_overrides)

    def workspace_bytes(self, plan, opts) -> int:
        return tlqr.tlqr_factor_workspace_bytes(plan, opts)

    def create_factor(self, plan, opts):
        self.torch.cuda.set_device(self.device)
        return tlqr.tlqr_factor_create(plan, opts)

    def destroy_factor(self, f):
        tlqr.tlqr_factor_destroy(f)

    def stream(self):
        return self.torch.cuda.Stream(device=self.device)

    def outputs(self, req: Request):
        t = self.torch
        kw = dict(dtype=t.float64, device=self.device)
        return t.zeros((req.N, req.n), **kw), t.zeros((req.N, req.m), **kw), t.zeros((req.N, req.n), **kw)

    def solve(self, f, data, x, u, y, stream):
        self.torch.cuda.set_device(self.device)
        with self.torch.cuda.stream(stream):
            tlqr.tlqr_solve(f, data, x, u, y, stream=stream)
        return tlqr.tlqr_last_info(f)

    def ipm(self, plan, f, data, lo, hi, x, u, y, max_iter, stream):
        """Interior-point driver with a fixed Newton budget; reaching the budget
        before the gap tolerance is a normal end for a real-time request."""
        t = self.torch
        t.cuda.set_device(self.device)
        ll, lh = t.zeros_like(u), t.zeros_like(u)
        with t.cuda.stream(stream):
            try:
                info = tlqr.tlqr_ipm_box(plan, f, data, lo, hi, x, u, y, ll, lh, max_iter=max_iter,
                                         no_fp64_fallback=True, stream=stream)
                info["budget_exhausted"] = False
            except tlqr.TLQRError as e:
                if e.code != 8:                     # TLQR_ERR_NO_CONVERGENCE: the budget ran out
                    raise
                info = {"budget_exhausted": True}
        return info

    def synchronize(self, stream):
        stream.synchronize()


class Server:
    def __init__(self, slots: int = 8, memory_budget: int | None = None, backend=None, plan_cache: int = 256):
        self.backend = backend if backend is not None else TlqrBackend()
        if memory_budget is None:
            import torch
            free, _ = torch.cuda.mem_get_info()
            memory_budget = int(0.8 * free)
        self.budget = int(memory_budget)
        self.slots = int(slots)
        self.plan_cache_size = int(plan_cache)
        self.lock = threading.Condition()
        self.pending: collections.deque[Request] = collections.deque()
        self.plans: collections.OrderedDict = collections.OrderedDict()    # key -> [plan, refs]
        self.idle: collections.OrderedDict = collections.OrderedDict()     # (key, opts) -> [(factor, bytes)]
        self.in_use = 0            # bytes held by live factors (running or idle) + running requests' buffers
        self.peak = 0
        self.running = 0
        self.stats = collections.Counter()
        self.closed = False
        self.work: list[collections.deque] = [collections.deque() for _ in range(self.slots)]
        self.free_slots = list(range(self.slots))
        self.threads = [threading.Thread(target=self._slot_loop, args=(s,), daemon=True) for s in range(self.slots)]
        self.dispatcher = threading.Thread(target=self._dispatch_loop, daemon=True)
        for t in self.threads:
            t.start()
        self.dispatcher.start()

    # ------------------------------------------------------------------ public
    def submit(self, req: Request, arrival: float | None = None) -> Request:
        req.arrival = time.perf_counter() if arrival is None else arrival
        with self.lock:
            if self.closed:
                raise RuntimeError("server closed")
            self.pending.append(req)
            self.lock.notify_all()
        return req

    def drain(self):
        with self.lock:
            while self.pending or self.running:
                self.lock.wait()

    def close(self):
        self.drain()
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        self.dispatcher.join()
        for t in self.threads:
            t.join()
        for lst in self.idle.values():
            for f, _ in lst:
                self.backend.destroy_factor(f)
        self.idle.clear()
        for plan, _ in self.plans.values():
            self.backend.destroy_plan(plan)
        self.plans.clear()

    # ------------------------------------------------------------ scheduling
    def _plan_for(self, key, parent):
        ent = self.plans.get(key)
        if ent is not None:
            self.plans.move_to_end(key)
            self.stats["plan_hits"] += 1
            return ent
        self.stats["plan_misses"] += 1
        ent = [self.backend.plan(parent), 0]
        self.plans[key] = ent
        # drop unreferenced plans beyond the cache size
        for k in list(self.plans):
            if len(self.plans) <= self.plan_cache_size:
                break
            if self.plans[k][1] == 0 and k != key and not any(kk[0] == k for kk in self.idle):
                self.backend.destroy_plan(self.plans.pop(k)[0])
        return ent

    def _evict_idle(self, need: int) -> bool:
        """Free idle factors (LRU) until `need` more bytes fit; only while
        nothing runs.  True when the request now fits."""
        while self.in_use + need > self.budget and self.idle and self.running == 0:
            k, lst = next(iter(self.idle.items()))
            f, b = lst.pop()
            if not lst:
                del self.idle[k]
            self.backend.destroy_factor(f)
            self.in_use -= b
            self.plans[k[0]][1] -= 1
            self.stats["evictions"] += 1
        return self.in_use + need <= self.budget

    def _dispatch_loop(self):
        with self.lock:
            while True:
                while not self.closed and not self.pending:
                    self.lock.wait()
                if self.closed and not self.pending:
                    return
                req = self.pending[0]                       # FIFO: the head waits, nothing overtakes it
                if getattr(req, "_prep", None) is None:
                    key = topology_key(req.parent)
                    try:
                        ent = self._plan_for(key, req.parent)
                        opts = self.backend.options(req)
                    except BaseException as e:              # bad topology or options: fail the request
                        self.pending.popleft()
                        req.error, req.finished = e, time.perf_counter()
                        req.done.set()
                        self.lock.notify_all()
                        continue
                    req._prep = (key, ent, opts)
                key, ent, opts = req._prep
                okey = (key, req.n, req.m, req.precision, req.has_delta)
                bufs = solution_bytes(req.N, req.n, req.m) + problem_bytes(req.N, req.n, req.m, req.has_delta)
                if req.bounds is not None:
                    bufs += ipm_bytes(req.N, req.n, req.m)
                reuse = bool(self.idle.get(okey))
                wbytes = 0 if reuse else self.backend.workspace_bytes(ent[0], opts)
                need = wbytes + bufs
                if need > self.budget:
                    self.pending.popleft()
                    req.error = MemoryError(f"request needs {need} bytes, budget {self.budget}")
                    req.finished = time.perf_counter()
                    req.done.set()
                    self.lock.notify_all()
                    continue
                if not self.free_slots or not (self.in_use + need <= self.budget or self._evict_idle(need)):
                    self.lock.wait(timeout=0.05)
                    continue
                self.pending.popleft()
                slot = self.free_slots.pop()
                factor = None
                if reuse:
                    factor, wbytes = self.idle[okey].pop()
                    if not self.idle[okey]:
                        del self.idle[okey]
                    self.stats["factor_reuse"] += 1
                else:
                    ent[1] += 1
                    self.stats["factor_new"] += 1
                self.in_use += need
                self.peak = max(self.peak, self.in_use)
                self.running += 1
                req.admitted = time.perf_counter()
                req.reused_factor = reuse
                self.work[slot].append((req, ent, opts, okey, factor, wbytes, bufs))
                self.lock.notify_all()

    def _slot_loop(self, slot: int):
        stream = self.backend.stream()
        while True:
            with self.lock:
                while not self.work[slot] and not self.closed:
                    self.lock.wait()
                if not self.work[slot]:
                    return
                req, ent, opts, okey, factor, wbytes, bufs = self.work[slot].popleft()
            try:
                if factor is None:
                    factor = self.backend.create_factor(ent[0], opts)
                x, u, y = self.backend.outputs(req)
                if req.bounds is not None:
                    lo, hi = req.bounds(stream)
                    req.infos.append(self.backend.ipm(ent[0], factor, req.data(0, stream), lo, hi, x, u, y,
                                                      req.iterations, stream))
                else:
                    for it in range(req.iterations):
                        data = req.data(it, stream)
                        req.infos.append(self.backend.solve(factor, data, x, u, y, stream))
                self.backend.synchronize(stream)
                req.x, req.u, req.y = x, u, y
            except BaseException as e:
                req.error = e
            req.finished = time.perf_counter()
            with self.lock:
                if factor is not None:
                    self.idle.setdefault(okey, []).append((factor, wbytes))
                    self.idle.move_to_end(okey)
                    self.in_use -= bufs
                else:                                   # creation failed: nothing is held
                    self.in_use -= wbytes + bufs
                    ent[1] -= 1
                self.running -= 1
                self.free_slots.append(slot)
                self.stats["completed"] += 1
                self.lock.notify_all()
            req.done.set()


def latency_summary(reqs) -> dict:
    lat = np.array([r.latency for r in reqs if r.error is None])
    wait = np.array([r.admitted - r.arrival for r in reqs if r.error is None])
    if len(lat) == 0:
        return {"completed": 0}
    return {"completed": int(len(lat)), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(lat.mean()),
            "admission_wait_p50_ms": 1e3 * float(np.percentile(wait, 50)),
            "admission_wait_p99_ms": 1e3 * float(np.percentile(wait, 99))}
