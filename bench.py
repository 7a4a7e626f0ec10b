"""Benchmark: tree-LQR nodes/s on the long-trunk irregular tree.

Workload: trunk of 4,096 nodes with random side branches, N = 65,536,
n = 12, m = 4, Delta = 1e-6 I on a seeded 10 % of the nonroot nodes, data as in
the input recipe (synthetic, seeded).  One step = one complete solve of the
tree (Alg. 1: factor + solve, plus FP64 iterative refinement in mixed
precision) with the problem already resident in HBM.  The headline is the
mixed-precision solver at eta <= 1e-8; the plain FP64 contraction on the same
GPU is measured in the same run for comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--mode mixed|fp64]
                    [--workload long_trunk|batch|spine]

The other workloads (a batch of 1,024 random recursive trees solved as one
forest; the N = 2^20 spine hybrid at n = 32, m = 8) print the same line with
their own config, a per-round roofline of the factorisation and no e2e leg
unless asked (their host copies are 15-20 GB).

Multi-GPU (torchrun): the single-tree path has no sharded form here, so every
rank solves its own replica of the workload (weak scaling, no collective on the
data path); value = nodes solved by all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2608_01332_b300 import inputs  # noqa: E402

METRIC = "tree-LQR nodes/sec at 1e-8 rel KKT residual vs plain FP64; p50/p99 solve latency"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Fallbacks when the on-device FMA microbenchmark (tlqr_pipe_peak) cannot run:
# FP32 lanes per SM x SMs x 2 flop per FMA x max SM clock (recipe figures); FP64 nominal.
FP32_PEAK_TFLOPS = 128 * 148 * 2 * 2.032e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def alu_peaks():
    """FP32 and FP64 FMA throughput measured on this GPU (TFLOP/s) with the
    library's FMA-chain microbenchmark, and where each number came from."""
    from paper_2608_01332_b300 import tlqr
    out = {}
    for key, prec, fallback, what in (("fp32", tlqr.TLQR_PREC_MIXED, FP32_PEAK_TFLOPS,
                                       "derived: 148 SM x 128 FP32 lanes x 2 x 2.032 GHz"),
                                      ("fp64", tlqr.TLQR_PREC_FP64, FP64_PEAK_TFLOPS, "nominal FP64 1.25 TFLOP/s")):
        try:
            out[key] = (tlqr.tlqr_pipe_peak(prec), "measured: FMA-chain microbenchmark on this GPU, this run")
        except Exception as e:                     # pragma: no cover - only without a working device
            out[key] = (fallback, f"{what} (microbenchmark failed: {e})")
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="long_trunk", choices=list(WORKLOADS),
                    help="long_trunk: the headline tree (N=65,536, n=12, m=4); batch: 1,024 random recursive "
                         "trees (n=16, m=4) solved as one forest; spine: N=2^20 spine hybrid (n=32, m=8)")
    ap.add_argument("--total", type=int, default=None, help="tree size (default: the workload's own)")
    ap.add_argument("--count", type=int, default=1024, help="batch: number of trees")
    ap.add_argument("--kappa", type=float, default=1e2, help="spine: condition number of R")
    ap.add_argument("--slots", type=int, default=8, help="serve: concurrent requests")
    ap.add_argument("--requests", type=int, default=200, help="serve: requests per arrival rate")
    ap.add_argument("--serve-mode", default="ipm", choices=["ipm", "perturb"],
                    help="serve: each request is a box-constrained interior-point solve with a 20-Newton-solve "
                         "budget (ipm), or 20 solves with randomly perturbed barrier-like diagonals (perturb)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--ref-seconds", type=float, default=180.0,
                    help="reference arm: CPU seconds for warm-up + timed steps together")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer leg")
    ap.add_argument("--e2e", action="store_true", help="run the end-to-end leg for the 10^6-node workloads too")
    ap.add_argument("--no-spine", action="store_true",
                    help="skip the per-round roofline of the N=2^20 spine tree in the default line")
    ap.add_argument("--pdl", type=int, default=None, choices=[0, -1],
                    help="programmatic dependent launch of the pass kernels (0 on, -1 off); default: on")
    ap.add_argument("--fp64-resolve", type=int, default=None, choices=[0, -1],
                    help="FP64 re-solves of ill-conditioned eliminations (0 on, -1 off); default: on")
    ap.add_argument("--residual", type=int, default=None, choices=[0, 1, 2],
                    help="refinement residual kernels (1 rows, 2 node-organised); default: the tuned table's")
    ap.add_argument("--quick", action="store_true",
                    help="time the headline mode only (no FP64 comparison, e2e or CPU legs); for profiler runs")
    return ap.parse_args()


WORKLOADS = {
    "long_trunk": "trunk 4,096 + random side branches, N=65,536, n=12, m=4, Delta=1e-6 I on 10% of edges",
    "serve": "Poisson arrivals of driving-style scenario trees (N in [500, 50000], n=6, m=2), 20 interior-point "
             "solves per request with fresh data each, continuous batching over slots",
    "batch": "1,024 random recursive trees, N log-uniform in [64, 16384], n=16, m=4, one forest",
    "spine": "2^16-node spine + random recursive subtrees of mean size 16, N=2^20, n=32, m=8, kappa(R) swept",
}


# ----------------------------------------------------------------- serving workload
class ServeTraffic:
    """Requests of the serving workload: a pool of driving-style topologies
    (N uniform in [500, 50000]), each with its model matrices drawn once on the
    device (the plant of one scenario-tree shape; drawing Haar-orthogonal A
    blocks for every request would cost more host time than the solves); a
    request picks a topology and draws its own gradient (q, r) -- and, as an
    interior-point request, its own control bounds; in the perturbation mode
    each of its solves also perturbs the barrier-like diagonal of Q and R --
    in place, so that the buffers (and the factor's captured graphs) stay the
    same across its solves."""

    def __init__(self, device, seed=inputs.BASE_SEED + 4, topologies=16, n=6, m=2, iterations=20,
                 lo=500, hi=50000, ipm=True):
        rng = inputs.rng_for(seed)
        self.device, self.seed, self.n, self.m, self.iterations = device, seed, n, m, iterations
        self.ipm = ipm
        self.trees = [inputs.driving_tree(rng, int(rng.integers(lo, hi + 1))) for _ in range(topologies)]
        self.rng = rng
        self.bases = [inputs.problem_data_device(p, n, m, seed * 1000 + t, device) for t, p in enumerate(self.trees)]

    def request(self, k, precision, t=None):
        """Request k (its data are a function of k alone) on topology t (drawn when None)."""
        import torch
        from paper_2608_01332_b300 import serve
        if t is None:
            t = int(self.rng.integers(len(self.trees)))
        parent = self.trees[t]
        g = torch.Generator(device=self.device)
        g.manual_seed(self.seed * 7919 + k)
        N, n, m = len(parent), self.n, self.m
        nr = torch.from_numpy(parent >= 0).to(self.device)
        base = dict(self.bases[t])
        base["q"] = torch.randn((N, n), generator=g, dtype=torch.float64, device=self.device)
        base["r"] = torch.randn((N, m), generator=g, dtype=torch.float64, device=self.device) * nr[:, None]

        live = None

        def data(it, stream):
            nonlocal live
            with torch.cuda.stream(stream):
                if live is None:                # the request's own copies, made on its slot's stream
                    live = {kk: (None if v is None else v.clone()) for kk, v in base.items()}
                sq = torch.rand((N, n), generator=g, dtype=torch.float64, device=self.device)
                sr = torch.rand((N, m), generator=g, dtype=torch.float64, device=self.device) * nr[:, None]
                live["Q"].copy_(base["Q"]).diagonal(dim1=1, dim2=2).add_(sq)
                live["R"].copy_(base["R"]).diagonal(dim1=1, dim2=2).add_(sr)
                live["q"].normal_(generator=g)
                live["r"].normal_(generator=g).mul_(nr[:, None])
            return live
        if not self.ipm:
            return serve.Request(parent=parent, n=n, m=m, iterations=self.iterations, data=data,
                                 precision=precision, tag=(k, t))

        # interior-point request: control bounds +-(0.3 + U[0, 1]) on every nonroot edge, solved by the
        # primal-dual driver with a budget of `iterations` Newton solves (each a fresh tree KKT system)
        def box(stream):
            with torch.cuda.stream(stream):
                lo = -(0.3 + torch.rand((N, m), generator=g, dtype=torch.float64, device=self.device))
                hi = 0.3 + torch.rand((N, m), generator=g, dtype=torch.float64, device=self.device)
                lo[~nr] = -float("inf")
                hi[~nr] = float("inf")
            return lo, hi

        def first(it, stream):
            return base
        return serve.Request(parent=parent, n=n, m=m, iterations=self.iterations, data=first, precision=precision,
                             tag=(k, t), bounds=box)


def run_serve(args, rank, world, dist):
    """Closed-loop capacity, then Poisson arrivals at 0.25 ... 1.1 x capacity."""
    import torch
    from paper_2608_01332_b300 import serve, tlqr

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = tlqr.TLQR_PREC_MIXED if args.mode == "mixed" else tlqr.TLQR_PREC_FP64
    traffic = ServeTraffic(dev, ipm=args.serve_mode == "ipm")
    slots = args.slots
    over = {k: v for k, v in (("pdl", args.pdl), ("fp64_resolve", args.fp64_resolve)) if v is not None}
    srv = serve.Server(slots=slots, backend=serve.TlqrBackend(**over))
    k = 0
    # warm-up: every topology once (plans, factors, graphs)
    warm = []
    for t in range(len(traffic.trees)):
        warm.append(traffic.request(k, prec))
        k += 1
    torch.cuda.synchronize(dev)                 # request data are drawn on this thread's stream
    for r in warm:
        srv.submit(r)
    srv.drain()
    # capacity: a closed burst of requests
    burst = [traffic.request(k + i, prec) for i in range(args.requests)]
    k += args.requests
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for r in burst:
        srv.submit(r)
    srv.drain()
    span = time.perf_counter() - t0
    errors = [repr(r.error) for r in warm + burst if r.error is not None]
    print(json.dumps({"serve_progress": "burst", "requests": len(burst), "seconds": span, "errors": errors[:3]}),
          file=sys.stderr, flush=True)

    def solves(r):                              # Newton solves a request ran (IPM requests may stop early)
        if r.bounds is None:
            return r.iterations
        return sum(i.get("iterations", r.iterations) for i in r.infos)

    def eta_of(i):
        return i.get("eta", i.get("last_eta"))

    nodes = sum(r.N * solves(r) for r in burst)
    capacity_rps = len(burst) / span
    value = nodes / span
    rates = []
    for fct in (0.25, 0.5, 0.75, 0.9, 1.1):
        lam = fct * capacity_rps
        reqs = [traffic.request(k + i, prec) for i in range(args.requests)]
        k += args.requests
        gaps = traffic.rng.exponential(1.0 / lam, size=len(reqs))
        torch.cuda.synchronize(dev)
        t_start = time.perf_counter()
        at = t_start
        for r, gap in zip(reqs, gaps):
            at += gap
            now = time.perf_counter()
            if at > now:
                time.sleep(at - now)
            srv.submit(r, arrival=at)
        srv.drain()
        t_end = max(r.finished for r in reqs)
        errors += [repr(r.error) for r in reqs if r.error is not None]
        summ = serve.latency_summary(reqs)
        summ.update({"rate_factor": fct, "rate_rps": lam,
                     "throughput_nodes_s": sum(r.N * solves(r) for r in reqs) / (t_end - t_start),
                     "max_eta": max((eta_of(i) for r in reqs for i in r.infos if eta_of(i) is not None),
                                    default=None),
                     "ipm_iterations_p50": float(np.median([i.get("iterations", traffic.iterations)
                                                            for r in reqs for i in r.infos]))
                     if traffic.ipm else None})
        rates.append(summ)
        print(json.dumps({"serve_progress": "rate", **{k: v for k, v in summ.items() if not isinstance(v, list)},
                          "errors": [repr(r.error) for r in reqs if r.error is not None][:3]}),
              file=sys.stderr, flush=True)
    stats = dict(srv.stats)
    peak = srv.peak
    srv.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world, "steps": len(burst),
        "warmup": len(warm), "ms_per_step": 1e3 * span / len(burst), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == tlqr.TLQR_PREC_MIXED else "f64",
        "data": "synthetic (seeded; drawn on the device)",
        "config": {"workload": "serve_driving_trees_n6_m2", "description": WORKLOADS["serve"], "slots": slots,
                   "requests_per_rate": args.requests, "iterations_per_request": traffic.iterations,
                   "topologies": len(traffic.trees), "precision": args.mode,
                   "step": ("one request: a box-constrained problem solved by the interior-point driver with "
                            "a budget of 20 Newton solves (each factor + solve + refinement)") if traffic.ipm else
                           "one request (20 solves, each factor + solve + refinement to eta <= 1e-8)"},
        "capacity_rps": capacity_rps, "burst_latency": serve.latency_summary(burst),
        "serving": rates, "server_stats": stats, "peak_admitted_bytes": peak, "errors": errors[:5],
    }
    print(json.dumps(line), flush=True)


def workload(args, device=None):
    """(Workload, forest?) -- host numpy data for the headline tree, device data
    (drawn on the GPU) for the 10^6-node workloads."""
    if args.workload == "long_trunk":
        return inputs.long_trunk(total=args.total or 65536), False
    if args.workload == "serve":                    # the oracle's view: the topology pool as one batch
        rng = inputs.rng_for(inputs.BASE_SEED + 4)
        trees = [inputs.driving_tree(rng, int(rng.integers(500, 50001))) for _ in range(16)]
        par, offs = inputs.forest(trees)
        return inputs.Workload("serve_driving_trees_n6_m2", par, 6, 2, inputs.problem_data(par, 6, 2, rng),
                               info=dict(offsets=offs)), True
    if device is None:
        import torch
        device = "cuda" if torch.cuda.is_available() else "cpu"
    if args.workload == "batch":
        return inputs.recursive_batch_device(device, count=args.count), True
    N = args.total or (1 << 20)                     # spine of N / 16 nodes (2^16 at full size)
    return inputs.spine_hybrid_device(device, N=N, spine=max(1, N >> 4), kappa_R=args.kappa), False


def host_slice(w, a, b):
    """Problem data of nodes [a, b) as host numpy arrays."""
    out = {}
    for k, v in w.data.items():
        if v is None:
            out[k] = None
        elif isinstance(v, np.ndarray):
            out[k] = np.ascontiguousarray(v[a:b])
        else:
            out[k] = v[a:b].cpu().numpy()
    return out


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# DRAM bytes per operation (dram__bytes_read.sum + dram__bytes_write.sum of one
# launch divided by its operation count) from one `ncu --set full` capture of
# the round-1 launch of the headline workload; keyed by (kernel kind, n, m,
# precision).  Entries must be dropped when the kernel changes.
# residual (float-float row kernel, refinement launches skipping zero Delta
# rows) on the long trunk, N = 65,536: dram__bytes_read.sum + write.sum =
# 274.67 MB and 271.72 MB for the two launches of a step (with / without the
# ||K|| row sums), i.e. 4,168.6 bytes per node (profiles/k_residual_ff_long_trunk_N65536.md)
NCU_BYTES_PER_OP = {("residual", 12, 4, "mixed"): 4168.6}


# ----------------------------------------------------------------- algorithmic work per unit
def per_unit(kind, n, m, wbytes, has_delta_frac=0.0):
    """(flops, bytes) of one local operation, leading-order dense counts with
    packed symmetric blocks (s = n(n+1)/2, f = n^2) as the minimal traffic."""
    s, f = n * (n + 1) / 2, n * n
    if kind == "rake":
        return 26 / 3 * n ** 3 + n ** 2, (f + 4 * s) * wbytes
    if kind == "compress":
        return 50 / 3 * n ** 3 + n ** 2, (3 * f + 8 * s) * wbytes
    if kind == "expand":
        return 26 / 3 * n ** 3, (f + 4 * s) * wbytes
    if kind == "compose_T":
        return 2 * n ** 3, 3 * f * wbytes
    if kind == "local_factor":
        fl = 6 * n * n * m + 4 * n * m * m + m ** 3 / 3 + has_delta_frac * 20 / 3 * n ** 3
        return fl, (s + f + 2 * n * m + m * m / 2 + m * n + f + m * m / 2) * wbytes + f * 8
    if kind == "residual":
        # FP64 rows of eq. (kkt): Q x, A^T y, A x, B u, B^T y, R u (+ Delta y twice) per node
        fl = 2 * (3 * n * n + 2 * n * m + m * m) + has_delta_frac * 4 * n * n
        return fl, (2 * f + n * m + m * m + has_delta_frac * f + 8 * n + 4 * m) * 8
    if kind == "condense":
        return m ** 3 / 3 + 2 * n * m * m + 2 * n * n * m, (f + n * m + m * m / 2 + 2 * s) * 8
    return None, None


class ClockSampler:
    """Samples SM clock and throttle reasons with NVML during the timed region."""

    def __init__(self, index):
        self.index, self.samples, self.reasons, self.stop_ev = index, [], set(), threading.Event()
        self.max_mhz = None
        self.ok = False
        self.error = None
        self.proc = None
        try:
            import pynvml
            pynvml.nvmlInit()
            self.nv = pynvml
            self.h = pynvml.nvmlDeviceGetHandleByIndex(index)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
            self.samples.append(pynvml.nvmlDeviceGetClockInfo(self.h, pynvml.NVML_CLOCK_SM))
            self.samples.clear()
            self.ok = True
        except Exception as e:
            self.error = f"nvml: {e!r}"


    def _run(self):
        nv = self.nv
        names = {getattr(nv, "nvmlClocksEventReasonHwSlowdown", 0x8): "hw_slowdown",
                 getattr(nv, "nvmlClocksEventReasonHwThermalSlowdown", 0x40): "hw_thermal_slowdown",
                 getattr(nv, "nvmlClocksEventReasonSwThermalSlowdown", 0x20): "sw_thermal_slowdown",
                 getattr(nv, "nvmlClocksEventReasonSwPowerCap", 0x4): "sw_power_cap",
                 getattr(nv, "nvmlClocksEventReasonHwPowerBrakeSlowdown", 0x80): "hw_power_brake"}
        while not self.stop_ev.is_set():
            try:
                self.samples.append(nv.nvmlDeviceGetClockInfo(self.h, nv.NVML_CLOCK_SM))
                r = nv.nvmlDeviceGetCurrentClocksEventReasons(self.h)
                for bit, name in names.items():
                    if r & bit:
                        self.reasons.add(name)
            except Exception:
                pass
            self.stop_ev.wait(0.05)

    def _run_smi(self):
        import subprocess
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception as e:
            self.error = f"nvidia-smi: {e}"
            return
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            f = [v.strip() for v in line.split(",")]
            try:
                self.samples.append(float(f[0]))
                self.max_mhz = float(f[1])
                for nm, v in zip(names, f[2:]):
                    if v.lower() == "active":
                        self.reasons.add(nm)
            except (ValueError, IndexError):
                pass

    def __enter__(self):
        target = self._run if self.ok else self._run_smi
        self.t = threading.Thread(target=target, daemon=True)
        self.t.start()
        time.sleep(0.2)
        return self

    def __exit__(self, *a):
        self.stop_ev.set()
        if getattr(self, "proc", None) is not None:
            time.sleep(0.1)
            self.proc.terminate()
        self.t.join(timeout=5)

    def summary(self):
        src = "nvml" if self.ok else "nvidia-smi"
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"], "source": src,
                    "error": self.error}
        return {"sm_mhz": float(np.median(self.samples)), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples), "source": src}


# ----------------------------------------------------------------- CPU oracle legs
def oracle_units(w, forest):
    """Independent pieces the oracle can time: whole trees of a batch, else the
    tree itself (a prefix of the labels when it is too large; every parent label
    is below its child's, so a prefix is a connected subtree)."""
    if forest:
        offs = [int(v) for v in w.info["offsets"]] + [len(w.parent)]
        return [(offs[t], offs[t + 1]) for t in range(len(offs) - 1)]
    return [(0, len(w.parent))]


def oracle_leg(w, forest, budget_s=12.0, max_reps=50):
    """Time the FP64 oracle (single thread) for about budget_s on the workload:
    the full tree (repeated), consecutive trees of a batch, or a prefix of a tree
    too large for the budget.  Returns (nodes/s, description, solution of the
    full tree or None)."""
    from oracle import riccati
    riccati.build()
    units = oracle_units(w, forest)
    N = len(w.parent)
    if not forest and N > 200_000:                      # too large: a timed prefix
        probe = 4096
        d = host_slice(w, 0, probe)
        t0 = time.perf_counter()
        riccati.tree_riccati(w.parent[:probe], w.n, w.m, d)
        per_node = (time.perf_counter() - t0) / probe
        k = int(min(N, max(probe, budget_s / 2 / per_node)))
        d = host_slice(w, 0, k)
        times = []
        t_start = time.perf_counter()
        while len(times) < 2 and (not times or time.perf_counter() - t_start < budget_s):
            t0 = time.perf_counter()
            riccati.tree_riccati(w.parent[:k], w.n, w.m, d)
            times.append(time.perf_counter() - t0)
        return k / float(np.median(times)), f"prefix of {k} of {N} nodes (labels 0..{k - 1}) x {len(times)}", None
    nodes, secs, sol, done = 0, 0.0, None, 0
    t_start = time.perf_counter()
    reps = 0
    while time.perf_counter() - t_start < budget_s and reps < max_reps:
        for a, b in units:
            p = w.parent[a:b] - np.where(w.parent[a:b] >= 0, a, 0)
            d = host_slice(w, a, b)
            t0 = time.perf_counter()
            out = riccati.tree_riccati(p.astype(np.int32), w.n, w.m, d)
            secs += time.perf_counter() - t0
            nodes += b - a
            done += 1
            if len(units) == 1:
                sol = out
            if time.perf_counter() - t_start > budget_s:
                break
        reps += 1
    if forest:
        desc = f"{done} trees of the batch ({nodes} nodes), one at a time"
    else:
        desc = f"full workload ({N} nodes) x {reps} runs"
    return nodes / secs, desc, sol


def run_reference(args, rank):
    if rank != 0:
        return
    w, forest = workload(args)
    N = len(w.parent)
    steps, warm = args.steps, args.warmup
    from oracle import riccati
    riccati.build()
    units = oracle_units(w, forest)
    # one step = the oracle over a bounded sample of the workload, sized so
    # that warm-up + timed steps take about three minutes in total
    a0, b0 = units[0]
    probe_b = min(b0, a0 + 4096)
    p = (w.parent[a0:probe_b] - np.where(w.parent[a0:probe_b] >= 0, a0, 0)).astype(np.int32)
    d = host_slice(w, a0, probe_b)
    t0 = time.perf_counter()
    riccati.tree_riccati(p, w.n, w.m, d)
    per_node = (time.perf_counter() - t0) / (probe_b - a0)
    budget_nodes = max(256, int(args.ref_seconds / (steps + warm) / per_node))
    sample = []
    tot = 0
    for a, b in units:
        if tot >= budget_nodes:
            break
        b = min(b, a + budget_nodes - tot)     # a label prefix of a tree is a subtree
        pp = (w.parent[a:b] - np.where(w.parent[a:b] >= 0, a, 0)).astype(np.int32)
        sample.append((pp, host_slice(w, a, b)))
        tot += int(b - a)
    for _ in range(warm):
        for pp, dd in sample:
            riccati.tree_riccati(pp, w.n, w.m, dd)
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        for pp, dd in sample:
            riccati.tree_riccati(pp, w.n, w.m, dd)
        ts.append(time.perf_counter() - t0)
    total_s = sum(ts)
    value = tot * steps / total_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * total_s / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "N": N, "n": w.n, "m": w.m, "sample_nodes": tot},
        "p50_ms": 1e3 * float(np.percentile(ts, 50)), "p99_ms": 1e3 * float(np.percentile(ts, 99)),
        "cpu_baseline": {"value": value, "unit": "nodes/s", "cores": 1, "kind": "oracle",
                         "sample": f"{tot} of {N} nodes per step ({len(sample)} tree(s) or label prefixes), "
                                   f"single-threaded C FP64 sequential tree Riccati"},
        "e2e": {"value": value, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- per-round roofline
ROUND_KINDS = ("rake", "absorb", "compress", "expand", "compose_T", "factor_tail")


def round_roofline(launches, rnd, op, n, m, wbytes, hbm_gbs, alu_tflops, rake_code, comp_code):
    """Per structural round of the factorisation: algorithmic flops and bytes of
    its rake, absorb and compress launches (and of the reverse expansion and
    T-composite launches of the same round), the measured time, and the
    roofline time max(bytes / HBM, flops / ALU peak).  The late rounds that the
    library runs in its level-asynchronous launch (contraction and expansion,
    kind factor_tail), together with their T-composite launches, form one row.

    launches: (kind, operations, ms) in launch order for one factorisation."""
    R = int(rnd.max()) if len(rnd) else 0
    nr = np.bincount(rnd[op == rake_code], minlength=R + 1)
    nc = np.bincount(rnd[op == comp_code], minlength=R + 1)
    seq = [rec for rec in launches if rec[0] in ROUND_KINDS]
    pos = 0
    s = n * (n + 1) / 2
    rows = {r: dict(round=r, rakes=int(nr[r]), compresses=int(nc[r]), flops=0.0, bytes=0.0, ms=0.0)
            for r in range(1, R + 1)}

    def take(kind, r, units_expected=None):
        nonlocal pos
        if pos >= len(seq) or seq[pos][0] != kind:
            got = seq[pos][0] if pos < len(seq) else "end"
            raise RuntimeError(f"round {r}: expected a {kind} launch, found {got}")
        _, units, ms = seq[pos]
        pos += 1
        if units_expected is not None and units != units_expected:
            raise RuntimeError(f"round {r}: {kind} launch of {units} operations, plan has {units_expected}")
        return units, ms

    def work(kind, units, n_contrib=0):
        if kind == "absorb":                       # sum contributions into U_i: reads nr + 2 ns packed blocks
            return n * n * n_contrib, (n_contrib + 2 * units) * s * wbytes
        fl1, by1 = per_unit(kind, n, m, wbytes)
        return fl1 * units, by1 * units

    def add(r, kind, units, ms, n_contrib=0):
        fl, by = work(kind, units, n_contrib)
        rows[r]["flops"] += fl
        rows[r]["bytes"] += by
        rows[r]["ms"] += ms

    r0 = R + 1                                      # first round of the tail (none: R + 1)
    for r in range(1, R + 1):                       # forward rounds
        if pos < len(seq) and seq[pos][0] == "factor_tail":
            r0 = r
            break
        if nr[r]:
            u, ms = take("rake", r, int(nr[r]))
            add(r, "rake", u, ms)
            u, ms = take("absorb", r)
            add(r, "absorb", u, ms, int(nr[r]))
        if nc[r]:
            u, ms = take("compress", r, int(nc[r]))
            add(r, "compress", u, ms)
    tail_ms = 0.0
    if r0 <= R:
        tail_ms += take("factor_tail", r0)[1]
    for r in range(min(R, r0 - 1), 0, -1):          # reverse expansion of the head rounds
        if nc[r]:
            u, ms = take("expand", r, int(nc[r]))
            add(r, "expand", u, ms)
    for r in range(1, R + 1):                       # T composites, every round
        if nc[r]:
            u, ms = take("compose_T", r, int(nc[r]))
            if r < r0:
                add(r, "compose_T", u, ms)
            else:
                tail_ms += ms
    out = []
    for r in range(1, min(R, r0 - 1) + 1):
        out.append(rows[r])
    if r0 <= R:
        t = dict(round=f"{r0}-{R} (tail)", rakes=int(nr[r0:].sum()), compresses=int(nc[r0:].sum()),
                 flops=0.0, bytes=0.0, ms=tail_ms)
        for r in range(r0, R + 1):
            for kind, cnt in (("rake", nr[r]), ("compress", nc[r]), ("expand", nc[r]), ("compose_T", nc[r])):
                fl, by = work(kind, int(cnt))
                t["flops"] += fl
                t["bytes"] += by
        out.append(t)
    for row in out:
        t_roof = max(row["bytes"] / (hbm_gbs * 1e9), row["flops"] / (alu_tflops * 1e12))
        row["roof_ms"] = 1e3 * t_roof
        row["frac"] = (1e3 * t_roof / row["ms"]) if row["ms"] > 0 else None
        row["bound"] = "hbm" if row["bytes"] / (hbm_gbs * 1e9) >= row["flops"] / (alu_tflops * 1e12) else "alu"
    return out


def profiled_rounds(solver, solve, N, n, m, wbytes, hbm, alu, dev):
    """Per-round roofline rows of one factorisation (launches of the round kinds
    timed one by one with CUDA events in a separate, untimed step)."""
    import torch
    from paper_2608_01332_b300 import tlqr
    solve()
    tlqr.tlqr_profile_mask(solver.f, ROUND_KINDS)
    solve()
    solve()
    torch.cuda.synchronize(dev)
    launches = tlqr.tlqr_profile_launches(solver.f)
    tlqr.tlqr_profile_mask(solver.f, ())
    tlqr.tlqr_profile_read(solver.f)
    rnd, op = tlqr.tlqr_plan_schedule(solver.plan, N)
    try:
        half = len(launches) // 2                  # two identical steps were recorded: keep the second
        return round_roofline(launches[half:], rnd, op, n, m, wbytes, hbm, alu,
                              tlqr.TLQR_OP_RAKE, tlqr.TLQR_OP_COMPRESS)
    except RuntimeError as e:
        return {"error": str(e)}


def spine_round_roofline(dev, hbm, fp32_peak):
    """Per-round roofline of the factorisation of the N = 2^20 spine hybrid
    (n = 32, m = 8, kappa(R) = 1e2, mixed precision), measured in the same run
    as the headline; rounds 1-3 hold 95 % of its operations."""
    import torch
    from paper_2608_01332_b300 import tlqr
    w = inputs.spine_hybrid_device(dev)
    N, n, m = len(w.parent), w.n, w.m
    dd = w.data
    x = torch.zeros((N, n), dtype=torch.float64, device=dev)
    u = torch.zeros((N, m), dtype=torch.float64, device=dev)
    y = torch.zeros((N, n), dtype=torch.float64, device=dev)
    s = tlqr.TreeLQR(w.parent, n, m, tlqr.TLQR_PREC_MIXED)
    try:
        solve = lambda: tlqr.tlqr_solve(s.f, dd, x, u, y)  # noqa: E731
        for _ in range(2):
            solve()
        rows = profiled_rounds(s, solve, N, n, m, 4, hbm, fp32_peak[0], dev)
        eta = tlqr.tlqr_last_info(s.f).get("eta")
    finally:
        s.close()
    del dd, x, u, y, w
    torch.cuda.empty_cache()
    if not isinstance(rows, list):
        return rows
    tot_meas = sum(r["ms"] for r in rows)
    tot_roof = sum(r["roof_ms"] for r in rows)
    head = [r for r in rows if isinstance(r["round"], int) and r["round"] <= 3]
    return {"workload": f"spine_hybrid_N{N}_n{n}_m{m}_kR100 (mixed)", "eta": eta,
            "frac": tot_roof / tot_meas if tot_meas > 0 else None, "measured_ms": tot_meas, "roof_ms": tot_roof,
            "frac_rounds_1_3": (sum(r["roof_ms"] for r in head) / sum(r["ms"] for r in head)) if head else None,
            "alu_peak_tflops": fp32_peak[0], "alu_peak_source": fp32_peak[1], "hbm_gbs": hbm,
            "rounds": [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in r.items()} for r in rows]}


# ----------------------------------------------------------------- our arm
def run_ours(args, rank, world, dist):
    import torch
    from paper_2608_01332_b300 import tlqr

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, forest = workload(args, dev)
    N, n, m = len(w.parent), w.n, w.m
    mixed = args.mode == "mixed"
    prec = tlqr.TLQR_PREC_MIXED if mixed else tlqr.TLQR_PREC_FP64
    has_delta = w.data["Delta"] is not None
    dd = {k: (None if v is None else (torch.from_numpy(v).to(dev) if isinstance(v, np.ndarray) else v))
          for k, v in w.data.items()}
    x = torch.zeros((N, n), dtype=torch.float64, device=dev)
    u = torch.zeros((N, m), dtype=torch.float64, device=dev)
    y = torch.zeros((N, n), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream(dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    def timed(solver, K, call, profile_kinds=()):
        tlqr.tlqr_profile_mask(solver.f, profile_kinds)
        call()                                       # (re)capture graphs outside the timing
        tlqr.tlqr_profile_read(solver.f)             # reset counters
        ts = []
        barrier()
        for _ in range(K):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        barrier()
        tlqr.tlqr_profile_mask(solver.f, ())
        return ts, tlqr.tlqr_profile_read(solver.f)

    # execution shape chosen by the autotuner for this workload (committed table), mixed precision only
    from paper_2608_01332_b300 import autotune
    tuned = autotune.tuned_options(args.workload) if mixed and args.total is None else {}
    if args.residual is not None:
        tuned["residual"] = args.residual
    if args.pdl is not None:
        tuned["pdl"] = args.pdl
    if args.fp64_resolve is not None:
        tuned["fp64_resolve"] = args.fp64_resolve
    solver = tlqr.TreeLQR(w.parent, n, m, prec, has_delta=has_delta, forest=forest, **tuned)
    stats = solver.stats()

    def solve():
        tlqr.tlqr_solve(solver.f, dd, x, u, y, stream=stream)

    # warm-up, and one fully profiled step to find the dominant kernel
    for _ in range(max(3, args.warmup)):
        solve()
    _, prof_all = timed(solver, 1, solve, tlqr.KERNEL_KINDS)
    # the dominant kernel among those with an algorithmic work model (per_unit)
    modeled = [k for k in prof_all if per_unit(k, n, m, 4 if mixed else 8)[0] is not None]
    dominant = max(modeled, key=lambda k: prof_all[k]["ms"])
    with ClockSampler(local) as clk:
        # the headline: K steps with no event inside the step; then the same K
        # steps again with CUDA events around each launch of the dominant kernel,
        # for its roofline (events in the launch graph lengthen the step)
        ts, prof_plain = timed(solver, args.steps, solve, ())
        ts_k, prof = timed(solver, args.steps, solve, (dominant,))
    info = tlqr.tlqr_last_info(solver.f)
    tot_ms = max_over_ranks(sum(ts), dist, dev)
    ms_per_step = tot_ms / args.steps
    value = world * N / (ms_per_step / 1e3)
    gpu_launches = int(sum(p["launches"] for p in prof_plain.values()))
    # accuracy of the last timed solution (per tree for a batch)
    res = tlqr.tlqr_kkt_residual(solver.f, dd, x, u, y)
    tree_eta = tlqr.tlqr_tree_residuals(solver.f, stats["n_trees"])[1]

    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "nodes/s", "ms_per_step": ms_per_step,
                              "steps": args.steps, "eta": res["eta"], "quick": True, "workload": w.name,
                              "kernel_ms_per_step": {k: v["ms"] for k, v in prof_all.items() if v["ms"] > 0}}),
                  flush=True)
        solver.close()
        return
    sol_dev = dict(x=x.cpu().numpy(), u=u.cpu().numpy(), y=y.cpu().numpy()) if N <= 200_000 else None

    # factor and solve separately (factor; one FP32/FP64 pass through the factors, no refinement)
    K_split = max(3, min(args.steps, 20))
    ts_f, _ = timed(solver, K_split, lambda: tlqr.tlqr_factor(solver.f, dd, stream=stream))
    xs, us, ys = torch.empty_like(x), torch.empty_like(u), torch.empty_like(y)
    ts_s, _ = timed(solver, K_split, lambda: tlqr.tlqr_solve_rhs(solver.f, dd["q"], dd["r"], dd["c"], xs, us, ys,
                                                                  stream=stream))
    split = {"factor_ms": float(np.median(ts_f)), "solve_rhs_ms": float(np.median(ts_s)),
             "note": "medians; solve_rhs = one pass through the factors without refinement"}
    # several right-hand sides with one factor: a panel of 8 against 8 separate passes
    multi = None
    if N <= 200_000:
        K = 8
        qk = dd["q"].unsqueeze(0).repeat(K, 1, 1).contiguous()
        rk = dd["r"].unsqueeze(0).repeat(K, 1, 1).contiguous()
        ck = dd["c"].unsqueeze(0).repeat(K, 1, 1).contiguous()
        qk += torch.randn_like(qk); ck += torch.randn_like(ck)
        xk, uk, yk = torch.empty_like(qk), torch.empty_like(rk), torch.empty_like(qk)
        ts_p, _ = timed(solver, K_split, lambda: tlqr.tlqr_solve_rhs_panel(solver.f, qk, rk, ck, xk, uk, yk,
                                                                          stream=stream))

        def one_by_one():
            for k in range(K):
                tlqr.tlqr_solve_rhs(solver.f, qk[k], rk[k], ck[k], xk[k], uk[k], yk[k], stream=stream)
        ts_o, _ = timed(solver, K_split, one_by_one)
        multi = {"nrhs": K, "panel_ms": float(np.median(ts_p)), "one_by_one_ms": float(np.median(ts_o)),
                 "speedup": float(np.median(ts_o) / np.median(ts_p)),
                 "note": "one pass through the factors per right-hand side (no refinement), medians"}
        del qk, rk, ck, xk, uk, yk

    # per-round roofline of the factorisation (one profiled step, launches timed one by one)
    wbytes = 4 if mixed else 8
    hbm, hbm_src = load_peaks()
    peaks = alu_peaks()
    alu, alu_src = peaks["fp32"] if mixed else peaks["fp64"]
    per_round = profiled_rounds(solver, solve, N, n, m, wbytes, hbm, alu, dev)

    # plain FP64 contraction on the same GPU (the comparison of the metric)
    fp64 = None
    if mixed:
        s64 = tlqr.TreeLQR(w.parent, n, m, tlqr.TLQR_PREC_FP64, has_delta=has_delta, forest=forest)
        call64 = lambda: tlqr.tlqr_solve(s64.f, dd, x, u, y, stream=stream)  # noqa: E731
        for _ in range(2):
            call64()
        ts64, _ = timed(s64, max(3, min(args.steps, 10)), call64)
        r64 = tlqr.tlqr_kkt_residual(s64.f, dd, x, u, y)
        ms64 = sum(ts64) / len(ts64)
        fp64 = {"value": world * N / (ms64 / 1e3), "unit": "nodes/s", "ms_per_step": ms64, "eta": r64["eta"],
                "p50_ms": float(np.percentile(ts64, 50)), "p99_ms": float(np.percentile(ts64, 99))}
        s64.close()

    # end to end through the public API with pinned host buffers
    e2e = e2e_update = None
    if not args.no_e2e and (args.workload == "long_trunk" or args.e2e):
        hd = {k: (None if v is None else v.cpu().pin_memory()) for k, v in dd.items()}
        hx = torch.zeros((N, n), dtype=torch.float64).pin_memory()
        hu = torch.zeros((N, m), dtype=torch.float64).pin_memory()
        hy = torch.zeros((N, n), dtype=torch.float64).pin_memory()
        tlqr.tlqr_solve(solver.f, hd, hx, hu, hy, stream=stream)
        h2d = sum(v.numel() * 8 for v in hd.values() if v is not None)
        d2h = (hx.numel() + hu.numel() + hy.numel()) * 8
        barrier()
        e2e_t = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            tlqr.tlqr_solve(solver.f, hd, hx, hu, hy, stream=stream)
            e2e_t.append(time.perf_counter() - t0)
        barrier()
        e2e_tot = max_over_ranks(sum(e2e_t), dist, dev)
        e2e = {"value": world * N * args.steps / e2e_tot, "unit": "nodes/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
        # the interior-point / receding-horizon pattern through tlqr_update_solve: diagonal
        # increments of Q and R and the right-hand side cross the bus, the rest stays resident;
        # the increments alternate in sign so the problem returns to the original every 2 steps
        hdq = torch.full((N, n), 1e-2, dtype=torch.float64).pin_memory()
        hdr = torch.full((N, m), 1e-2, dtype=torch.float64).pin_memory()
        hdqn, hdrn = (-hdq).pin_memory(), (-hdr).pin_memory()
        upd_in = dict(q=hd["q"], r=hd["r"], c=hd["c"])
        tlqr.tlqr_update_solve(solver.f, hx, hu, hy, dq=hdq, dr=hdr, stream=stream, **upd_in)
        tlqr.tlqr_update_solve(solver.f, hx, hu, hy, dq=hdqn, dr=hdrn, stream=stream, **upd_in)
        barrier()
        upd_t = []
        for k in range(args.steps):
            t0 = time.perf_counter()
            tlqr.tlqr_update_solve(solver.f, hx, hu, hy, dq=hdq if k % 2 == 0 else hdqn,
                                   dr=hdr if k % 2 == 0 else hdrn, stream=stream, **upd_in)
            upd_t.append(time.perf_counter() - t0)
        barrier()
        upd_tot = max_over_ranks(sum(upd_t), dist, dev)
        e2e_update = {"value": world * N * args.steps / upd_tot, "unit": "nodes/s",
                      "h2d_bytes_per_step": (hdq.numel() + hdr.numel() + sum(v.numel() for v in upd_in.values())) * 8,
                      "d2h_bytes_per_step": d2h,
                      "call": "tlqr_update_solve: Q, R diagonal increments and q, r, c uploaded each step; "
                              "A, B, Delta and the off-diagonal entries stay resident; factor + solve + refinement"}

    if rank != 0:
        solver.close()
        return
    # roofline of the dominant kernel
    dfrac = float((dd["Delta"].reshape(N, -1) != 0).any(dim=1).double().mean()) if has_delta else 0.0
    fl, by = per_unit(dominant, n, m, wbytes, dfrac)
    pd = prof[dominant]
    roof = None
    if fl is not None and pd["timed"] > 0 and pd["ms"] > 0:
        sec = pd["ms"] / 1e3
        flops = fl * pd["units"] / sec
        bw = by * pd["units"] / sec
        fp32_kernel = mixed                        # in mixed precision every kernel runs on the FP32 pipe
                                                   # (the residual in float-float arithmetic)
        peak_alu, peak_alu_src = peaks["fp32"] if fp32_kernel else peaks["fp64"]
        peak_alu *= 1e12
        t_alu = fl / peak_alu
        t_mem = by / (hbm * 1e9)
        if t_mem >= t_alu:
            roof = {"bound": "hbm", "achieved": bw / 1e9, "peak": hbm, "unit": "GB/s", "frac": bw / 1e9 / hbm,
                    "traffic": None, "peak_source": hbm_src}
        else:
            roof = {"bound": "alu", "achieved": flops / 1e12, "peak": peak_alu / 1e12, "unit": "TFLOP/s",
                    "frac": flops / peak_alu, "traffic": None, "peak_source": peak_alu_src}
        roof.update({"kernel": f"k_{dominant}", "launches": pd["timed"], "units": pd["units"],
                     "avg_launch_ms": pd["ms"] / pd["timed"], "flops_per_unit": fl, "bytes_per_unit": by,
                     "timing": "CUDA events around each launch of the kernel on its stream, over a second timed "
                               "pass of the same K steps (the headline steps run without events)",
                     "instrumented_ms_per_step": sum(ts_k) / len(ts_k)})
        bpo = NCU_BYTES_PER_OP.get((dominant, n, m, args.mode))
        if bpo is not None:
            roof["traffic"] = bpo * pd["units"] / pd["timed"]
            roof["traffic_note"] = ("ncu DRAM bytes per unit of this kernel (capture summarised under profiles/) "
                                    "x this run's average units per launch (bytes per launch)")

    cfg = {"workload": w.name, "N": N, "n": n, "m": m, "precision": args.mode, "rounds": stats["rounds"],
           "execution": tuned or "library defaults",
           "height": stats["height"], "trees": stats["n_trees"], "description": WORKLOADS[args.workload],
           "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}"}
    if args.workload == "spine":
        cfg["kappa_R"] = args.kappa
    line = {
        "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64",
        "data": "synthetic (seeded; host numpy)" if args.workload == "long_trunk"
        else "synthetic (seeded; drawn on the device)",
        "config": cfg,
        "p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
        "eta": res["eta"], "refine_steps": info["refine_steps"] if mixed else 0,
        "fp64_resolves": info.get("fp64_resolves", 0),
        "tree_eta": {"max": float(tree_eta.max()), "p50": float(np.percentile(tree_eta, 50))} if forest else None,
        "factor_solve": split,
        "multi_rhs": multi,
        "plain_fp64": fp64,
        "e2e": e2e,
        "e2e_update": e2e_update,
        "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
        "roofline": roof,
        "kernel_ms_per_step": {k: v["ms"] for k, v in prof_all.items() if v["ms"] > 0},
    }
    if isinstance(per_round, list):
        tot_meas = sum(r["ms"] for r in per_round)
        tot_roof = sum(r["roof_ms"] for r in per_round)
        line["round_roofline"] = {
            "frac": tot_roof / tot_meas if tot_meas > 0 else None, "measured_ms": tot_meas, "roof_ms": tot_roof,
            "alu_peak_tflops": alu, "alu_peak_source": alu_src, "hbm_gbs": hbm,
            "rounds": [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in r.items()} for r in per_round]}
    else:
        line["round_roofline"] = per_round
    line["alu_peaks_tflops"] = {k: {"value": v[0], "source": v[1]} for k, v in peaks.items()}
    if args.workload == "long_trunk" and not args.no_spine and rank == 0:
        line["spine_round_roofline"] = spine_round_roofline(dev, hbm, peaks["fp32"])
    if not args.no_baseline:
        v_cpu, desc, ref = oracle_leg(w, forest)
        line["cpu_baseline"] = {"value": v_cpu, "unit": "nodes/s", "cores": 1, "kind": "oracle",
                                "sample": desc + ", single-threaded C FP64 sequential tree Riccati"}
        if ref is not None and sol_dev is not None:
            from oracle import riccati
            line["forward_error_vs_oracle"] = riccati.forward_error(sol_dev, ref, w.parent)
    solver.close()
    print(json.dumps(line), flush=True)


def max_over_ranks(value: float, dist, device) -> float:
    """The largest `value` over the ranks of the job (the value itself with no
    process group): the timed region of the slowest replica sets the job's time."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        backend = "nccl" if args.impl == "ours" and torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group(backend=backend)
        dist = tdist
    try:
        if args.impl == "reference":
            run_reference(args, rank)
        elif args.workload == "serve":
            run_serve(args, rank, world, dist)
        else:
            run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
