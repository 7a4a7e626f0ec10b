"""Benchmark: tree-LQR nodes/s on the long-trunk irregular tree.

Workload: trunk of 4,096 nodes with random side branches, N = 65,536,
n = 12, m = 4, Delta = 1e-6 I on a seeded 10 % of the nonroot nodes, data as in
the input recipe (synthetic, seeded).  One step = one complete solve of the
tree (Alg. 1: factor + solve, plus FP64 iterative refinement in mixed
precision) with the problem already resident in HBM.  The headline is the
mixed-precision solver at eta <= 1e-8; the plain FP64 contraction on the same
GPU is measured in the same run for comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--mode mixed|fp64]

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
# FP32 lanes per SM x SMs x 2 flop per FMA x max SM clock (recipe figures); FP64 nominal.
FP32_PEAK_TFLOPS = 128 * 148 * 2 * 2.032e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--total", type=int, default=65536, help="tree size (default: the benchmark workload)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--quick", action="store_true",
                    help="time the headline mode only (no FP64 comparison, e2e or CPU legs); for profiler runs")
    return ap.parse_args()


def workload(total):
    return inputs.long_trunk(total=total)


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


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
def oracle_leg(w, budget_s=12.0, min_reps=1, max_reps=50):
    """Time the FP64 oracle (single thread) on the full workload for about budget_s."""
    from oracle import riccati
    riccati.build()
    times = []
    sol = None
    t_start = time.perf_counter()
    while len(times) < max_reps and (len(times) < min_reps or time.perf_counter() - t_start < budget_s):
        t0 = time.perf_counter()
        sol = riccati.tree_riccati(w.parent, w.n, w.m, w.data)
        times.append(time.perf_counter() - t0)
    return times, sol


def run_reference(args, rank):
    if rank != 0:
        return
    w = workload(args.total)
    N = len(w.parent)
    steps, warm = args.steps, args.warmup
    from oracle import riccati
    riccati.build()
    # each step is the full tree unless that would exceed ~3 minutes in total
    est = None
    t0 = time.perf_counter()
    riccati.tree_riccati(w.parent, w.n, w.m, w.data)
    est = time.perf_counter() - t0
    sub = N
    if est * (steps + warm) > 180:
        sub = max(1024, int(N * 180 / (est * (steps + warm))))
    wp = w
    if sub < N:      # breadth-first prefix of the tree: a connected subtree
        keep = np.arange(sub)
        wp = inputs.Workload(w.name + f"_prefix{sub}", w.parent[:sub].copy(), w.n, w.m,
                             {k: (None if v is None else v[:sub].copy()) for k, v in w.data.items()})
    for _ in range(warm):
        riccati.tree_riccati(wp.parent, wp.n, wp.m, wp.data)
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        riccati.tree_riccati(wp.parent, wp.n, wp.m, wp.data)
        ts.append(time.perf_counter() - t0)
    tot = sum(ts)
    value = len(wp.parent) * steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * tot / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "N": N, "n": w.n, "m": w.m, "sample_nodes": len(wp.parent)},
        "p50_ms": 1e3 * float(np.percentile(ts, 50)), "p99_ms": 1e3 * float(np.percentile(ts, 99)),
        "cpu_baseline": {"value": value, "unit": "nodes/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(wp.parent)} of {N} nodes per step, single-threaded C FP64 "
                                   f"sequential tree Riccati"},
        "e2e": {"value": value, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- our arm
def run_ours(args, rank, world, dist):
    import torch
    from paper_2608_01332_b300 import tlqr

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.total)
    N, n, m = len(w.parent), w.n, w.m
    mixed = args.mode == "mixed"
    prec = tlqr.TLQR_PREC_MIXED if mixed else tlqr.TLQR_PREC_FP64
    has_delta = w.data["Delta"] is not None
    dd = {k: (None if v is None else torch.from_numpy(v).to(dev)) for k, v in w.data.items()}
    x = torch.zeros((N, n), dtype=torch.float64, device=dev)
    u = torch.zeros((N, m), dtype=torch.float64, device=dev)
    y = torch.zeros((N, n), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MiB > L2
    stream = torch.cuda.current_stream(dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    def timed_steps(solver, K, profile_kinds=()):
        tlqr.tlqr_profile_mask(solver.f, profile_kinds)
        tlqr.tlqr_solve(solver.f, dd, x, u, y, stream=stream)   # (re)capture graphs outside the timing
        tlqr.tlqr_profile_read(solver.f)                     # reset counters
        ts = []
        barrier()
        for _ in range(K):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            tlqr.tlqr_solve(solver.f, dd, x, u, y, stream=stream)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        barrier()
        tlqr.tlqr_profile_mask(solver.f, ())
        return ts, tlqr.tlqr_profile_read(solver.f)

    solver = tlqr.TreeLQR(w.parent, n, m, prec, has_delta=has_delta)
    stats = solver.stats()
    # warm-up, and one fully profiled step to find the dominant kernel
    for _ in range(max(3, args.warmup)):
        tlqr.tlqr_solve(solver.f, dd, x, u, y, stream=stream)
    _, prof_all = timed_steps(solver, 1, tlqr.KERNEL_KINDS)
    dominant = max(prof_all, key=lambda k: prof_all[k]["ms"])
    with ClockSampler(local) as clk:
        ts, prof = timed_steps(solver, args.steps, (dominant,))
    info = tlqr.tlqr_last_info(solver.f)
    tot_ms = sum(ts)
    if dist is not None:
        t = torch.tensor([tot_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    ms_per_step = tot_ms / args.steps
    value = world * N / (ms_per_step / 1e3)
    gpu_launches = int(sum(p["launches"] for p in prof.values()))
    # accuracy of the last timed solution
    res = tlqr.tlqr_kkt_residual(solver.f, dd, x, u, y)
    sol_dev = dict(x=x.cpu().numpy(), u=u.cpu().numpy(), y=y.cpu().numpy())

    # plain FP64 contraction on the same GPU (the comparison of the metric)
    fp64 = None
    if mixed and not args.quick:
        s64 = tlqr.TreeLQR(w.parent, n, m, tlqr.TLQR_PREC_FP64, has_delta=has_delta)
        for _ in range(2):
            tlqr.tlqr_solve(s64.f, dd, x, u, y, stream=stream)
        ts64, _ = timed_steps(s64, max(3, min(args.steps, 10)))
        r64 = tlqr.tlqr_kkt_residual(s64.f, dd, x, u, y)
        ms64 = sum(ts64) / len(ts64)
        fp64 = {"value": N / (ms64 / 1e3), "unit": "nodes/s", "ms_per_step": ms64, "eta": r64["eta"],
                "p50_ms": float(np.percentile(ts64, 50)), "p99_ms": float(np.percentile(ts64, 99))}
        s64.close()

    # end to end through the public API with pinned host buffers
    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "nodes/s", "ms_per_step": ms_per_step,
                              "steps": args.steps, "eta": res["eta"], "quick": True,
                              "kernel_ms_per_step": {k: v["ms"] for k, v in prof_all.items() if v["ms"] > 0}}),
                  flush=True)
        solver.close()
        return
    hd = {k: (None if v is None else torch.from_numpy(v).pin_memory()) for k, v in w.data.items()}
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
    e2e_tot = sum(e2e_t)
    if dist is not None:
        t = torch.tensor([e2e_tot], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_tot = float(t.item())
    e2e_value = world * N * args.steps / e2e_tot

    if rank != 0:
        solver.close()
        return
    # roofline of the dominant kernel
    wbytes = 4 if mixed else 8
    dfrac = float((w.data["Delta"].reshape(N, -1) != 0).any(axis=1).mean()) if has_delta else 0.0
    fl, by = per_unit(dominant, n, m, wbytes, dfrac)
    pd = prof[dominant]
    roof = None
    hbm, hbm_src = load_peaks()
    if fl is not None and pd["timed"] > 0 and pd["ms"] > 0:
        sec = pd["ms"] / 1e3
        flops = fl * pd["units"] / sec
        bw = by * pd["units"] / sec
        fp32_kernel = mixed and dominant != "residual"
        peak_alu = (FP32_PEAK_TFLOPS if fp32_kernel else FP64_PEAK_TFLOPS) * 1e12
        t_alu = fl / peak_alu
        t_mem = by / (hbm * 1e9)
        if t_mem >= t_alu:
            roof = {"bound": "hbm", "achieved": bw / 1e9, "peak": hbm, "unit": "GB/s", "frac": bw / 1e9 / hbm,
                    "traffic": None, "peak_source": hbm_src}
        else:
            roof = {"bound": "alu", "achieved": flops / 1e12, "peak": peak_alu / 1e12, "unit": "TFLOP/s",
                    "frac": flops / peak_alu, "traffic": None,
                    "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 x 2.032 GHz" if fp32_kernel
                    else "nominal FP64 1.25 TFLOP/s"}
        roof.update({"kernel": f"k_{dominant}", "launches": pd["timed"], "units": pd["units"],
                     "avg_launch_ms": pd["ms"] / pd["timed"], "flops_per_unit": fl, "bytes_per_unit": by})

    line = {
        "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": w.name, "N": N, "n": n, "m": m, "trunk": 4096, "delta_fraction": 0.1,
                   "precision": args.mode, "rounds": stats["rounds"], "height": stats["height"],
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
        "eta": res["eta"], "refine_steps": info["refine_steps"] if mixed else 0,
        "plain_fp64": fp64,
        "e2e": {"value": e2e_value, "unit": "nodes/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
        "roofline": roof,
        "kernel_ms_per_step": {k: v["ms"] for k, v in prof_all.items() if v["ms"] > 0},
    }
    if not args.no_baseline:
        times, ref = oracle_leg(w)
        from oracle import riccati
        line["cpu_baseline"] = {"value": N / float(np.median(times)), "unit": "nodes/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"full workload ({N} nodes) x {len(times)} runs, single-threaded "
                                          f"C FP64 sequential tree Riccati, median"}
        line["forward_error_vs_oracle"] = riccati.forward_error(sol_dev, ref, w.parent)
    solver.close()
    print(json.dumps(line), flush=True)


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
        else:
            run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
