"""CPU tests of the benchmark harness: the reference arm (the oracle timed on
host cores) prints one well-formed JSON line, also as rank 0 of a two-rank
gloo job whose other rank exits without work; and the per-round roofline
bookkeeping matches launches to the plan's rounds exactly."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2608_01332_b300 import inputs, tlqr
from tests.conftest import ROOT

sys.path.insert(0, ROOT)
import bench  # noqa: E402

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(args, env=None, timeout=600):
    out = subprocess.run([sys.executable, *args], cwd=ROOT, capture_output=True, text=True, timeout=timeout,
                         env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    return out.stdout


def test_reference_arm_line():
    line = _run(["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1", "--total", "2048",
                 "--ref-seconds", "2"])
    rows = [json.loads(s) for s in line.splitlines() if s.startswith("{")]
    assert len(rows) == 1
    d = rows[0]
    assert KEYS <= set(d) and d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["config"]["N"] == 2048


@pytest.mark.parametrize("workload,extra", [("batch", ["--count", "6"]), ("serve", [])])
def test_reference_arm_other_workloads(workload, extra):
    """The reference arm on a batch (whole trees of the forest) and on the
    serving topologies: one line, the oracle's sample named in it."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    line = _run(["bench.py", "--impl", "reference", "--workload", workload, *extra, "--steps", "1", "--warmup",
                 "1", "--ref-seconds", "1"], env=env)
    d = [json.loads(s) for s in line.splitlines() if s.startswith("{")][-1]
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["sample_nodes"] > 0
    assert "tree(s)" in d["cpu_baseline"]["sample"]


def test_reference_arm_two_rank_gloo():
    """torchrun with two CPU ranks: rank 0 alone prints; the job exits 0."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    line = _run(["-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2", "--master-addr=127.0.0.1",
                 "--master-port=29517", "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                 "--warmup", "1", "--total", "1024", "--ref-seconds", "1"], env=env)
    rows = [json.loads(s) for s in line.splitlines() if s.startswith("{")]
    assert len(rows) == 1 and rows[0]["n_gpus"] == 2


def _fake_launches(parent, seed=0, tail_from=None):
    """The launch sequence run_factor issues for this plan (kinds, operation
    counts in the order of the rounds; the contraction and expansion of rounds
    >= tail_from in one level-asynchronous launch, the T composites of every
    round as separate launches), with made-up durations."""
    h = tlqr.tlqr_plan_create(parent)
    try:
        rnd, op = tlqr.tlqr_plan_schedule(h, len(parent))
    finally:
        tlqr.tlqr_plan_destroy(h)
    R = int(rnd.max())
    nr = np.bincount(rnd[op == tlqr.TLQR_OP_RAKE], minlength=R + 1)
    nc = np.bincount(rnd[op == tlqr.TLQR_OP_COMPRESS], minlength=R + 1)
    rng = np.random.default_rng(seed)
    head = R if tail_from is None else tail_from - 1
    L = []
    for r in range(1, head + 1):
        if nr[r]:
            L.append(("rake", int(nr[r]), float(rng.uniform(0.01, 0.02))))
            L.append(("absorb", max(1, int(nr[r]) // 2), 0.005))
        if nc[r]:
            L.append(("compress", int(nc[r]), float(rng.uniform(0.01, 0.03))))
    if head < R:
        L.append(("factor_tail", 1, 0.05))
    for r in range(head, 0, -1):
        if nc[r]:
            L.append(("expand", int(nc[r]), 0.01))
    for r in range(1, R + 1):
        if nc[r]:
            L.append(("compose_T", int(nc[r]), 0.004))
    return L, rnd, op, nr, nc


@pytest.mark.parametrize("tree", ["long_trunk", "recursive", "chain"])
def test_round_roofline_bookkeeping(tree):
    rng = inputs.rng_for(90)
    parent = {"long_trunk": lambda: inputs.long_trunk_tree(rng, trunk=300, total=3000),
              "recursive": lambda: inputs.random_recursive(2000, rng),
              "chain": lambda: inputs.chain(500)}[tree]()
    L, rnd, op, nr, nc = _fake_launches(parent)
    n, m = 12, 4
    rows = bench.round_roofline(L, rnd, op, n, m, 4, 6500.0, 76.9, tlqr.TLQR_OP_RAKE, tlqr.TLQR_OP_COMPRESS)
    assert [r["round"] for r in rows] == list(range(1, int(rnd.max()) + 1))
    assert abs(sum(r["ms"] for r in rows) - sum(x[2] for x in L)) < 1e-12
    fr, br = bench.per_unit("rake", n, m, 4)
    fc, bc = bench.per_unit("compress", n, m, 4)
    for r in rows:
        k = r["round"]
        assert r["rakes"] == nr[k] and r["compresses"] == nc[k]
        assert r["flops"] >= fr * nr[k] + fc * nc[k]
        assert r["roof_ms"] > 0 and r["bound"] in ("hbm", "alu")
    # a launch list that disagrees with the plan is refused
    bad = [(k, u + 1, t) if k == "compress" else (k, u, t) for k, u, t in L]
    if any(k == "compress" for k, _, _ in L):
        with pytest.raises(RuntimeError):
            bench.round_roofline(bad, rnd, op, n, m, 4, 6500.0, 76.9, tlqr.TLQR_OP_RAKE, tlqr.TLQR_OP_COMPRESS)


def test_round_roofline_with_tail_rounds():
    rng = inputs.rng_for(91)
    parent = inputs.long_trunk_tree(rng, trunk=300, total=3000)
    L, rnd, op, nr, nc = _fake_launches(parent, tail_from=6)
    rows = bench.round_roofline(L, rnd, op, 12, 4, 4, 6500.0, 76.9, tlqr.TLQR_OP_RAKE, tlqr.TLQR_OP_COMPRESS)
    R = int(rnd.max())
    assert [r["round"] for r in rows[:-1]] == [1, 2, 3, 4, 5]
    tail_ms = 0.05 + 0.004 * int((nc[6:] > 0).sum())
    assert rows[-1]["round"] == f"6-{R} (tail)" and abs(rows[-1]["ms"] - tail_ms) < 1e-12
    assert rows[-1]["rakes"] == int(nr[6:].sum()) and rows[-1]["compresses"] == int(nc[6:].sum())
    assert abs(sum(r["ms"] for r in rows) - sum(x[2] for x in L)) < 1e-12


def _max_worker(rank, world, port, out):
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(1.5 + rank, tdist, "cpu")
    finally:
        tdist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    """The job time of the repo arm is the slowest rank's: every rank of a
    two-rank gloo job gets the larger of the two values; without a process
    group the value is returned as is."""
    import torch.multiprocessing as mp
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_max_worker, args=(r, 2, 29531, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 2.5, 1: 2.5}


def test_committed_autotune_table_gives_valid_options():
    """Every workload of the committed autotuner table maps to options that
    the library accepts (the values the tuner tries), and its best entry is
    the fastest of the candidates it recorded."""
    from paper_2608_01332_b300 import autotune
    table = autotune.load_table()
    assert set(table) >= {"long_trunk", "batch", "spine", "serve"}
    for name, entry in table.items():
        opts = autotune.tuned_options(name)
        assert opts["async_ops"] in (-1, 256, 1024, 4096)
        assert opts["async_solve"] in (-1, 1)
        assert opts["tail_ops"] in (-1, 0, 64, 128, 512)
        assert opts.get("residual", 0) in (0, 1, 2)
        o = tlqr.make_options(entry["n"], entry["m"], tlqr.TLQR_PREC_MIXED, **opts)
        assert o.async_ops == opts["async_ops"]
        ok = [c for c in entry["candidates"] if c["status"] == 0 and c["ms"] > 0]
        best = min(ok, key=lambda c: c["ms"])
        assert all(best[k] == entry["best"][k] for k in ("async_ops", "async_solve", "tail_ops"))


def test_work_model_matches_the_stated_counts():
    """The roofline's algorithmic work per operation: the leading-order dense
    counts (c3, n = 32: rake 26/3 n^3 + n^2 ~ 285 kflop, compression
    50/3 n^3 + n^2 ~ 547 kflop, reconstruction 26/3 n^3, composite 2 n^3) and
    the residual's FP64 bytes per node at c1 (n = 12, m = 4, 10 % of Delta
    blocks nonzero): Q, A (2 f), B, R, the nonzero Delta and 8n + 4m vector
    entries, 3,827.2 bytes."""
    n = 32
    fl, _ = bench.per_unit("rake", n, 8, 4)
    assert abs(fl - (26 / 3 * n ** 3 + n ** 2)) < 1e-6 and 284e3 < fl < 286e3
    fl, _ = bench.per_unit("compress", n, 8, 4)
    assert 546e3 < fl < 548e3
    assert bench.per_unit("expand", n, 8, 4)[0] == pytest.approx(26 / 3 * n ** 3)
    assert bench.per_unit("compose_T", n, 8, 4)[0] == 2 * n ** 3
    _, by = bench.per_unit("residual", 12, 4, 8, 0.1)
    assert by == pytest.approx(3827.2)
    # packed symmetric traffic: a rake reads A (f) and U, C, P and writes its contribution (4 s words)
    _, by = bench.per_unit("rake", 12, 4, 4)
    assert by == (144 + 4 * 78) * 4
