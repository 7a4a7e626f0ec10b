"""Autotune the execution shape of the benchmark workloads and write the table.

    python -m paper_2608_01332_b300.autotune [--out FILE] [--trials K] [--workloads a,b]

For each workload (the seeded synthetic trees of the benchmark: long_trunk,
batch, spine, serve) this calls tlqr_autotune on a B300 in mixed precision
and records the fastest (async_ops, async_solve, tail_ops, residual) with the
timing of every candidate.  bench.py reads the committed table (autotune_table.json next
to this file) and creates its solver with the chosen options.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "autotune_table.json")


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned_options(workload: str, path: str = TABLE) -> dict:
    """Options chosen for a workload: dict(async_ops, async_solve, tail_ops[, residual]), or {}."""
    e = load_table(path).get(workload)
    return {k: int(v) for k, v in e["best"].items()
            if k in ("async_ops", "async_solve", "tail_ops", "residual")} if e else {}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--trials", type=int, default=5)
    ap.add_argument("--workloads", default="long_trunk,batch,spine,serve")
    args = ap.parse_args(argv)
    import torch

    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2608_01332_b300 import inputs, tlqr

    dev = torch.device("cuda", 0)
    table = load_table(args.out)
    for name in args.workloads.split(","):
        if name == "long_trunk":
            w = inputs.long_trunk()
            data = {k: (None if v is None else torch.from_numpy(v).to(dev)) for k, v in w.data.items()}
            forest = False
        elif name == "batch":
            w = inputs.recursive_batch_device(dev)
            data, forest = w.data, True
        elif name == "spine":
            w = inputs.spine_hybrid_device(dev)
            data, forest = w.data, False
        else:                                   # a serving-sized driving tree
            rng = inputs.rng_for(inputs.BASE_SEED + 4)
            p = inputs.driving_tree(rng, 25000)
            data = inputs.problem_data_device(p, 6, 2, inputs.BASE_SEED + 4, dev)
            w = inputs.Workload("driving_N25000_n6_m2", p, 6, 2, data)
            forest = False
        has_delta = data.get("Delta") is not None
        plan = tlqr.tlqr_plan_create_forest(w.parent) if forest else tlqr.tlqr_plan_create(w.parent)
        try:
            base = tlqr.make_options(w.n, w.m, tlqr.TLQR_PREC_MIXED, has_delta=has_delta)
            best, rows = tlqr.tlqr_autotune(plan, base, data, trials=args.trials)
        finally:
            tlqr.tlqr_plan_destroy(plan)
        table[name] = {"workload": w.name, "N": len(w.parent), "n": w.n, "m": w.m, "precision": "mixed",
                       "gpu": torch.cuda.get_device_name(dev),
                       "best": {"async_ops": best.async_ops, "async_solve": best.async_solve,
                                "tail_ops": best.tail_ops, "residual": best.residual},
                       "candidates": rows}
        print(json.dumps({name: table[name]["best"], "ms": min(r["ms"] for r in rows if r["ms"] > 0)}), flush=True)
        del data, w
        torch.cuda.empty_cache()
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1)


if __name__ == "__main__":
    main()
