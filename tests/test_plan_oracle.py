"""Pins of the literal schedule oracle (oracle/plan.py) against what the paper prints
and proves: the Fig. 2 schedules, the star row of Tab. I, Lemma 2 (geometric
progress and its tightness example), Lemma 3 (k-1 combinations, level bound)
and Lemma 4 (dependency-level bound D_N)."""
import math

import numpy as np
import pytest

from oracle import plan
from paper_2608_01332_b300 import inputs
from tests.conftest import read_golden


def fig2_cases():
    lines = read_golden("fig2_schedules.txt")
    out = []
    for t in range(0, len(lines), 3):
        name = lines[t].split()[1]
        parent = [int(v) for v in lines[t + 1].split()[1:]]
        labels = lines[t + 2].split()[1:]
        out.append((name, parent, labels))
    return out


@pytest.mark.parametrize("case", fig2_cases(), ids=lambda c: c[0])
def test_fig2_schedules(case):
    _, parent, labels = case
    ops = plan.node_ops(parent)
    got = ["-" if ops[i][1] == "-" else f"{ops[i][1]}{ops[i][0]}" for i in range(len(parent))]
    assert got == labels


def table1():
    rows = {}
    for ln in read_golden("table1_levels.txt"):
        f = ln.split()
        rows[f[0]] = ([int(v) for v in f[1:6]], f[6] == "yes")
    return rows


def test_table1_star_row():
    vals, pinned = table1()["star"]
    assert pinned
    got = [plan.dependency_levels(inputs.star(N))["levels"] for N in (16, 64, 256, 1024, 4096)]
    assert got == vals


def D_N(N):
    return math.floor(math.log2(2 * N - 1) + math.ceil(math.log(N, 1.5)) * math.log2(36))


def _trees():
    rng = inputs.rng_for(3)
    out = [("chain", inputs.chain(300)), ("star", inputs.star(300)), ("balanced", inputs.balanced(300)),
           ("comb", inputs.comb(300)), ("tight", inputs.tightness_tree(16))]
    for t in range(6):
        N = int(rng.integers(2, 400))
        p = inputs.random_recursive(N, rng)
        p, _ = inputs.permute_labels(p, rng)
        out.append((f"rr{t}", p))
    out.append(("longtrunk", inputs.long_trunk_tree(rng, trunk=200, total=1500)))
    return out


@pytest.mark.parametrize("tree", _trees(), ids=lambda t: t[0])
def test_progress_and_counts(tree):
    """Every nonroot node is removed exactly once (#rake + #compress = N-1,
    Sec. IX-B), each round removes >= ceil(N_r/3) nodes, rounds <=
    ceil(log_{3/2} N) (Lemma 2), levels <= D_N (Lemma 4), and the compress set
    is pairwise nonadjacent."""
    _, parent = tree
    N = len(parent)
    rounds = plan.structural_schedule(parent)
    removed = []
    alive = N
    for rd in rounds:
        k = len(rd["rakes"]) + len(rd["compresses"])
        assert k >= math.ceil(alive / 3)
        centres = {j for j, _, _ in rd["compresses"]}
        for j, i, kk in rd["compresses"]:
            assert i not in centres and kk not in centres
        removed += [j for j, _ in rd["rakes"]] + [j for j, _, _ in rd["compresses"]]
        alive -= k
    assert sorted(removed) == sorted(j for j in range(N) if parent[j] >= 0)
    assert len(rounds) <= math.ceil(math.log(N, 1.5))
    lv = plan.dependency_levels(parent)
    assert lv["levels"] <= D_N(N)
    assert lv["n_rake"] + lv["n_compress"] == N - 1


def test_tightness_example():
    """Lemma 2: unary root over a full binary tree with k leaves, one extra child
    per leaf: 3k nodes; the first round rakes exactly the k extra children and
    compresses nothing (exactly one third removed)."""
    for k in (2, 4, 8, 32):
        p = inputs.tightness_tree(k)
        assert len(p) == 3 * k
        rd = plan.structural_schedule(p)[0]
        assert len(rd["rakes"]) == k and len(rd["compresses"]) == 0


def test_readiness_reduction_lemma3():
    """Lemma 3: k-1 combinations, order preserved, final level <= ceil(log2 W)+1."""
    rng = inputs.rng_for(4)
    for _ in range(200):
        k = int(rng.integers(1, 40))
        lv = [int(v) for v in rng.integers(0, 8, size=k)]
        final, ncomb, depths = plan.readiness_reduction(lv)
        assert ncomb == k - 1
        W = sum(2 ** l for l in lv)
        assert final <= math.ceil(math.log2(W)) + 1
        assert final == max(l + d for l, d in zip(lv, depths))
    # equal weights reduce to a balanced tree: depth ceil(log2 k)
    for k in (2, 3, 5, 8, 15, 16, 17):
        final, _, _ = plan.readiness_reduction([0] * k)
        assert final == math.ceil(math.log2(k))


def test_forest_schedule_is_each_trees_own_schedule():
    """In a forest every tree is contracted by the same rule in the same rounds:
    a tree's (round, operation) labels are those it gets alone."""
    rng = inputs.rng_for(42)
    trees = [inputs.random_recursive(int(rng.integers(1, 200)), rng) for _ in range(6)] + [inputs.chain(50)]
    par, offs = inputs.forest(trees)
    ops = plan.node_ops(par)
    for t, p in enumerate(trees):
        alone = plan.node_ops(p)
        for i in range(len(p)):
            assert ops[offs[t] + i] == alone[i]
