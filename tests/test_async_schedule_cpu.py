"""CPU checks of the level-asynchronous factorisation tail's operation list
(the host logic behind the persistent kernel; no GPU needed).

The list is executed symbolically: every datum (node data U_i, edge slot E_j,
Riccati matrix P_j, rake contributions) carries a version, and every operation
records the versions it reads.  The reference is the round-by-round order of
Sec. X-A (rakes, absorptions, compressions per round; expansions in reverse
round order).  The list is then run in orders that respect only its own (flag, target) dependencies -- the
freedom the GPU has; one adversarial (latest ready position first), two
random -- and each operation
must read exactly the versions it reads in the reference, every operation must
run (no deadlock), and the warp layout must hold: one kind per warp, no
dependency inside a warp, every dependency on an earlier position.
"""
from collections import defaultdict

import numpy as np
import pytest

from oracle import plan as oplan
from paper_2608_01332_b300 import inputs, tlqr

RAKE, ABSORB, COMPRESS, EXPAND = 0, 1, 2, 3
COMPOSE_S, EXPAND_C, EXPAND_R = 4, 5, 6           # state pass


def _reference(parent, r0):
    rounds = oplan.structural_schedule(parent)
    R = len(rounds)
    verU, verE = defaultdict(int), defaultdict(int)
    reads = {}
    comp_child = {}
    for r in range(r0, R):
        rd = rounds[r]
        by_parent = defaultdict(list)
        for j, i in rd["rakes"]:
            reads[(RAKE, j)] = (verU[j], verE[j])
            by_parent[i].append(j)
        for i, js in by_parent.items():
            reads[(ABSORB, i, r + 1)] = (verU[i], tuple(sorted(js)))
            verU[i] += 1
        for j, i, k in rd["compresses"]:
            reads[(COMPRESS, j)] = (verU[j], verE[j], verE[k])
            verE[k] += 1
            verE[j] += 1
            comp_child[j] = k
    verP = {}
    for r in range(R - 1, r0 - 1, -1):
        for j, i, k in rounds[r]["compresses"]:
            reads[(EXPAND, j)] = (verE[j], verP.get(k, ("U", verU[k])))
            verP[j] = ("X", j)
    return reads, comp_child, rounds


def _hazards(parent, r0):
    """Reference order: for every operation, the operations whose results it
    reads (read after write) and the earlier readers of every datum it
    overwrites (write after read).  Keys as in _reference."""
    rounds = oplan.structural_schedule(parent)
    R = len(rounds)
    writer = {}                         # datum -> key of its last writer
    readers = defaultdict(list)         # datum -> keys that read its current value
    need = defaultdict(set)

    def read(key, d):
        if d in writer:
            need[key].add(writer[d])
        readers[d].append(key)

    def write(key, d):
        need[key].update(r for r in readers[d] if r != key)
        readers[d] = []
        writer[d] = key

    for r in range(r0, R):
        rd = rounds[r]
        by_parent = defaultdict(list)
        for j, i in rd["rakes"]:
            key = (RAKE, j)
            read(key, ("U", j)); read(key, ("E", j)); write(key, ("c", j))
            by_parent[i].append(j)
        for i, js in by_parent.items():
            key = (ABSORB, i, r + 1)
            for j in js:
                read(key, ("c", j))
            read(key, ("U", i)); write(key, ("U", i))
        for j, i, k in rd["compresses"]:
            key = (COMPRESS, j)
            read(key, ("U", j)); read(key, ("E", j)); read(key, ("E", k))
            write(key, ("E", k)); write(key, ("E", j))
    for r in range(R - 1, r0 - 1, -1):
        for j, i, k in rounds[r]["compresses"]:
            key = (EXPAND, j)
            read(key, ("E", j)); read(key, ("U", k)); write(key, ("U", j))
    return need


def _state_hazards(parent):
    """The state pass in the reference order: offset compositions b_k <- Tr_j
    b_j + b_k in forward round order, then per round in reverse order the
    state expansions x_j = T_j x_i + b_j of the compressed centres and then of
    the raked leaves; b and a root's x exist before the pass."""
    rounds = oplan.structural_schedule(parent)
    writer, readers, need = {}, defaultdict(list), defaultdict(set)

    def read(key, d):
        if d in writer:
            need[key].add(writer[d])
        readers[d].append(key)

    def write(key, d):
        need[key].update(r for r in readers[d] if r != key)
        readers[d] = []
        writer[d] = key

    for rd in rounds:
        for j, i, k in rd["compresses"]:
            key = (COMPOSE_S, j)
            read(key, ("b", j)); read(key, ("b", k)); write(key, ("b", k))
    for rd in reversed(rounds):
        for j, i, k in rd["compresses"]:
            key = (EXPAND_C, j)
            read(key, ("b", j)); read(key, ("x", i)); write(key, ("x", j))
        for j, i in rd["rakes"]:
            key = (EXPAND_R, j)
            read(key, ("b", j)); read(key, ("x", i)); write(key, ("x", j))
    return need


def _check_hazards_implied(parent, s, need=None):
    """Every hazard of the reference order is an ancestor in the list's DAG."""
    P = s["n_ops"]
    kind, node, rnd = s["kind"], s["node"], s["round"]
    deps = s["dep_flag"]
    key_of, pos_of = {}, {}
    seg_rakes = defaultdict(list)
    for p in range(P):
        if node[p] < 0:
            continue
        k = int(kind[p])
        key = (k, int(node[p]), int(rnd[p])) if k == ABSORB else (k, int(node[p]))
        key_of[p], pos_of[key] = key, p
        if int(s["signal"][p]) >= 0:
            seg_rakes[int(s["signal"][p])].append(p)
    anc = {}
    for p in sorted(key_of):                       # dependencies sit at earlier positions
        a = 0
        for f in deps[p]:
            f = int(f)
            if f < 0:
                continue
            preds = [f] if f < P else seg_rakes[f]
            for q in preds:
                a |= anc[q] | (1 << q)
        anc[p] = a
    if need is None:
        need = _hazards(parent, s["r0"])
    assert sorted(pos_of) == sorted(set(need) | {k for k in pos_of})
    for key, want in need.items():
        p = pos_of[key]
        for w in want:
            assert (anc[p] >> pos_of[w]) & 1, f"{key} may run before {w}"


def _simulate(parent, s, reads, comp_child, rounds, rng, ops_per_warp, latest_first=False):
    P = s["n_ops"]
    kind, node, rnd = s["kind"], s["node"], s["round"]
    deps, tgts, sig = s["dep_flag"], s["dep_target"], s["signal"]
    # warp layout
    for b in range(0, P, ops_per_warp):
        assert len(set(kind[b:b + ops_per_warp].tolist())) == 1
        assert node[b] >= 0, "a warp's first slot must hold a real operation (padding repeats it)"
        for p in range(b, b + ops_per_warp):
            for f in deps[p]:
                if 0 <= f < P:
                    assert f < b, "dependency inside a warp or on a later position"
    real = [p for p in range(P) if node[p] >= 0]
    # operation multiset = the reference's
    keys = []
    for p in real:
        k = int(kind[p])
        keys.append((k, int(node[p]), int(rnd[p])) if k == ABSORB else (k, int(node[p])))
    assert sorted(keys) == sorted(reads.keys())
    # random executions under the list's own dependencies
    flags = np.zeros(s["n_flags"], dtype=np.int64)
    waiting = defaultdict(list)
    missing = {}
    ready = []
    for p in real:
        need = [(int(f), int(t)) for f, t in zip(deps[p], tgts[p]) if f >= 0]
        missing[p] = len(need)
        for f, t in need:
            waiting[f].append((p, t))
        if not need:
            ready.append(p)
    verU, verE, verP = defaultdict(int), defaultdict(int), {}
    made = set()
    executed = 0
    while ready:
        # latest_first: an adversarial order that runs the latest ready position first, so
        # that an operation made ready too early overtakes its missing producer
        t = int(np.argmax(ready)) if latest_first else int(rng.integers(len(ready)))
        p = ready.pop(t)
        k, v = int(kind[p]), int(node[p])
        if k == RAKE:
            got, key = (verU[v], verE[v]), (RAKE, v)
            made.add(v)
        elif k == ABSORB:
            key = (ABSORB, v, int(rnd[p]))
            js = reads[key][1]
            assert all(j in made for j in js), "absorption before all its rakes"
            got = (verU[v], js)
            verU[v] += 1
        elif k == COMPRESS:
            kk = comp_child[v]
            got, key = (verU[v], verE[v], verE[kk]), (COMPRESS, v)
            verE[kk] += 1
            verE[v] += 1
        else:
            kk = comp_child[v]
            got, key = (verE[v], verP.get(kk, ("U", verU[kk]))), (EXPAND, v)
            verP[v] = ("X", v)
        assert got == reads[key], (key, got, reads[key])
        executed += 1
        for f in [p] + ([int(sig[p])] if sig[p] >= 0 else []):
            flags[f] += 1
            for q, t in waiting[f]:
                if flags[f] == t:
                    missing[q] -= 1
                    if missing[q] == 0:
                        ready.append(q)
    assert executed == len(real), "some operations never became ready (deadlock)"


def _trees():
    rng = inputs.rng_for(77)
    out = [("chain", inputs.chain(300)), ("star", inputs.star(200)), ("balanced", inputs.balanced(255)),
           ("comb", inputs.comb(301)), ("tight", inputs.tightness_tree(32)),
           ("longtrunk", inputs.long_trunk_tree(rng, trunk=200, total=1500)),
           ("driving", inputs.driving_tree(rng, 1200))]
    p, _ = inputs.permute_labels(inputs.random_recursive(1500, rng), rng)
    out.append(("recursive", p))
    f, _ = inputs.forest([inputs.random_recursive(int(k), rng) for k in (40, 300, 3, 700)])
    out.append(("forest", f))
    return out


@pytest.mark.parametrize("tree", _trees(), ids=lambda t: t[0])
@pytest.mark.parametrize("n", [4, 12, 32])
@pytest.mark.parametrize("async_ops", [1 << 30, 64])
def test_async_list_reads_what_the_rounds_read(tree, n, async_ops):
    name, parent = tree
    forest = (np.asarray(parent) < 0).sum() > 1
    plan = tlqr.tlqr_plan_create_forest(parent) if forest else tlqr.tlqr_plan_create(parent)
    try:
        s = tlqr.tlqr_async_schedule(plan, n, async_ops)
    finally:
        tlqr.tlqr_plan_destroy(plan)
    reads, comp_child, rounds = _reference(parent, s["r0"])
    if async_ops == 1 << 30:
        assert s["r0"] == 0
    else:
        assert all(len(rd["rakes"]) + len(rd["compresses"]) <= async_ops for rd in rounds[s["r0"]:])
    G = 4 if n <= 4 else 8 if n <= 8 else 16 if n <= 16 else 32
    rng = inputs.rng_for(5 + n)
    _check_hazards_implied(parent, s)
    _simulate(parent, s, reads, comp_child, rounds, rng, 32 // G, latest_first=True)
    for _ in range(2):
        _simulate(parent, s, reads, comp_child, rounds, rng, 32 // G)


def test_async_levels_at_most_twice_the_rounds():
    """Each structural round adds at most a rake, an absorption and a
    compression to a dependency chain, and the expansions at most one level per
    round: the list's depth is bounded by 4 R (it is usually far below)."""
    rng = inputs.rng_for(78)
    p = inputs.long_trunk_tree(rng, trunk=400, total=4000)
    plan = tlqr.tlqr_plan_create(p)
    try:
        s = tlqr.tlqr_async_schedule(plan, 12, 1 << 30)
        R = tlqr.tlqr_plan_stats(plan)["rounds"]
    finally:
        tlqr.tlqr_plan_destroy(plan)
    assert 0 < s["levels"] <= 4 * R


@pytest.mark.parametrize("tree", _trees(), ids=lambda t: t[0])
@pytest.mark.parametrize("n", [4, 12, 32])
def test_state_pass_list(tree, n):
    """The state pass's list: every operation of the reference once, every
    hazard implied by the DAG, one kind per warp, dependencies on earlier
    warps only, and an adversarial execution that never stalls."""
    name, parent = tree
    forest = (np.asarray(parent) < 0).sum() > 1
    plan = tlqr.tlqr_plan_create_forest(parent) if forest else tlqr.tlqr_plan_create(parent)
    try:
        s = tlqr.tlqr_async_schedule(plan, n, which=2)
        a = tlqr.tlqr_async_schedule(plan, n, which=1)
        f = tlqr.tlqr_async_schedule(plan, n, async_ops=1 << 30, which=0)
    finally:
        tlqr.tlqr_plan_destroy(plan)
    # the affine pass runs the factorisation's list over every round
    for k in ("kind", "node", "round", "dep_flag", "dep_target", "signal"):
        np.testing.assert_array_equal(a[k], f[k])
    need = _state_hazards(parent)
    P = s["n_ops"]
    G = 4 if n <= 4 else 8 if n <= 8 else 16 if n <= 16 else 32
    W = 32 // G
    keys = sorted((int(s["kind"][p]), int(s["node"][p])) for p in range(P) if s["node"][p] >= 0)
    assert keys == sorted(need)
    for b in range(0, P, W):
        assert len(set(s["kind"][b:b + W].tolist())) == 1 and s["node"][b] >= 0
        for p in range(b, b + W):
            assert all(f < b for f in s["dep_flag"][p] if f >= 0)
    _check_hazards_implied(parent, s, need)
    # execute latest-ready-first under the list's own flags: everything runs
    done = np.zeros(P, dtype=bool)
    ready = [p for p in range(P) if s["node"][p] >= 0 and all(f < 0 for f in s["dep_flag"][p])]
    waiting = defaultdict(list)
    missing = {}
    for p in range(P):
        if s["node"][p] < 0:
            continue
        fl = [int(f) for f in s["dep_flag"][p] if f >= 0]
        missing[p] = len(fl)
        for f in fl:
            waiting[f].append(p)
    count = 0
    while ready:
        p = ready.pop(int(np.argmax(ready)))
        done[p] = True
        count += 1
        for q in waiting[p]:
            missing[q] -= 1
            if missing[q] == 0:
                ready.append(q)
    assert count == len(missing)
