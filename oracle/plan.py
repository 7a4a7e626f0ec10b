"""ORACLE -- test infrastructure only.

The topology-only contraction schedule of Sec. IV and Sec. X-A, taken
literally and without any attention to speed:

  * a structural round first rakes every nonroot leaf, then compresses a
    maximal set of pairwise nonadjacent unary nonroot nodes, chosen greedily in
    increasing node index: a unary node is selected unless its current parent
    or its current child is already selected (Sec. X-A);
  * rounds repeat until only the root is left.

Dependency levels follow eq. (earliest-level): every initial node or edge
datum has level 0, an operation has level 1 + the largest level of its inputs,
and its output datum inherits that level.  The four primitive operations are
rake, binary combination of sibling contributions, absorption and compression
(Sec. X-B).  Sibling contributions to one parent are combined in increasing
node index order by the readiness-weighted alphabetic reduction of
eq. (readiness-code-data) (Lemma 3), computed here with exact rational
arithmetic.
"""
from __future__ import annotations

from fractions import Fraction


def _children(parent):
    ch = {i: set() for i in range(len(parent))}
    for j, i in enumerate(parent):
        if i >= 0:
            ch[i].add(j)
    return ch


def structural_schedule(parent):
    """Return a list of rounds; each round is dict(rakes=[(j, i)], compresses=[(j, i, k)]).

    parent may hold several roots (a forest); every tree is contracted by the
    same rule in the same rounds.

    (j, i) = raked leaf and its current parent; (j, i, k) = compressed centre,
    its current parent and its current (only) child.  Lists are in increasing j.
    """
    parent = [int(p) for p in parent]
    N = len(parent)
    roots = {i for i in range(N) if parent[i] < 0}
    if not roots:
        raise ValueError("parent array must have a root")
    cur_parent = list(parent)
    ch = _children(parent)
    alive = set(range(N))
    rounds = []
    while len(alive) > len(roots):
        rakes = []
        for j in sorted(alive):
            if j not in roots and not ch[j]:
                rakes.append((j, cur_parent[j]))
        for j, i in rakes:
            ch[i].discard(j)
            alive.discard(j)
        selected = []
        sel = set()
        for j in sorted(alive):
            if j in roots or len(ch[j]) != 1:
                continue
            k = next(iter(ch[j]))
            i = cur_parent[j]
            if i in sel or k in sel:
                continue
            selected.append((j, i, k))
            sel.add(j)
        for j, i, k in selected:
            ch[i].discard(j)
            ch[i].add(k)
            cur_parent[k] = i
            alive.discard(j)
        rounds.append(dict(rakes=rakes, compresses=selected))
        if not rakes and not selected:
            raise RuntimeError("no progress")
    return rounds


def node_ops(parent):
    """Per node: (round index starting at 1, 'R' or 'C'); root -> (0, '-')."""
    out = {}
    for t, rd in enumerate(structural_schedule(parent), start=1):
        for j, _ in rd["rakes"]:
            out[j] = (t, "R")
        for j, _, _ in rd["compresses"]:
            out[j] = (t, "C")
    for i, p in enumerate(parent):
        if p < 0:
            out[i] = (0, "-")
    return out


def _ceil_log2_ratio(num: int, den: int) -> int:
    """Smallest integer d >= 0 with 2^d >= num/den (num >= den > 0)."""
    d = 0
    while (den << d) < num:
        d += 1
    return d


def readiness_reduction(levels):
    """Order-preserving reduction tree of eq. (readiness-code-data) (Lemma 3).

    levels: producer levels l_1..l_k of the sibling contributions, in sibling
    order.  Returns (final_level, n_combinations, depths).
    """
    k = len(levels)
    if k == 1:
        return levels[0], 0, [0]
    w = [2 ** l for l in levels]
    W = sum(w)
    codes = []
    F = Fraction(0)
    for j in range(k):
        pj = Fraction(w[j], W)
        d0 = _ceil_log2_ratio(W, w[j]) + 1          # ceil(log2(1/p_j)) + 1
        mid = F + pj / 2
        r = int(mid * (2 ** d0))                     # first d0 binary digits of the midpoint
        codes.append(format(r, "b").zfill(d0))
        F += pj
    n_comb = 0
    depths = [0] * k

    def build(items, pos, depth):
        nonlocal n_comb
        if len(items) == 1:
            depths[items[0]] = depth
            return levels[items[0]]
        zero = [t for t in items if codes[t][pos] == "0"]
        one = [t for t in items if codes[t][pos] == "1"]
        if not zero or not one:                      # unary trie vertex: contracted
            return build(items, pos + 1, depth)
        n_comb += 1
        return 1 + max(build(zero, pos + 1, depth + 1), build(one, pos + 1, depth + 1))

    final = build(list(range(k)), 0, 0)
    return final, n_comb, depths


def dependency_levels(parent):
    """Number of nonempty dependency levels of the forward elimination graph.

    Returns dict(levels, rounds, n_rake, n_compress, n_combine, n_absorb).
    """
    parent = [int(p) for p in parent]
    N = len(parent)
    lvU = [0] * N          # producer level of node data U_i
    lvE = [0] * N          # producer level of the data of the edge entering i
    max_level = 0
    n_rake = n_comp = n_comb = n_abs = 0
    rounds = structural_schedule(parent)
    for rd in rounds:
        by_parent = {}
        for j, i in rd["rakes"]:
            lv = 1 + max(lvU[j], lvE[j])
            max_level = max(max_level, lv)
            by_parent.setdefault(i, []).append((j, lv))
            n_rake += 1
        for i, lst in by_parent.items():
            lst.sort()
            agg, nc, _ = readiness_reduction([lv for _, lv in lst])
            n_comb += nc
            lvU[i] = 1 + max(lvU[i], agg)
            max_level = max(max_level, agg, lvU[i])
            n_abs += 1
        for j, i, k in rd["compresses"]:
            lv = 1 + max(lvU[j], lvE[j], lvE[k])
            lvE[k] = lv
            max_level = max(max_level, lv)
            n_comp += 1
    return dict(levels=max_level, rounds=len(rounds), n_rake=n_rake, n_compress=n_comp,
                n_combine=n_comb, n_absorb=n_abs)
