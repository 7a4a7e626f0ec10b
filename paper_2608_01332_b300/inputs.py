"""Seeded synthetic inputs for branched dual-regularized LQR problems.

This module only draws random numbers and assembles parent arrays and problem
data in the edge-control normal form of Sec. III-A (eq. (1)); it contains none of
the solver's arithmetic.  Both the CPU oracle and the CUDA path are fed from it.

Conventions (shared by every consumer):
  * ``parent`` is an int32 array of length N with exactly one entry equal to -1
    (the root); a batch of trees is a forest with one -1 per tree.  Edge e=(i,j) is identified with its child j, so every edge
    array is indexed by the child node and the root slot is unused (zeros).
  * Node arrays: Q (N,n,n), q (N,n), c (N,n), Delta (N,n,n) or None.
    Edge arrays (child-indexed): M (N,n,m) or None, R (N,m,m), r (N,m),
    A (N,n,n), B (N,n,m).  All float64, C-contiguous, row-major blocks.
  * Normal distributions are written N(mean, variance).

Workload families follow the synthetic trees of the scaling study (Sec. XI-A:
chain, complete binary, comb, star) and the problem families named for the
benchmark configurations (long-trunk irregular tree, batches of random
recursive trees, a spine-plus-subtree hybrid, driving-style scenario trees).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2608013320


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# Topologies
# --------------------------------------------------------------------------

def chain(N: int) -> np.ndarray:
    p = np.arange(-1, N - 1, dtype=np.int32)
    return p


def star(N: int) -> np.ndarray:
    p = np.zeros(N, dtype=np.int32)
    p[0] = -1
    return p


def balanced(N: int) -> np.ndarray:
    """Complete binary tree in heap order, parent[i] = (i-1)//2."""
    p = (np.arange(N, dtype=np.int64) - 1) // 2
    p[0] = -1
    return p.astype(np.int32)


def comb(N: int) -> np.ndarray:
    """Trunk with one side leaf hanging off every trunk node.

    Node 0 is the root; trunk nodes are the even labels, side leaves the odd
    labels (each odd k hangs off k-1).  This is one reading of a topology that
    "alternates a trunk with side leaves" (Sec. X-B, Tab. I).
    """
    p = np.empty(N, dtype=np.int32)
    p[0] = -1
    for k in range(1, N):
        if k % 2 == 1:
            p[k] = k - 1          # side leaf of trunk node k-1
        else:
            p[k] = k - 2          # trunk continues
    return p


def random_recursive(N: int, rng: np.random.Generator) -> np.ndarray:
    """Node k attaches to a uniformly chosen earlier node."""
    p = np.empty(N, dtype=np.int32)
    p[0] = -1
    if N > 1:
        k = np.arange(1, N)
        p[1:] = np.floor(rng.random(N - 1) * k).astype(np.int32)
    return p


def tightness_tree(k: int) -> np.ndarray:
    """Unary root above a full binary tree with k leaves, one extra child per leaf.

    Sec. X-A, Lemma 2 (tightness): 3k nodes, one round removes exactly one third.
    k must be a power of two.
    """
    assert k >= 1 and (k & (k - 1)) == 0
    parent = [-1]
    # full binary tree with k leaves has 2k-1 nodes; place it below node 0
    nb = 2 * k - 1
    base = 1
    for t in range(nb):
        parent.append(0 if t == 0 else base + (t - 1) // 2)
    leaves = [base + t for t in range(k - 1, nb)]
    for leaf in leaves:
        parent.append(leaf)
    return np.asarray(parent, dtype=np.int32)


def permute_labels(parent: np.ndarray, rng: np.random.Generator):
    """Relabel nodes by a random permutation (destroys topological order).

    Returns (new_parent, perm) with new label perm[old] for every old label.
    """
    N = len(parent)
    perm = rng.permutation(N).astype(np.int32)
    newp = np.empty(N, dtype=np.int32)
    for old in range(N):
        po = parent[old]
        newp[perm[old]] = -1 if po < 0 else perm[po]
    return newp, perm


def permute_data(data: dict, perm: np.ndarray) -> dict:
    """Move node/edge arrays to the new labels of ``permute_labels``."""
    out = {}
    for k, v in data.items():
        if v is None or not isinstance(v, np.ndarray):
            out[k] = v
            continue
        w = np.empty_like(v)
        w[perm] = v
        out[k] = w
    return out


def long_trunk_tree(rng: np.random.Generator, trunk: int = 4096, total: int = 65536,
                    p_branch: float = 0.05, p_prune: float = 0.02) -> np.ndarray:
    """Long-trunk irregular tree.

    A trunk of ``trunk`` nodes (root 0).  Every trunk node spawns, with
    probability ``p_branch``, a side branch point carrying U{2,3,4} children.
    Every branch child starts a path; a path node is pruned (gets no
    continuation) with probability ``p_prune`` per level, and otherwise carries
    one continuation child, and it also spawns, with probability ``p_branch``,
    a further branch point of U{2,3,4} children.  Branch nodes are grown in
    breadth-first order until the tree holds exactly ``total`` nodes.
    """
    parent = list(range(-1, trunk - 1))
    frontier = []
    for t in range(trunk):
        if rng.random() < p_branch:
            for _ in range(int(rng.integers(2, 5))):
                frontier.append(t)
    n_nodes = trunk
    head = 0
    # each frontier entry is the parent of a node still to be created
    while n_nodes < total:
        if head >= len(frontier):
            # process died out: reseed a branch at a random trunk node
            t = int(rng.integers(0, trunk))
            for _ in range(int(rng.integers(2, 5))):
                frontier.append(t)
            continue
        par = frontier[head]
        head += 1
        me = n_nodes
        parent.append(par)
        n_nodes += 1
        if rng.random() >= p_prune:
            frontier.append(me)
        if rng.random() < p_branch:
            for _ in range(int(rng.integers(2, 5))):
                frontier.append(me)
    return np.asarray(parent, dtype=np.int32)


def spine_hybrid_tree(rng: np.random.Generator, N: int = 1 << 20, spine: int = 1 << 16) -> np.ndarray:
    """Caterpillar-plus-random-recursive hybrid: a spine with random recursive subtrees.

    The N - spine extra nodes are spread over the spine nodes by a uniform
    multinomial; the extras of each spine node form a random recursive tree
    rooted at that spine node.  Labels: spine 0..spine-1, then each subtree's
    nodes in creation order.
    """
    counts = rng.multinomial(N - spine, np.full(spine, 1.0 / spine))
    parent = np.empty(N, dtype=np.int32)
    parent[:spine] = np.arange(-1, spine - 1, dtype=np.int32)
    pos = spine
    u = rng.random(N - spine)
    upos = 0
    for s in range(spine):
        cnt = int(counts[s])
        if cnt == 0:
            continue
        # subtree local labels 0 (= spine node s) .. cnt; node k>=1 attaches to U{0..k-1}
        k = np.arange(1, cnt + 1)
        loc = np.floor(u[upos:upos + cnt] * k).astype(np.int64)
        upos += cnt
        glob = np.where(loc == 0, s, pos + loc - 1)
        parent[pos:pos + cnt] = glob
        pos += cnt
    return parent


def driving_tree(rng: np.random.Generator, N_target: int) -> np.ndarray:
    """Irregular driving-style scenario tree of about N_target nodes.

    Base shape: a root path, then 1-3 split depths chosen at random, where each
    live path branches into 2-5 children, and every branch ends at its own
    terminal depth drawn from 20..80.  Time is then refined: all split and
    terminal depths are scaled by one integer factor until N is within 2 % of
    the target (or the smallest factor that exceeds it).
    """
    n_splits = int(rng.integers(1, 4))
    split_depths = sorted(int(d) for d in rng.choice(np.arange(2, 20), size=n_splits, replace=False))
    fanouts = [int(rng.integers(2, 6)) for _ in range(n_splits)]
    n_leaves = int(np.prod(fanouts))
    term = [int(rng.integers(20, 81)) for _ in range(n_leaves)]

    def build(scale: int) -> np.ndarray:
        parent = [-1]
        # live paths: (node id, leaf-index range lo, hi)
        live = [(0, 0, n_leaves)]
        depth = 0
        si = 0
        maxd = max(term) * scale
        while live and depth < maxd:
            depth += 1
            nxt = []
            split_now = si < n_splits and depth == split_depths[si] * scale
            for node, lo, hi in live:
                if split_now:
                    f = fanouts[si]
                    w = (hi - lo) // f
                    for b in range(f):
                        blo = lo + b * w
                        parent.append(node)
                        nxt.append((len(parent) - 1, blo, blo + w))
                else:
                    if depth > term[lo] * scale and hi - lo == 1:
                        continue
                    if hi - lo == 1 or depth <= max(term[lo:hi]) * scale:
                        parent.append(node)
                        nxt.append((len(parent) - 1, lo, hi))
            if split_now:
                si += 1
            live = nxt
        return np.asarray(parent, dtype=np.int32)

    scale = 1
    p = build(scale)
    while len(p) < 0.98 * N_target:
        scale += 1
        p = build(scale)
    return p


# --------------------------------------------------------------------------
# Problem data
# --------------------------------------------------------------------------

def haar_orthogonal(rng: np.random.Generator, count: int, n: int) -> np.ndarray:
    g = rng.standard_normal((count, n, n))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diagonal(r, axis1=1, axis2=2))
    d[d == 0] = 1.0
    return q * d[:, None, :]


def children_lists(parent: np.ndarray):
    ch = [[] for _ in range(len(parent))]
    for j, i in enumerate(parent):
        if i >= 0:
            ch[i].append(j)
    return ch


def problem_data(parent: np.ndarray, n: int, m: int, rng: np.random.Generator, *,
                 M_scale: float = 0.0, delta: str | None = None, delta_value: float = 1e-6,
                 delta_fraction: float = 0.1, kappa_R: float | None = None,
                 A_scale: float = 0.95) -> dict:
    """Data of the benchmark family.

    A = 0.95 Q_orth (Haar), B ~ N(0, 1/n), c ~ N(0, 0.1), Q = G G^T + 0.1 I with
    G ~ N(0,1), R = I + H H^T with H ~ N(0,1) (or U diag(logspace(0,log10 kappa))U^T
    when ``kappa_R`` is given), q, r ~ N(0,1).  M = 0 unless ``M_scale`` > 0, in
    which case M ~ N(0, M_scale^2) and every Q_i gets + sum_children M M^T, which
    keeps the local convexity condition of Def. 1 because R >= I.

    ``delta``: None (all zero), "subset" (delta_value*I on a seeded
    ``delta_fraction`` of nonroot nodes), "all" (delta_value*I everywhere) or
    "random" (a random PSD block of scale delta_value on every node).
    """
    N = len(parent)
    parent = np.asarray(parent, dtype=np.int32)
    nonroot = parent >= 0
    A = np.zeros((N, n, n))
    A[nonroot] = A_scale * haar_orthogonal(rng, int(nonroot.sum()), n)
    B = np.zeros((N, n, m))
    B[nonroot] = rng.standard_normal((int(nonroot.sum()), n, m)) * math.sqrt(1.0 / n)
    c = rng.standard_normal((N, n)) * math.sqrt(0.1)
    G = rng.standard_normal((N, n, n))
    Q = G @ G.transpose(0, 2, 1) + 0.1 * np.eye(n)
    R = np.zeros((N, m, m))
    if kappa_R is None:
        H = rng.standard_normal((int(nonroot.sum()), m, m))
        R[nonroot] = np.eye(m) + H @ H.transpose(0, 2, 1)
    else:
        U = haar_orthogonal(rng, int(nonroot.sum()), m)
        ev = np.logspace(0.0, math.log10(kappa_R), m)
        R[nonroot] = (U * ev[None, None, :]) @ U.transpose(0, 2, 1)
    q = rng.standard_normal((N, n))
    r = np.zeros((N, m))
    r[nonroot] = rng.standard_normal((int(nonroot.sum()), m))
    M = None
    if M_scale > 0:
        M = np.zeros((N, n, m))
        M[nonroot] = rng.standard_normal((int(nonroot.sum()), n, m)) * M_scale
        MMt = M @ M.transpose(0, 2, 1)
        np.add.at(Q, parent[nonroot], MMt[nonroot])
    Delta = None
    if delta is not None:
        Delta = np.zeros((N, n, n))
        if delta == "subset":
            idx = np.nonzero(nonroot)[0]
            k = max(1, int(round(delta_fraction * len(idx)))) if len(idx) else 0
            pick = rng.choice(idx, size=k, replace=False) if k else np.zeros(0, dtype=int)
            Delta[pick] = delta_value * np.eye(n)
        elif delta == "all":
            Delta[:] = delta_value * np.eye(n)
        elif delta == "random":
            D = rng.standard_normal((N, n, n))
            Delta = delta_value * (D @ D.transpose(0, 2, 1)) / n
        else:
            raise ValueError(delta)
    return dict(Q=np.ascontiguousarray(Q), q=q, M=M, R=R, r=r, A=A, B=B, c=c, Delta=Delta)


def rhs_data(parent: np.ndarray, n: int, m: int, rng: np.random.Generator) -> dict:
    """A fresh right-hand side (q, r, c) for factor-reuse solves."""
    N = len(parent)
    r = rng.standard_normal((N, m))
    r[np.asarray(parent) < 0] = 0.0
    return dict(q=rng.standard_normal((N, n)), r=r,
                c=rng.standard_normal((N, n)) * math.sqrt(0.1))


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    parent: np.ndarray
    n: int
    m: int
    data: dict
    info: dict = field(default_factory=dict)


def binary_depth6(seed: int = BASE_SEED + 0) -> Workload:
    """Complete binary scenario tree of depth 6 (N=127), n=4, m=2, Delta=0."""
    rng = rng_for(seed)
    parent = balanced(127)
    data = problem_data(parent, 4, 2, rng)
    return Workload("binary_depth6_N127_n4_m2", parent, 4, 2, data)


def long_trunk(seed: int = BASE_SEED + 1, total: int = 65536, n: int = 12, m: int = 4) -> Workload:
    """Long-trunk irregular tree (trunk 4096, N=65,536), n=12, m=4,
    Delta = 1e-6 I on a seeded 10 % of nonroot nodes."""
    rng = rng_for(seed)
    parent = long_trunk_tree(rng, trunk=min(4096, total), total=total)
    data = problem_data(parent, n, m, rng, delta="subset", delta_value=1e-6, delta_fraction=0.1)
    return Workload(f"long_trunk_N{total}_n{n}_m{m}", parent, n, m, data)


def recursive_batch_sizes(rng: np.random.Generator, count: int = 1024, lo: int = 64, hi: int = 16384):
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def spine_hybrid(seed: int = BASE_SEED + 3, N: int = 1 << 20, spine: int = 1 << 16,
                 n: int = 32, m: int = 8, kappa_R: float = 1e2) -> Workload:
    rng = rng_for(seed)
    parent = spine_hybrid_tree(rng, N=N, spine=spine)
    data = problem_data(parent, n, m, rng, kappa_R=kappa_R)
    return Workload(f"spine_hybrid_N{N}_n{n}_m{m}_kR{kappa_R:g}", parent, n, m, data)


def forest(parents, rng: np.random.Generator | None = None):
    """Concatenate trees into one forest parent array (labels offset tree by
    tree; optionally a random relabelling of the whole forest).  Returns
    (parent, offsets) with offsets[t] = first label of tree t before relabelling."""
    offs, out, base = [], [], 0
    for p in parents:
        p = np.asarray(p, dtype=np.int64)
        offs.append(base)
        out.append(np.where(p < 0, -1, p + base))
        base += len(p)
    par = np.concatenate(out).astype(np.int32)
    return par, np.asarray(offs)


def concat_data(datas: list) -> dict:
    """Concatenate per-tree problem data in forest order."""
    out = {}
    for k in datas[0]:
        if datas[0][k] is None:
            out[k] = None
        else:
            out[k] = np.ascontiguousarray(np.concatenate([d[k] for d in datas]))
    return out


def recursive_batch(seed: int = BASE_SEED + 2, count: int = 1024, n: int = 16, m: int = 4,
                    lo: int = 64, hi: int = 16384) -> Workload:
    """Batch of random recursive trees (node k attaches to a uniform earlier
    node), sizes log-uniform in [lo, hi], solved together as one forest."""
    rng = rng_for(seed)
    sizes = recursive_batch_sizes(rng, count, lo, hi)
    parents = [random_recursive(int(N), rng) for N in sizes]
    par, offs = forest(parents)
    data = problem_data(par, n, m, rng)
    return Workload(f"recursive_batch_{count}x_n{n}_m{m}", par, n, m, data,
                    info=dict(sizes=sizes, offsets=offs))


# --------------------------------------------------------------------------
# Device-side generation for the largest workloads
# --------------------------------------------------------------------------

def problem_data_device(parent: np.ndarray, n: int, m: int, seed: int, device, *,
                        kappa_R: float | None = None, delta_fraction: float = 0.0,
                        delta_value: float = 1e-6, A_scale: float = 0.95, chunk: int = 1 << 16) -> dict:
    """The distributions of ``problem_data`` (M = 0) drawn on a CUDA device with
    torch's seeded generator, chunk by chunk -- for workloads of 10^6 nodes and
    n = 16..32 whose host generation would take minutes and tens of GB of host
    memory.  Returns float64 device tensors keyed like ``problem_data``.  The
    values are a deterministic function of (parent, n, m, seed, device type),
    not the same numbers ``problem_data`` draws."""
    import torch

    N = len(parent)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = dict(dtype=torch.float64, device=device)
    nonroot = torch.from_numpy(np.asarray(parent) >= 0).to(device)
    A = torch.empty((N, n, n), **f64)
    B = torch.empty((N, n, m), **f64)
    Q = torch.empty((N, n, n), **f64)
    R = torch.empty((N, m, m), **f64)
    eye_n = torch.eye(n, **f64)
    eye_m = torch.eye(m, **f64)
    ev = None
    if kappa_R is not None:
        ev = torch.logspace(0.0, math.log10(kappa_R), m, **f64)

    def haar(cnt, k):
        q, r = torch.linalg.qr(torch.randn((cnt, k, k), generator=g, **f64))
        d = torch.sign(torch.diagonal(r, dim1=1, dim2=2))
        d[d == 0] = 1.0
        return q * d[:, None, :]

    for b in range(0, N, chunk):
        e = min(N, b + chunk)
        cnt = e - b
        nr = nonroot[b:e]
        A[b:e] = torch.where(nr[:, None, None], A_scale * haar(cnt, n), 0.0)
        B[b:e] = torch.where(nr[:, None, None], torch.randn((cnt, n, m), generator=g, **f64) / math.sqrt(n), 0.0)
        G = torch.randn((cnt, n, n), generator=g, **f64)
        Q[b:e] = G @ G.transpose(1, 2) + 0.1 * eye_n
        if ev is None:
            H = torch.randn((cnt, m, m), generator=g, **f64)
            Rc = eye_m + H @ H.transpose(1, 2)
        else:
            U = haar(cnt, m)
            Rc = (U * ev[None, None, :]) @ U.transpose(1, 2)
        R[b:e] = torch.where(nr[:, None, None], Rc, 0.0)
    c = torch.randn((N, n), generator=g, **f64) * math.sqrt(0.1)
    q = torch.randn((N, n), generator=g, **f64)
    r = torch.randn((N, m), generator=g, **f64) * nonroot[:, None]
    Delta = None
    if delta_fraction > 0:
        pick = (torch.rand((N,), generator=g, **f64) < delta_fraction) & nonroot
        Delta = torch.zeros((N, n, n), **f64)
        Delta[pick] = delta_value * eye_n
    return dict(Q=Q, q=q, M=None, R=R, r=r, A=A, B=B, c=c, Delta=Delta)


def spine_hybrid_device(device, seed: int = BASE_SEED + 3, N: int = 1 << 20, spine: int = 1 << 16,
                        n: int = 32, m: int = 8, kappa_R: float = 1e2) -> Workload:
    """The spine-plus-random-recursive-subtrees tree (N = 2^20, n = 32, m = 8)
    with its data drawn on the device (R = U diag(logspace(0, log10 kappa, m)) U^T)."""
    rng = rng_for(seed)
    parent = spine_hybrid_tree(rng, N=N, spine=spine)
    data = problem_data_device(parent, n, m, seed, device, kappa_R=kappa_R)
    return Workload(f"spine_hybrid_N{N}_n{n}_m{m}_kR{kappa_R:g}", parent, n, m, data)


def recursive_batch_device(device, seed: int = BASE_SEED + 2, count: int = 1024, n: int = 16, m: int = 4,
                           lo: int = 64, hi: int = 16384) -> Workload:
    """``recursive_batch`` (1,024 random recursive trees, sizes log-uniform in
    [64, 16384], n = 16, m = 4) with its data drawn on the device."""
    rng = rng_for(seed)
    sizes = recursive_batch_sizes(rng, count, lo, hi)
    parents = [random_recursive(int(k), rng) for k in sizes]
    par, offs = forest(parents)
    data = problem_data_device(par, n, m, seed, device)
    return Workload(f"recursive_batch_{count}x_n{n}_m{m}", par, n, m, data,
                    info=dict(sizes=sizes, offsets=offs))
