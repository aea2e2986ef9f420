"""First sampling pass and light coarsening (Sec. 4, Eq. 2; reuse of samples, Sec. 5).

For one slice with m' rows the global cut is coarsened from sparse samples:

1. Rows per cut node (Sec. 4): the number of test pixels of node c grows linearly
   with its intensity and the pixels are uniform inside the slice.  Reading:
       kappa = max(2, rate1 * m'),   x_c = (kappa * C) * (I_c / I_root),
       k_c   = min(max(floor(x_c + 1/2), 2), 64, m')
   in float32 (an integer decided by floating point, taken in the kernel's
   precision).  I_root is the sum of the cut intensities (the cut partitions the
   leaves).  If k_c >= m' the node takes every row; otherwise rows come from the
   Philox draws floor(w * m' / 2^32) with w = word 0 of counter
   (t, c, slice, PASS1), t = 0, 1, ..., keeping the first k_c distinct rows in draw
   order (at most 65536 draws).
2. The entries V_c on those rows are computed (shadow rays).  The slice's mean-pixel
   estimate is S_hat = sum_c mean(V_c) over the cut nodes.
3. Coarsening (Sec. 4): whenever both children a, b of a tree node f are in the
   slice's cut, the pair is tested on zeta_f = zeta_a U zeta_b (the union rule; the
   paper draws fresh rows only for the first level, the union is used throughout so
   that the row count stays proportional to I_f and every sample is reused).  The
   missing entries of V_a and V_b on zeta_f are computed.  With p the child whose
   representative f inherits and q the other:
       eps(f)  = max_{i in zeta_f} | V_q(i) - V_p(i) I_q / I_p |        (Sec. 4)
       cost(f) = eps(f) + cost(q),   cost = 0 on the global cut         (Eq. 2)
   and f replaces a, b when cost(f) < tau * S_hat, with V_f = V_p I_f / I_p (no new
   rays).  In a dark slice (S_hat = 0) the bound is zero and a pair of cost exactly
   zero merges (see merges()).  A pair's decision depends only on its own subtree, so the order in which
   pairs are tested does not change the result; the oracle tests in rounds.
4. Output: the coarsened cut in leaf order (the slice's columns), the observed
   entries of each column and g(c) = max - min of them (Sec. 5, Eq. for g).  A
   column whose parent pair was rejected keeps the entries computed for that test
   on zeta_f; every other column keeps its own zeta_c.  A column with fewer than two
   entries gets the largest g of the slice.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import philox, shading
from .tree import LightTree, node_scale

MAX_ROWS_PER_NODE = 64
MAX_DRAWS = 1 << 16


@dataclasses.dataclass
class Forest:
    """The light tree truncated at the global cut: leaves 0..C-1 are the cut in leaf
    order, internal nodes C..2C-2 are their ancestors (ascending tree node id)."""
    C: int
    node: np.ndarray      # [2C-1] tree node id
    child: np.ndarray     # [2C-1, 2] local ids, -1 on leaves
    parent: np.ndarray    # [2C-1] local id, -1 at the root


def build_forest(tree: LightTree, cut) -> Forest:
    cut = [int(c) for c in cut]
    C = len(cut)
    anc = set()
    for c in cut:
        x = int(tree.parent[c])
        while x >= 0 and x not in anc:
            anc.add(x)
            x = int(tree.parent[x])
    inner = sorted(anc)
    node = np.array(cut + inner, dtype=np.int64)
    local = {int(t): i for i, t in enumerate(node)}
    child = np.full((len(node), 2), -1, dtype=np.int64)
    parent = np.full(len(node), -1, dtype=np.int64)
    for i in range(C, len(node)):
        a, b = tree.child[node[i]]
        child[i] = (local[int(a)], local[int(b)])
        parent[local[int(a)]] = i
        parent[local[int(b)]] = i
    return Forest(C=C, node=node, child=child, parent=parent)


def rows_per_node(tree: LightTree, cut, m_s: int, rate1: float) -> np.ndarray:
    """k_c for every global-cut node (float32 decision, see module docstring)."""
    f32 = np.float32
    cut = np.asarray(cut, dtype=np.int64)
    C = cut.size
    kappa = max(f32(2.0), f32(f32(rate1) * f32(m_s)))
    x = f32(kappa * f32(C)) * (tree.I[cut].astype(np.float32) / f32(tree.I[0]))
    k = np.floor((x + f32(0.5)).astype(np.float32)).astype(np.int64)
    return np.minimum(np.minimum(np.maximum(k, 2), MAX_ROWS_PER_NODE), m_s)


def draw_rows(seed: int, s: int, c: int, k: int, m_s: int) -> np.ndarray:
    """First k distinct rows of the Philox draws of node c in slice s (sorted)."""
    if k >= m_s:
        return np.arange(m_s, dtype=np.int64)
    got = []
    seen = set()
    t0 = 0
    while len(got) < k:
        if t0 >= MAX_DRAWS:
            raise RuntimeError("pass-1 draw limit reached")
        t = np.arange(t0, min(t0 + 256, MAX_DRAWS), dtype=np.uint64)
        w = philox.draw(seed, t, c, s, philox.TAG_PASS1)[0]
        for r in philox.uniform_index(w, m_s):
            r = int(r)
            if r not in seen:
                seen.add(r)
                got.append(r)
                if len(got) == k:
                    break
        t0 += 256
    return np.array(sorted(got), dtype=np.int64)


@dataclasses.dataclass
class Pass1Slice:
    col_node: np.ndarray    # [n'] tree node ids of the coarsened cut, leaf order
    rows: np.ndarray        # [e] local row of each observed entry
    cols: np.ndarray        # [e] local column
    vals: np.ndarray        # [e] A(row, col)
    g: np.ndarray           # [n'] column importance
    s_hat: float
    log: list               # (f, eps, cost, threshold, merged, p, q, zeta_f, V_p, V_q) per test
    n_rays: int


def forest_heights(forest: Forest) -> np.ndarray:
    """Height of every forest node (0 on the cut, 1 + the larger child height above)."""
    nf = 2 * forest.C - 1
    height = np.full(nf, -1, dtype=np.int64)
    height[:forest.C] = 0
    changed = True
    while changed:
        changed = False
        for f in range(forest.C, nf):
            a, b = forest.child[f]
            if height[f] < 0 and height[a] >= 0 and height[b] >= 0:
                height[f] = 1 + max(height[a], height[b])
                changed = True
    return height


def merges(cost: float, thr: float, s_hat: float) -> bool:
    """The Sec. 4 test: merge while the cost is below the bound tau * S_hat.  In a
    dark slice (S_hat = 0, every pass-1 entry zero) the bound is zero; it is read as
    met by a pair whose cost is exactly zero, whose entries agree on every sampled
    row, so that the slice coarsens as far as its samples cannot tell lights apart."""
    return cost < thr or (s_hat == 0.0 and cost == 0.0)


def coarsen_slice(tree: LightTree, forest: Forest, points_s, vpls, boxes, s: int, row0: int,
                  m_s: int, rate1: float, tau: float, seed: int, d_min=0.01,
                  order_rng: np.random.Generator | None = None, target: int | None = None) -> Pass1Slice:
    """Pass 1 + coarsening of slice s (rows row0 .. row0+m_s-1 of the slice-ordered points).

    With `target` the coarsening runs until the cut holds at most `target` nodes
    instead of against tau (Sec. 4, last paragraph): the testable sibling pairs are
    ordered by cost and merged from the least; a merge whose parent pair becomes
    testable tests it and adds it to the order.  Ties of cost go to the pair of lower
    forest height, then to the lower forest id (the paper leaves ties open)."""
    C = forest.C
    nf = 2 * C - 1
    if m_s == 0:
        z = np.zeros(0, dtype=np.int64)
        return Pass1Slice(col_node=z, rows=z, cols=z, vals=np.zeros(0), g=np.zeros(0), s_hat=0.0,
                          log=[], n_rays=0)
    rep = tree.rep
    scale = node_scale(tree, vpls, forest.node)
    n_rays = 0

    def entries(local_node, rows):
        nonlocal n_rays
        n_rays += len(rows)
        t = forest.node[local_node]
        return shading.node_entries(points_s, vpls, row0 + np.asarray(rows, dtype=np.int64),
                                    np.full(len(rows), rep[t]), np.full(len(rows), scale[local_node]),
                                    boxes, d_min)

    k = rows_per_node(tree, forest.node[:C], m_s, rate1)
    rows = {}
    vals = {}
    for c in range(C):
        rows[c] = draw_rows(seed, s, c, int(k[c]), m_s)
        vals[c] = entries(c, rows[c])
    s_hat = float(sum(v.mean() for v in (vals[c] for c in range(C)) if v.size))
    thr = tau * s_hat if target is None else float("inf")

    alive = np.zeros(nf, dtype=bool)
    alive[:C] = True
    tested = np.zeros(nf, dtype=bool)
    cost = np.zeros(nf)
    rejected = {}
    log = []

    def test_pair(f):
        """Sec. 4 test of the pair under forest node f on zeta_f = zeta_a U zeta_b."""
        a, b = (int(x) for x in forest.child[f])
        ta, tb = forest.node[a], forest.node[b]
        p, q = (a, b) if tree.I[ta] >= tree.I[tb] else (b, a)
        rf = np.union1d(rows[a], rows[b])
        full = {}
        for x in (a, b):
            v = np.empty(rf.size)
            have = np.isin(rf, rows[x])
            v[have] = vals[x]           # rows[x] is sorted and a subset of rf
            if np.any(~have):
                v[~have] = entries(x, rf[~have])
            full[x] = v
        Ip = float(tree.I[forest.node[p]])
        Iq = float(tree.I[forest.node[q]])
        eps = float(np.max(np.abs(full[q] - full[p] * (Iq / Ip)))) if rf.size else 0.0
        tested[f] = True
        return dict(f=f, a=a, b=b, p=p, q=q, rf=rf, full=full, eps=eps, cost=eps + cost[q])

    def merge(t):
        f, a, b, p = t["f"], t["a"], t["b"], t["p"]
        alive[a] = alive[b] = False
        alive[f] = True
        rows[f] = t["rf"]
        vals[f] = t["full"][p] * (float(tree.I[forest.node[f]]) / float(tree.I[forest.node[p]]))
        cost[f] = t["cost"]

    def ready(f):
        return not tested[f] and alive[forest.child[f, 0]] and alive[forest.child[f, 1]]

    if target is None:
        while True:
            todo = [f for f in range(C, nf) if ready(f)]
            if not todo:
                break
            if order_rng is not None:
                order_rng.shuffle(todo)
            for f in todo:
                t = test_pair(f)
                merged = merges(t["cost"], thr, s_hat)
                log.append((f, t["eps"], t["cost"], thr, bool(merged), t["p"], t["q"], t["rf"],
                            t["full"][t["p"]], t["full"][t["q"]]))
                if merged:
                    merge(t)
                else:
                    rejected[f] = (t["rf"], t["full"][t["a"]], t["full"][t["b"]])
    else:
        height = forest_heights(forest)
        cand = {}
        for f in range(C, nf):
            if ready(f):
                cand[f] = test_pair(f)
        n_live = C
        while n_live > target and cand:
            f = min(cand, key=lambda x: (cand[x]["cost"], height[x], x))
            t = cand.pop(f)
            log.append((f, t["eps"], t["cost"], thr, True, t["p"], t["q"], t["rf"], t["full"][t["p"]],
                        t["full"][t["q"]]))
            merge(t)
            n_live -= 1
            par = int(forest.parent[f])
            if par >= 0 and ready(par):
                cand[par] = test_pair(par)
        for f, t in cand.items():  # tested and not merged
            rejected[f] = (t["rf"], t["full"][t["a"]], t["full"][t["b"]])

    live = np.nonzero(alive)[0]
    live = live[np.argsort(tree.first[forest.node[live]], kind="stable")]
    col_node = forest.node[live]
    er, ec, ev = [], [], []
    g = np.full(live.size, np.nan)
    for j, x in enumerate(live):
        par = forest.parent[x]
        if par >= 0 and int(par) in rejected:
            rf, va, vb = rejected[int(par)]
            r, v = rf, (va if forest.child[par, 0] == x else vb)
        else:
            r, v = rows[x], vals[x]
        er.append(r)
        ec.append(np.full(r.size, j))
        ev.append(v)
        if r.size >= 2:
            g[j] = v.max() - v.min()
    defined = ~np.isnan(g)
    g[~defined] = g[defined].max() if np.any(defined) else 0.0
    return Pass1Slice(col_node=col_node, rows=np.concatenate(er), cols=np.concatenate(ec),
                      vals=np.concatenate(ev), g=g, s_hat=s_hat, log=log, n_rays=n_rays)
