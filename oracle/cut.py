"""Conservative global light cut (Sec. 3 step 1; level-by-level splitting, Sec. 6).

The paper takes the global cut from the lightcuts papers: it is error-bounded for
the whole image and conservative because visibility is bounded by 1; the splitting
test runs for all nodes of a level in parallel.  Readings taken here:

* Test rows R: one shading point per 8x8 pixel block, the pixel at offset (4, 4).
* Estimate at x: sum over cut nodes c of A(x, c) with V = 1 (unoccluded).
* Upper bound of node c at x (cosines bounded by 1, visibility by 1):
      b_c(x) = I_c * B_c * fmax(x) / max(dist(x, AABB_c)^2, d_min^2)
  with B_c = max over the node's VPLs of f_max / albedo and fmax(x) the largest BRDF
  value at x.  It bounds the sum of the node's VPL contributions at x.
* Error of node c: max over x in R of b_c(x) / estimate(x), infinite where the
  estimate is zero (a zero estimate cannot certify any relative error).
* Level-synchronous refinement from the root: in each round every internal cut node
  whose error exceeds eps is a candidate; at most max(1, floor(growth * |cut|))
  candidates split (growth = 0.5), the largest errors first (order: error
  descending, node id ascending), each replaced by its two children.  Rounds repeat
  until nothing splits or the cut holds ``max_cut`` nodes.  Capping the growth of a
  round keeps the splitting budget on the nodes with the largest bound (the paper's
  cuts are error-bounded; a cap on the cut size needs an order).
* The cut is returned in leaf order (ascending first covered leaf), so the leaves
  under any tree node form a contiguous run of it.
"""
from __future__ import annotations

import numpy as np

from . import shading
from .tree import LightTree, node_scale


def test_rows(width: int, height: int, block: int = 8) -> np.ndarray:
    """Pixel indices of the per-block test rows (row-major pixel order)."""
    ys = np.arange(block // 2, height, block)
    xs = np.arange(block // 2, width, block)
    if ys.size == 0:
        ys = np.array([height // 2])
    if xs.size == 0:
        xs = np.array([width // 2])
    gy, gx = np.meshgrid(ys, xs, indexing="ij")
    return (gy * width + gx).ravel()


def node_bound(tree: LightTree, points, rows, nodes, d_min=0.01) -> np.ndarray:
    """b_c(x) for every (row, node) pair of the outer product rows x nodes."""
    P = np.asarray(points, dtype=np.float64)
    x = P[0, rows, :3][:, None, :]
    fx = shading.brdf_max(P[0, rows, 3], P[1, rows, 3])[:, None]
    lo = tree.lo[nodes].astype(np.float64)[None]
    hi = tree.hi[nodes].astype(np.float64)[None]
    gap = np.maximum(0.0, np.maximum(lo - x, x - hi))
    dist2 = np.sum(gap * gap, axis=-1)
    I = tree.I[nodes].astype(np.float64)[None]
    B = tree.B[nodes][None]
    return I * B * fx / np.maximum(dist2, d_min * d_min)


def estimate(tree: LightTree, points, vpls, rows, cut, d_min=0.01) -> np.ndarray:
    """Unoccluded estimate sum_c A(x, c) (V = 1) for each test row x."""
    cut = np.asarray(cut, dtype=np.int64)
    rr = np.repeat(rows, cut.size)
    cc = np.tile(cut, rows.size)
    val = shading.unoccluded(points, vpls, rr, tree.rep[cc], d_min) * node_scale(tree, vpls, cc)
    return val.reshape(rows.size, cut.size).sum(axis=1)


def node_errors(tree: LightTree, points, vpls, rows, cut, d_min=0.01) -> np.ndarray:
    """max over test rows of b_c(x) / estimate(x); a zero estimate counts as infinite."""
    est = estimate(tree, points, vpls, rows, cut, d_min)
    b = node_bound(tree, points, rows, np.asarray(cut), d_min)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(est[:, None] > 0, b / est[:, None], np.where(b > 0, np.inf, 0.0))
    return ratio.max(axis=0)


def build_global_cut(tree: LightTree, points, vpls, width, height, eps=0.05, max_cut=4096,
                     d_min=0.01, rows=None, growth=0.5):
    """Return the global cut (tree node ids in leaf order)."""
    rows = test_rows(width, height) if rows is None else np.asarray(rows)
    cut = [0]
    while True:
        err = node_errors(tree, points, vpls, rows, cut, d_min)
        cand = [(i, c) for i, c in enumerate(cut) if not tree.is_leaf(c) and err[i] > eps]
        if not cand:
            break
        room = max_cut - len(cut)
        if growth is not None:
            room = min(room, max(1, int(growth * len(cut))))
        stop = False
        if len(cand) > room:
            cand.sort(key=lambda ic: (-err[ic[0]], ic[1]))
            cand = cand[:max(0, room)]
            stop = len(cut) + len(cand) >= max_cut
        if not cand:
            break
        split = {c for _, c in cand}
        new = []
        for c in cut:
            if c in split:
                new.extend(int(x) for x in tree.child[c])
            else:
                new.append(c)
        cut = new
        if stop:
            break
    cut = np.asarray(cut, dtype=np.int64)
    return cut[np.argsort(tree.first[cut], kind="stable")]
