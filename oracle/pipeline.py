"""The five steps of Sec. 3 end to end on the CPU (float64 arithmetic).

global light cut -> matrix slicing -> pass 1 + coarsening -> pass 2 -> completion
-> image.  Each step can be given precomputed inputs (a cut, slices) so that a
stage of the CUDA path can be checked in isolation on exactly the oracle's inputs.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import adm, als, cut as cut_mod, pass1, pass2, render, shading, slices as slices_mod, tree as tree_mod
from .tree import node_scale


@dataclasses.dataclass
class SliceResult:
    p1: pass1.Pass1Slice
    p2_rows: np.ndarray
    p2_cols: np.ndarray
    p2_vals: np.ndarray
    U: np.ndarray
    V: np.ndarray
    hit_cap: bool

    @property
    def n_cols(self) -> int:
        return int(self.p1.col_node.size)

    def omega(self):
        """All observed entries (pass 1 then pass 2)."""
        return (np.concatenate([self.p1.rows, self.p2_rows]),
                np.concatenate([self.p1.cols, self.p2_cols]),
                np.concatenate([self.p1.vals, self.p2_vals]))


def setup(scene, cfg, cut=None, slicing=None):
    """Light tree, global cut, forest and slices (step 1 and 2)."""
    tree = tree_mod.build(scene.vpls)
    if cut is None:
        cut = cut_mod.build_global_cut(tree, scene.points, scene.vpls, scene.width, scene.height,
                                       eps=cfg["eps_cut"], max_cut=cfg["max_cut"], d_min=cfg["d_min"])
    forest = pass1.build_forest(tree, cut)
    if slicing is None and cfg.get("slicing", "kmeans") == "split6d":
        row_perm, slice_off = slices_mod.split6d_slices(scene.points, cfg["slice_size"],
                                                        cfg["slice_feature_normal_weight"])
    elif slicing is None:
        row_perm, slice_off, _, _ = slices_mod.kmeans_slices(
            scene.points, cfg["n_slices"], cfg["kmeans_iters"], cfg["slice_feature_normal_weight"])
        if cfg.get("slice_bounds"):
            lo, hi = cfg["slice_bounds"]
            row_perm, slice_off = slices_mod.bound_slices(scene.points, row_perm, slice_off, lo, hi,
                                                          cfg["slice_feature_normal_weight"])
    else:
        row_perm, slice_off = slicing
    pts_s = slices_mod.permute_points(scene.points, row_perm)
    return dict(tree=tree, cut=np.asarray(cut), forest=forest, row_perm=np.asarray(row_perm),
                slice_off=np.asarray(slice_off), pts_s=pts_s)


def run_slice(st, scene, cfg, s, seed, weights=None, order_rng=None, prev=None) -> SliceResult:
    tree, forest, pts_s = st["tree"], st["forest"], st["pts_s"]
    a, b = int(st["slice_off"][s]), int(st["slice_off"][s + 1])
    m_s = b - a
    p1 = pass1.coarsen_slice(tree, forest, pts_s, scene.vpls, scene.occluders, s, a, m_s, cfg["rate1"],
                             cfg["tau"], seed, cfg["d_min"], order_rng, target=target_cut(cfg))
    n_s = p1.col_node.size
    w = p1.g if weights is None else weights
    r2, c2, _, hit_cap = pass2.draw_pass2(seed, s, m_s, w, p1.rows * n_s + p1.cols, cfg["rate"])
    if r2.size:
        nodes = p1.col_node[c2]
        v2 = shading.node_entries(pts_s, scene.vpls, a + r2, tree.rep[nodes],
                                  node_scale(tree, scene.vpls, nodes), scene.occluders, cfg["d_min"])
    else:
        v2 = np.zeros(0)
    res = SliceResult(p1=p1, p2_rows=r2, p2_cols=c2, p2_vals=v2, U=None, V=None, hit_cap=hit_cap)
    rows, cols, vals = res.omega()
    if cfg.get("completion", "als") == "adm":
        res.U, res.V = adm.complete_slice_adm(rows, cols, vals, m_s, n_s, slice_rank(cfg, n_s), cfg["adm_iters"],
                                              cfg["adm_alpha_rel"], cfg["adm_gamma"], seed, s)
    else:
        r = slice_rank(cfg, n_s)
        V0 = None
        if prev is not None:  # the previous frame's result of this slice: start from its factors
            V0 = als.warm_start(seed, s, p1.col_node, vals, r, prev.p1.col_node, prev.V)
        res.U, res.V = als.complete_slice(rows, cols, vals, m_s, n_s, r, cfg["als_iters"], cfg["lam_rel"], seed, s,
                                          V0=V0)
    return res


def target_cut(cfg):
    """cfg["target_cut"] > 0: coarsen each slice to that many nodes by cost order
    (Sec. 4); otherwise against tau."""
    t = int(cfg.get("target_cut", 0))
    return t if t > 0 else None


def slice_rank(cfg, n_s: int) -> int:
    """The rank of a slice: cfg["rank"], or with cfg["rank_cols"] > 0 the per-slice
    rule min(rank, max(8, 8 ceil(n' / rank_cols))) (a multiple of 8 growing with the
    coarsened cut; our reading of the configuration's "rank 8-32 chosen per slice")."""
    cols = int(cfg.get("rank_cols", 0))
    if cols <= 0:
        return int(cfg["rank"])
    return int(min(cfg["rank"], max(8, 8 * -(-int(n_s) // cols))))


def render_frame(scene, cfg, st=None, seed=None, slices=None, prev=None):
    """Run steps 3-5 for every slice (or the listed ones); returns (image, per-slice
    results).  prev: the previous frame's per-slice results, whose factors start this
    frame's completion (als.warm_start)."""
    st = setup(scene, cfg) if st is None else st
    seed = cfg["frame_seed"] if seed is None else seed
    S = len(st["slice_off"]) - 1
    todo = range(S) if slices is None else slices
    results = {}
    for s in todo:
        results[s] = run_slice(st, scene, cfg, s, seed, prev=None if prev is None else prev.get(s))
    factors = []
    for s in range(S):
        if s in results:
            factors.append((results[s].U, results[s].V))
        else:
            factors.append((np.zeros((int(st["slice_off"][s + 1] - st["slice_off"][s]), 1)), np.zeros((0, 1))))
    img = render.render_slices(factors, st["row_perm"], st["slice_off"], scene.m)
    return img, results


def time_frame_sample(scene, cfg, st, slices, seed=None):
    """Wall time of steps 3-5 on the listed slices (the CPU baseline sample)."""
    t0 = time.perf_counter()
    render_frame(scene, cfg, st, seed, slices)
    return time.perf_counter() - t0
