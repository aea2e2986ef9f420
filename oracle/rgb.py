"""Colour: the three channels of a slice stacked as rows of one matrix (float64;
test infrastructure only).

The paper renders coloured scenes (Sec. 6) but prints only the scalar lighting
matrix.  Readings taken here:

* Channel k of an entry is the scalar entry of Sec. 3 with the colour of each factor
  in that channel: A_k(i, j) = Phi_k f_p,k f_q,k G V, with the point's albedo
  rho_p,k in f_p, the VPL's albedo rho_q,k in f_q and its flux Phi_k; a light-tree
  node acts as its representative scaled by I_c,k / I_rep,k with the per-channel
  intensity I_c,k = sum of Phi_k rho_q,k over the node's VPLs (Sec. 4 per channel).
* Sampling (pass 1, coarsening, pass 2) runs on the scalar scene, whose albedo and
  flux are the luminances of the colours; each sampled (pixel, column) pair then
  observes all three channels (one shadow ray serves them all).
* Slice s of m' pixels becomes a 3m' x n' matrix whose row 3i + k is channel k of
  pixel i, completed like a scalar slice, so one V is shared by the channels; the
  image of channel k at pixel i is max(0, u_{3i+k} . (V^T 1)).
"""
from __future__ import annotations

import numpy as np

from . import adm, als, bruteforce, pass1, pass2, pipeline, shading


def channel_vpls(vpls, rgb: dict, k: int):
    """The VPLs of channel k: albedo and flux replaced by their channel."""
    L = np.asarray(vpls, dtype=np.float64).copy()
    L[0, :, 3] = rgb["vpl_albedo"][:, k]
    L[2, :, 3] = rgb["vpl_flux"][:, k]
    return L


def channel_scene(points, vpls, rgb: dict, k: int):
    """The scalar arrays of channel k: albedos and flux replaced by their channel."""
    P = np.asarray(points, dtype=np.float64).copy()
    P[0, :, 3] = rgb["point_albedo"][:, k]
    return P, channel_vpls(vpls, rgb, k)


def channel_points(points_s, rgb: dict, row_perm, k: int):
    """Slice-ordered points of channel k (points_s = points permuted by row_perm)."""
    P = np.asarray(points_s, dtype=np.float64).copy()
    P[0, :, 3] = np.asarray(rgb["point_albedo"], dtype=np.float64)[np.asarray(row_perm), k]
    return P


def node_intensity(tree, rgb: dict) -> np.ndarray:
    """I_c,k for every tree node [2n-1, 3]: sum of Phi_k rho_k over the node's VPLs."""
    prod = np.asarray(rgb["vpl_flux"], dtype=np.float64) * np.asarray(rgb["vpl_albedo"], dtype=np.float64)
    cs = np.concatenate([np.zeros((1, 3)), np.cumsum(prod[tree.order], axis=0)])
    return cs[tree.last + 1] - cs[tree.first]


def node_entries(points_s, vpls, rgb: dict, row_perm, tree, rows, nodes, boxes, d_min=0.01) -> np.ndarray:
    """A_k(i, c) [len(rows), 3] for slice-ordered rows and tree nodes, straight from
    the per-channel definition."""
    rows = np.asarray(rows, dtype=np.int64)
    nodes = np.asarray(nodes, dtype=np.int64)
    out = np.zeros((rows.size, 3))
    if rows.size == 0:
        return out
    Ik = node_intensity(tree, rgb)
    rep = tree.rep[nodes]
    for k in range(3):
        P = channel_points(points_s, rgb, row_perm, k)
        L = channel_vpls(vpls, rgb, k)
        i_rep = L[2, rep, 3] * L[0, rep, 3]
        out[:, k] = shading.vpl_entries(P, L, rows, rep, boxes, d_min) * (Ik[nodes, k] / np.maximum(i_rep, 1e-300))
    return out


def bruteforce_rgb(points, vpls, rgb: dict, boxes, d_min=0.01) -> np.ndarray:
    """The full image over all VPLs per channel [m, 3]."""
    return np.stack([bruteforce.render(*channel_scene(points, vpls, rgb, k), boxes, d_min) for k in range(3)],
                    axis=1)


def stack(rows, cols, vals_rgb):
    """(row, col, [r, g, b]) entries -> entries of the stacked matrix (row 3i + k)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    r3 = (3 * rows[:, None] + np.arange(3)[None, :]).ravel()
    c3 = np.repeat(cols, 3)
    return r3, c3, np.asarray(vals_rgb, dtype=np.float64).ravel()


def complete_stacked(rows, cols, vals_rgb, m_s: int, n_s: int, r: int, cfg, seed: int, s: int):
    """Completion of the stacked 3m' x n' slice (ALS, or ADM when cfg selects it)."""
    r3, c3, v3 = stack(rows, cols, vals_rgb)
    if cfg.get("completion", "als") == "adm":
        return adm.complete_slice_adm(r3, c3, v3, 3 * m_s, n_s, r, cfg["adm_iters"], cfg["adm_alpha_rel"],
                                      cfg["adm_gamma"], seed, s)
    return als.complete_slice(r3, c3, v3, 3 * m_s, n_s, r, cfg["als_iters"], cfg["lam_rel"], seed, s)


def render_stacked(factors, row_perm, slice_off, m: int) -> np.ndarray:
    """img[pixel, k] = max(0, u_{3i+k} . (V^T 1)) for every slice [m, 3]."""
    img = np.zeros((m, 3))
    for s, (U, V) in enumerate(factors):
        a, b = int(slice_off[s]), int(slice_off[s + 1])
        if b == a:
            continue
        val = U @ V.sum(axis=0)
        img[np.asarray(row_perm)[a:b]] = np.maximum(val.reshape(b - a, 3), 0.0)
    return img


def render_frame(scene, cfg, st, seed=None, slices=None):
    """Steps 3-5 in colour: scalar sampling per slice, RGB values of the sampled pairs,
    stacked completion, RGB image [m, 3] (only the listed slices when given, the rest
    black).  Returns (image, per-slice (rows, cols, col_node, vals_rgb))."""
    seed = cfg["frame_seed"] if seed is None else seed
    tree, forest, pts_s = st["tree"], st["forest"], st["pts_s"]
    S = len(st["slice_off"]) - 1
    todo = set(range(S) if slices is None else slices)
    factors, omega = [], []
    for s in range(S):
        a, b = int(st["slice_off"][s]), int(st["slice_off"][s + 1])
        m_s = b - a
        if s not in todo:
            factors.append((np.zeros((3 * m_s, 1)), np.zeros((0, 1))))
            omega.append(None)
            continue
        p1 = pass1.coarsen_slice(tree, forest, pts_s, scene.vpls, scene.occluders, s, a, m_s, cfg["rate1"], cfg["tau"],
                                 seed, cfg["d_min"], target=pipeline.target_cut(cfg))
        n_s = p1.col_node.size
        r2, c2, _, _ = pass2.draw_pass2(seed, s, m_s, p1.g, p1.rows * n_s + p1.cols, cfg["rate"])
        rows = np.concatenate([p1.rows, r2]).astype(np.int64)
        cols = np.concatenate([p1.cols, c2]).astype(np.int64)
        vals = node_entries(pts_s, scene.vpls, scene.rgb, st["row_perm"], tree, a + rows, p1.col_node[cols],
                            scene.occluders, cfg["d_min"])
        factors.append(complete_stacked(rows, cols, vals, m_s, n_s, cfg["rank"], cfg, seed, s))
        omega.append((rows, cols, p1.col_node, vals))
    return render_stacked(factors, st["row_perm"], st["slice_off"], scene.m), omega
