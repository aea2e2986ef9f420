"""Entries of the lighting matrix and the shadow-ray visibility test (float64).

The paper defines A(i, j) as the illumination that light j sends to surface point i
(Sec. 3, "Overview") and computes visibility by casting shadow rays (Sec. 6).  It
does not print the shading model; the readings taken here are:

* Light j is a VPL at q with normal n_q, flux Phi, albedo rho_q, Phong exponent e_q
  and incoming direction w_in (unit, towards the light it came from).  Point i is at
  p with normal n_p, albedo rho_p, exponent e_p and view direction w_o (unit,
  towards the camera).  With d = q - p and w = d / |d|:
      A(i, j) = Phi * f_p(w -> w_o) * f_q(w_in -> -w) * G * V
      G = max(0, n_p.w) * max(0, -n_q.w) / max(|d|^2, d_min^2)
  d_min (0.01 by default) bounds the 1/d^2 singularity; every side (brute force,
  oracle pipeline, CUDA path) uses the same constant.
* BRDF: diffuse rho/pi; on glossy faces (e > 0) a normalised modified Phong mix
      f = 0.5 rho/pi + 0.5 rho (e+2)/(2 pi) max(0, cos a)^e,
  a = angle between the mirror of the incoming direction about n and the outgoing one.
* V: the segment from p + 1e-4 n_p to q + 1e-4 n_q, restricted to the parametric
  interval (1e-4, 1 - 1e-4), is blocked iff it meets a closed occluder box (slab
  test, t_enter <= t_exit).  The room's walls never occlude (the room is convex).
  The oracle tests every box; no acceleration structure is involved.
* When either cosine is not positive, G = 0 and no ray is needed.

A light-tree node c acts as its representative VPL rep(c) scaled in intensity
(Sec. 4: "L_f is the same as L_a except their intensity values"): with the intensity
I = Phi * rho summed over the node's VPLs,
      A(i, c) = A(i, rep(c)) * I_c / I_rep(c).
"""
from __future__ import annotations

import numpy as np

RAY_OFFSET = 1e-4
T_MIN = 1e-4
T_MAX = 1.0 - 1e-4


def brdf(albedo, gloss, nrm, w_in, w_out):
    """f(w_in -> w_out) at a surface with normal ``nrm`` (all arrays [..., 3])."""
    albedo = np.asarray(albedo, dtype=np.float64)
    gloss = np.asarray(gloss, dtype=np.float64)
    diffuse = albedo / np.pi
    refl = 2.0 * np.sum(nrm * w_in, axis=-1, keepdims=True) * nrm - w_in
    cos_a = np.maximum(0.0, np.sum(refl * w_out, axis=-1))
    glossy = 0.5 * albedo / np.pi + 0.5 * albedo * (gloss + 2.0) / (2.0 * np.pi) * np.power(
        cos_a, np.where(gloss > 0, gloss, 1.0))
    return np.where(gloss > 0, glossy, diffuse)


def brdf_max(albedo, gloss):
    """Largest value of :func:`brdf` over all direction pairs."""
    albedo = np.asarray(albedo, dtype=np.float64)
    gloss = np.asarray(gloss, dtype=np.float64)
    return np.where(gloss > 0, 0.5 * albedo / np.pi + 0.5 * albedo * (gloss + 2.0) / (2.0 * np.pi),
                    albedo / np.pi)


def _split_points(points, rows):
    P = np.asarray(points, dtype=np.float64)
    return (P[0, rows, :3], P[0, rows, 3], P[1, rows, :3], P[1, rows, 3], P[2, rows, :3])


def _split_vpls(vpls, cols):
    L = np.asarray(vpls, dtype=np.float64)
    return (L[0, cols, :3], L[0, cols, 3], L[1, cols, :3], L[1, cols, 3], L[2, cols, :3], L[2, cols, 3])


def unoccluded(points, vpls, rows, cols, d_min=0.01):
    """Phi * f_p * f_q * G for the (row, VPL) pairs, i.e. A(i, j) with V = 1."""
    p, rho_p, n_p, e_p, w_o = _split_points(points, rows)
    q, rho_q, n_q, e_q, w_in, flux = _split_vpls(vpls, cols)
    d = q - p
    dist2 = np.sum(d * d, axis=-1)
    w = d / np.sqrt(np.maximum(dist2, 1e-300))[..., None]
    cos_p = np.maximum(0.0, np.sum(n_p * w, axis=-1))
    cos_q = np.maximum(0.0, -np.sum(n_q * w, axis=-1))
    G = cos_p * cos_q / np.maximum(dist2, d_min * d_min)
    f_p = brdf(rho_p, e_p, n_p, w, w_o)
    f_q = brdf(rho_q, e_q, n_q, w_in, -w)
    return flux * f_p * f_q * G


def segment_hits_triangles(o, e, tris):
    """True where the segment o + t (e - o), t in (T_MIN, T_MAX), meets a closed
    triangle (Moller-Trumbore in float64; a segment in a triangle's plane does not
    hit it).  tris [nt, 3, 3].  Tests every triangle."""
    o = np.asarray(o, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    k = o.shape[0]
    hit = np.zeros(k, dtype=bool)
    T = np.asarray(tris, dtype=np.float64)
    if T.shape[0] == 0 or k == 0:
        return hit
    v0, e1, e2 = T[:, 0], T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]
    D = e - o
    chunk = max(1, 2_000_000 // T.shape[0])
    for s in range(0, k, chunk):
        DD = D[s:s + chunk, None, :]
        p = np.cross(DD, e2[None])
        det = np.sum(e1[None] * p, axis=-1)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / det
            sv = o[s:s + chunk, None, :] - v0[None]
            u = np.sum(sv * p, axis=-1) * inv
            q = np.cross(sv, e1[None])
            v = np.sum(DD * q, axis=-1) * inv
            t = np.sum(e2[None] * q, axis=-1) * inv
        ok = (det != 0) & (u >= 0) & (u <= 1) & (v >= 0) & (u + v <= 1) & (t > T_MIN) & (t < T_MAX)
        hit[s:s + chunk] = np.any(ok, axis=1)
    return hit


def segment_blocked(o, e, boxes):
    """True where the segment o + t (e - o), t in (T_MIN, T_MAX), meets a closed box
    (or, when ``boxes`` is a pair (boxes, triangles), a box or a triangle).

    o, e: [k, 3] float64; boxes [nb, 6].  Tests every box (slab method).
    """
    if isinstance(boxes, tuple):
        bx, tris = boxes
        blocked = segment_blocked(o, e, bx)
        rest = ~blocked
        if np.any(rest):
            blocked[rest] = segment_hits_triangles(np.asarray(o)[rest], np.asarray(e)[rest], tris)
        return blocked
    o = np.asarray(o, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    k = o.shape[0]
    blocked = np.zeros(k, dtype=bool)
    if boxes.shape[0] == 0 or k == 0:
        return blocked
    D = e - o
    bl = np.asarray(boxes[:, :3], dtype=np.float64)
    bh = np.asarray(boxes[:, 3:], dtype=np.float64)
    chunk = max(1, 4_000_000 // max(1, boxes.shape[0]))
    for s in range(0, k, chunk):
        oo = o[s:s + chunk, None, :]
        DD = D[s:s + chunk, None, :]
        par = DD == 0.0
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (bl[None] - oo) / DD
            tb = (bh[None] - oo) / DD
        tn = np.minimum(ta, tb)
        tf = np.maximum(ta, tb)
        # an axis the segment runs parallel to: inside the closed slab -> no constraint,
        # outside -> empty interval
        inside = (oo >= bl[None]) & (oo <= bh[None])
        tn = np.where(par, np.where(inside, -np.inf, np.inf), tn)
        tf = np.where(par, np.where(inside, np.inf, -np.inf), tf)
        t_enter = np.maximum(tn.max(axis=2), T_MIN)
        t_exit = np.minimum(tf.min(axis=2), T_MAX)
        blocked[s:s + chunk] = np.any(t_enter <= t_exit, axis=1)
    return blocked


def shadow_endpoints(points, vpls, rows, cols):
    """Offset segment endpoints of the shadow rays for (row, VPL) pairs."""
    P = np.asarray(points, dtype=np.float64)
    L = np.asarray(vpls, dtype=np.float64)
    o = P[0, rows, :3] + RAY_OFFSET * P[1, rows, :3]
    e = L[0, cols, :3] + RAY_OFFSET * L[1, cols, :3]
    return o, e


def visible(points, vpls, rows, cols, boxes):
    """V(i, j) in {0, 1} for (row, VPL) pairs."""
    o, e = shadow_endpoints(points, vpls, rows, cols)
    return ~segment_blocked(o, e, boxes)


def vpl_entries(points, vpls, rows, cols, boxes, d_min=0.01):
    """A(i, j) for (row, VPL) pairs, shadow rays cast only where G > 0."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    val = unoccluded(points, vpls, rows, cols, d_min)
    need = val > 0
    if np.any(need):
        vis = visible(points, vpls, rows[need], cols[need], boxes)
        val[need] = np.where(vis, val[need], 0.0)
    return val


def node_entries(points, vpls, rows, rep, scale, boxes, d_min=0.01):
    """A(i, c) for light-tree nodes: A(i, rep(c)) * I_c / I_rep(c).

    ``rep`` holds the representative VPL of each pair's node and ``scale`` the
    factor I_c / I_rep(c).
    """
    return vpl_entries(points, vpls, rows, rep, boxes, d_min) * np.asarray(scale, dtype=np.float64)
