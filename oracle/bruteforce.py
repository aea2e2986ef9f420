"""Brute-force render: the image is the column sum of the full lighting matrix.

Sec. 3 ("Overview"): the rendered image is Sigma_A, the sum of the columns of A,
one column per VPL.  This module evaluates every entry A(i, j) (float64, every
occluder box tested) and sums over j.  It is the ground truth every rel-RMSE is
measured against (the reference images of Fig. 2 are rendered this way).
"""
from __future__ import annotations

import numpy as np

from . import shading


def render_rows(points, vpls, boxes, rows, d_min=0.01, chunk=1 << 20):
    """Sum_j A(i, j) over all VPLs for the given rows (float64)."""
    rows = np.asarray(rows, dtype=np.int64)
    n = vpls.shape[1]
    out = np.zeros(rows.shape[0])
    per = max(1, chunk // max(1, n))
    for s in range(0, rows.shape[0], per):
        r = rows[s:s + per]
        rr = np.repeat(r, n)
        cc = np.tile(np.arange(n), r.shape[0])
        val = shading.vpl_entries(points, vpls, rr, cc, boxes, d_min)
        out[s:s + per] = val.reshape(r.shape[0], n).sum(axis=1)
    return out


def render(points, vpls, boxes, d_min=0.01):
    """The full brute-force image over every shading point (float64, [m])."""
    return render_rows(points, vpls, boxes, np.arange(points.shape[1]), d_min)


def rel_rmse(img, ref):
    """||img - ref||_2 / ||ref||_2 over all pixels.

    The paper reports an undefined "error=...%" (Figs. 4-5); this relative RMSE is
    the reading used throughout.
    """
    img = np.asarray(img, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(img - ref) / max(np.linalg.norm(ref), 1e-300))
