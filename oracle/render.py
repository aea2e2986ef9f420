"""The image from the completed factors (Sec. 3 step 5).

For slice s with factors M = X Y the image restricted to the slice is
I(s) = M e = X (Y e), e the all-ones vector, so the completed matrix is never formed.
With U = X and V = Y^T: t_s = V^T w (w = e for the column sum) and pixel i of the
slice is u_i . t_s.  Low-rank ALS factors can produce slightly negative sums, which
light cannot: the pixel is clamped at 0 (the clamped and unclamped images are both
available).
"""
from __future__ import annotations

import numpy as np


def render_slices(factors, row_perm, slice_off, m: int, weights=None, clamp=True):
    """Scatter u_i . (V^T w) of every slice to its pixels; ``factors`` = [(U, V), ...]."""
    img = np.zeros(m)
    for s, (U, V) in enumerate(factors):
        a, b = int(slice_off[s]), int(slice_off[s + 1])
        if b == a:
            continue
        w = np.ones(V.shape[0]) if weights is None else np.asarray(weights[s], dtype=np.float64)
        t = V.T @ w
        val = U @ t
        img[row_perm[a:b]] = np.maximum(val, 0.0) if clamp else val
    return img
