"""Matrix slicing: cluster the shading points by position and normal (Sec. 3 step 2).

The paper partitions the rows of A by clustering the 6-D (coordinate, normal)
vectors of the surface points, following the lightslice method, and implements it
as a recursive binary split on the GPU (Sec. 6; ``split6d_slices`` below).  The
default reading taken here is Lloyd's k-means into S slices:

* feature of point i: (p_x, p_y, p_z, w n_x, w n_y, w n_z), w = 0.3;
* initial centroids: the points of rank floor((k + 1/2) m / S), k = 0..S-1, in the
  Morton order of the positions (codes as in the light tree, normalised to the
  points' bounding box; ties by pixel index);
* ``iters`` rounds of (assign every point to the nearest centroid in squared
  Euclidean distance, ties to the lowest index; move every non-empty centroid to
  the mean of its points); then a final assignment;
* rows are made slice-contiguous: row_perm lists pixel indices sorted by (slice,
  pixel index) and slice_off[s] .. slice_off[s+1] is slice s.
"""
from __future__ import annotations

import numpy as np

from .tree import morton_codes


def features(points, w=0.3) -> np.ndarray:
    P = np.asarray(points, dtype=np.float64)
    return np.concatenate([P[0, :, :3], w * P[1, :, :3]], axis=1)


def assign(X: np.ndarray, C: np.ndarray, chunk: int = 8192) -> np.ndarray:
    out = np.empty(X.shape[0], dtype=np.int64)
    for s in range(0, X.shape[0], chunk):
        d2 = np.sum((X[s:s + chunk, None, :] - C[None, :, :]) ** 2, axis=-1)
        out[s:s + chunk] = np.argmin(d2, axis=1)
    return out


def kmeans_slices(points, n_slices: int, iters: int = 10, w: float = 0.3):
    """Return (row_perm [m], slice_off [S+1], labels [m], centroids [S, 6])."""
    X = features(points, w)
    m = X.shape[0]
    S = int(n_slices)
    codes = morton_codes(np.asarray(points, dtype=np.float32)[0, :, :3])
    keys = (codes << np.uint64(32)) | np.arange(m, dtype=np.uint64)
    order = np.argsort(keys, kind="stable")
    init = order[(2 * np.arange(S) + 1) * m // (2 * S)]
    C = X[init].copy()
    for _ in range(iters):
        lab = assign(X, C)
        for k in range(S):
            sel = lab == k
            if np.any(sel):
                C[k] = X[sel].mean(axis=0)
    lab = assign(X, C)
    row_perm = np.argsort(lab, kind="stable")
    counts = np.bincount(lab, minlength=S)
    slice_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return row_perm.astype(np.int64), slice_off, lab, C


def split_sizes(m: int, target: int) -> list[int]:
    """Slice sizes of the recursive binary split, left to right: a node of n > target
    points splits into floor(n/2) (left) and the rest; depends on m and target only."""
    if m <= target:
        return [m]
    return split_sizes(m // 2, target) + split_sizes(m - m // 2, target)


def split6d_slices(points, target: int, w: float = 0.3):
    """The paper's own slicing (Sec. 6 step 2; slices of about `target` pixels, Sec. 3):
    the 6-D vectors (p, w n) are split recursively into a binary tree.  Reading: a
    node with more than `target` points splits along the feature dimension of largest
    extent (float32 extents, first largest), at the median: the floor(n/2) points
    smallest in (feature value, pixel index) go left, keeping their order, the rest go
    right.  Returns (row_perm [m], slice_off [S+1]) with the leaves left to right;
    inside a slice the pixels stay in ascending order."""
    P = np.asarray(points, dtype=np.float32)
    X = np.concatenate([P[0, :, :3], np.float32(w) * P[1, :, :3]], axis=1).astype(np.float32)
    m = X.shape[0]
    out = []

    def split(idx):
        n = idx.size
        if n <= target:
            out.append(idx)
            return
        ext = X[idx].max(axis=0) - X[idx].min(axis=0)
        d = int(np.argmax(ext))
        order = np.lexsort((idx, X[idx, d]))  # by value, then pixel index
        left = np.zeros(n, dtype=bool)
        left[order[:n // 2]] = True
        split(idx[left])
        split(idx[~left])

    split(np.arange(m, dtype=np.int64))
    row_perm = np.concatenate(out) if out else np.zeros(0, dtype=np.int64)
    slice_off = np.concatenate([[0], np.cumsum([a.size for a in out])]).astype(np.int64)
    return row_perm, slice_off


def permute_points(points, row_perm) -> np.ndarray:
    """Shading points in slice order."""
    return np.ascontiguousarray(np.asarray(points)[:, row_perm, :])


def bound_slices(points, row_perm, slice_off, min_rows: int, max_rows: int, w: float = 0.3):
    """Slices held between min_rows and max_rows rows (the uneven slices of the
    batched workloads).  Reading: starting from given slices (k-means), while some
    slice has fewer than min_rows rows and more than one slice is left, the smallest
    such slice (ties: the lowest index) is merged into the slice whose centroid is
    nearest to its own; then every slice with more than max_rows rows is split by the
    recursive 6-D median split of ``split6d_slices`` into parts of at most max_rows,
    the parts taking its place left to right.  Centroids are float64 means of the
    float32 features (p, w n), summed in ascending pixel order; distances are squared
    Euclidean in float64, ties to the lowest slice index.  Inside a slice the pixels
    are in ascending order.  Every slice ends inside the bounds when
    max_rows >= 2 min_rows - 1 (a split halves).  Returns (row_perm [m], slice_off [S'+1])."""
    P = np.asarray(points, dtype=np.float32)
    X = np.concatenate([P[0, :, :3], np.float32(w) * P[1, :, :3]], axis=1).astype(np.float32)
    off = np.asarray(slice_off, dtype=np.int64)
    perm = np.asarray(row_perm, dtype=np.int64)
    sl = [np.sort(perm[off[s]:off[s + 1]]) for s in range(off.size - 1)]

    def centroid(idx):
        c = np.zeros(6)
        for d in range(6):
            c[d] = np.cumsum(X[idx, d].astype(np.float64))[-1] / idx.size if idx.size else 0.0
        return c

    cents = [centroid(a) for a in sl]
    while len(sl) > 1:
        small = [s for s in range(len(sl)) if sl[s].size < min_rows]
        if not small:
            break
        s = min(small, key=lambda t: (sl[t].size, t))
        best, bd = -1, np.inf
        for t in range(len(sl)):
            if t == s:
                continue
            diff = cents[s] - cents[t]
            d2 = 0.0
            for v in diff:
                d2 = d2 + v * v
            if d2 < bd:
                best, bd = t, d2
        sl[best] = np.sort(np.concatenate([sl[best], sl[s]]))
        cents[best] = centroid(sl[best])
        del sl[s]
        del cents[s]
    out = []

    def split(idx):
        n = idx.size
        if n <= max_rows:
            out.append(idx)
            return
        ext = X[idx].max(axis=0) - X[idx].min(axis=0)
        d = int(np.argmax(ext))
        order = np.lexsort((idx, X[idx, d]))
        left = np.zeros(n, dtype=bool)
        left[order[:n // 2]] = True
        split(idx[left])
        split(idx[~left])

    for a in sl:
        split(a)
    row_perm_out = np.concatenate(out) if out else np.zeros(0, dtype=np.int64)
    off_out = np.concatenate([[0], np.cumsum([a.size for a in out])]).astype(np.int64)
    return row_perm_out, off_out
