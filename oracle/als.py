"""Completion of one slice from its observed entries (Sec. 5; factor form M = X Y).

The paper completes each slice M (m' x n') as a product of rank-q factors fitted to
the sampled entries.  The completion used here is masked alternating least squares
(ALS) with a small ridge term, in float64.  With U = X (m' x r) and V = Y^T (n' x r):

* Initialisation: V0[j, k] = sqrt(mu / r) * (0.5 + w / 2^32), mu = mean observed
  value, w = word 0 of the Philox counter (k, j, slice, ALSINIT).
* One iteration = a U-step then a V-step.  U-step, for each row i with observed
  columns Omega_i:
      G_i = sum_{j in Omega_i} v_j v_j^T,   b_i = sum_{j in Omega_i} A_ij v_j,
      lambda_i = lam_rel * trace(G_i) / r,   u_i = (G_i + lambda_i I)^{-1} b_i;
  a row without entries, or with trace(G_i) = 0, gets u_i = 0.  The V-step is the
  same per column with the roles of U and V swapped.
* A fixed number of iterations is run (the paper stops on a tolerance or after 100).
* Across frames (warm_start): a column whose node was a column of the previous
  frame's slice starts from its previous V row.
"""
from __future__ import annotations

import numpy as np

from . import philox


def init_v(seed: int, s: int, n_s: int, r: int, mu: float) -> np.ndarray:
    k = np.arange(r, dtype=np.uint64)[None, :]
    j = np.arange(n_s, dtype=np.uint64)[:, None]
    w = philox.draw(seed, k, j, s, philox.TAG_ALSINIT)[0].astype(np.float64)
    return np.sqrt(max(mu, 0.0) / r) * (0.5 + w / 2.0 ** 32)


def warm_start(seed: int, s: int, col_node, vals, r: int, prev_col_node, prev_V) -> np.ndarray:
    """Start of a frame's completion from the previous frame's factors (temporal
    coherence, which the paper leaves to future work, Sec. 7; the form is ours): a
    column whose coarsened-cut node (tree node id) was also a column of the same slice
    in the previous frame starts from that column's V row (its first r components,
    zero beyond the previous rank), every other column from init_v."""
    vals = np.asarray(vals, dtype=np.float64)
    mu = float(vals.mean()) if vals.size else 0.0
    col_node = np.asarray(col_node)
    V = init_v(seed, s, col_node.size, r, mu)
    prev_V = np.asarray(prev_V, dtype=np.float64)
    where = {int(n): i for i, n in enumerate(np.asarray(prev_col_node).tolist())}
    for c, n in enumerate(col_node.tolist()):
        i = where.get(int(n))
        if i is not None:
            row = np.zeros(r)
            k = min(r, prev_V.shape[1])
            row[:k] = prev_V[i, :k]
            V[c] = row
    return V


def _half_step(idx_a, idx_b, vals, n_a, F, r, lam_rel):
    """Solve for the factor of side a given the fixed factor F of side b."""
    out = np.zeros((n_a, r))
    if vals.size == 0:
        return out
    order = np.argsort(idx_a, kind="stable")
    ia, ib, v = idx_a[order], idx_b[order], vals[order]
    starts = np.flatnonzero(np.r_[True, ia[1:] != ia[:-1]])
    owners = ia[starts]
    Fb = F[ib]                                   # [e, r]
    G = np.add.reduceat(Fb[:, :, None] * Fb[:, None, :], starts, axis=0)
    b = np.add.reduceat(Fb * v[:, None], starts, axis=0)
    tr = np.trace(G, axis1=1, axis2=2)
    ok = tr > 0
    lam = lam_rel * tr / r
    Greg = G + lam[:, None, None] * np.eye(r)[None]
    sol = np.zeros((owners.size, r))
    if np.any(ok):
        sol[ok] = np.linalg.solve(Greg[ok], b[ok][:, :, None])[:, :, 0]
    out[owners] = sol
    return out


def complete_slice(rows, cols, vals, m_s: int, n_s: int, r: int, iters: int, lam_rel: float,
                   seed: int, s: int, V0=None):
    """Masked ALS on one slice; returns (U [m', r], V [n', r]) in float64."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    mu = float(vals.mean()) if vals.size else 0.0
    V = init_v(seed, s, n_s, r, mu) if V0 is None else np.array(V0, dtype=np.float64)
    U = np.zeros((m_s, r))
    for _ in range(iters):
        U = _half_step(rows, cols, vals, m_s, V, r, lam_rel)
        V = _half_step(cols, rows, vals, n_s, U, r, lam_rel)
    return U, V
