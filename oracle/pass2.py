"""Second sampling pass: entries drawn from pdf(i, j) ~ f(i) g(j) (Sec. 5, Eq. 3).

Sec. 5 reuses the pass-1 entries and adds more until a prescribed count is reached:
a column is chosen by the light importance g, then a row (f(i) = 1, uniform); an
entry is computed only if it is not known yet.  Readings taken here:

* Target: T = ceil(rate * m' * n') observed entries in the slice (double precision,
  rate the float32 sampling rate); nothing is drawn when pass 1 already reached T.
* The column pdf is quantised to integers so that both sides draw identically:
  with w the column weights (g, or any other non-negative importance) and
  w_max = max w, q_c = 0 if w_c <= 0 else max(1, floor(float32(w_c / w_max) * 2^24)),
  the float32 ratio being the kernel's precision; if w_max <= 0 every q_c = 1.
  CDF = inclusive prefix sum of q (64-bit), total = CDF[n'-1].
* Draw t uses the Philox words (w0, w1) of counter (t, 0, slice, PASS2):
  u = floor(w0 * total / 2^32), column = first c with CDF[c] > u,
  row = floor(w1 * m' / 2^32).
* An entry is kept if it is neither a pass-1 entry nor an earlier kept draw; the
  first T - |Omega_1| kept draws in draw order form the pass-2 set.  At most
  64 T + 64 draws are made; a slice that runs out keeps what it has.
"""
from __future__ import annotations

import math

import numpy as np

from . import philox


def quantised_weights(w) -> np.ndarray:
    w = np.asarray(w, dtype=np.float32)
    if w.size == 0:
        return np.zeros(0, dtype=np.uint64)
    wmax = np.float32(w.max())
    if not wmax > 0:
        return np.ones(w.size, dtype=np.uint64)
    ratio = (w / wmax).astype(np.float32)
    q = np.floor((ratio * np.float32(16777216.0)).astype(np.float32)).astype(np.int64)
    q = np.where(w > 0, np.maximum(q, 1), 0)
    return q.astype(np.uint64)


def target_count(rate: float, m_s: int, n_s: int) -> int:
    return int(math.ceil(float(np.float32(rate)) * float(m_s) * float(n_s)))


def raw_draws(seed: int, s: int, m_s: int, cdf: np.ndarray, t: np.ndarray):
    """(row, column) of draws t (no de-duplication) from the integer CDF."""
    total = int(cdf[-1])
    w0, w1, _, _ = philox.draw(seed, np.asarray(t, dtype=np.uint64), 0, s, philox.TAG_PASS2)
    # exact floor(w0 * total / 2^32) in Python integers (the product needs > 64 bits)
    u = np.array([(int(x) * total) >> 32 for x in w0.tolist()], dtype=np.uint64)
    col = np.searchsorted(cdf, u, side="right")
    row = philox.uniform_index(w1, m_s)
    return row, col


def draw_pass2(seed: int, s: int, m_s: int, weights, observed_keys, rate: float):
    """Return (rows, cols, n_draws, hit_cap) of the pass-2 entries of slice s.

    ``observed_keys`` holds row * n' + col of the pass-1 entries.
    """
    n_s = len(weights)
    T = target_count(rate, m_s, n_s)
    seen = set(int(k) for k in observed_keys)
    need = T - len(seen)
    if need <= 0 or m_s == 0 or n_s == 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64), 0, False
    q = quantised_weights(weights)
    cdf = np.cumsum(q.astype(np.uint64))
    cap = 64 * T + 64
    rows, cols = [], []
    t0 = 0
    while len(rows) < need and t0 < cap:
        t = np.arange(t0, min(t0 + 4096, cap), dtype=np.uint64)
        row, col = raw_draws(seed, s, m_s, cdf, t)
        used = t.size
        for i, (r, c) in enumerate(zip(row.tolist(), col.tolist())):
            key = r * n_s + c
            if key not in seen:
                seen.add(key)
                rows.append(r)
                cols.append(c)
                if len(rows) == need:
                    used = i + 1
                    break
        t0 += used
    n_draws = t0
    return (np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64), n_draws,
            len(rows) < need)
