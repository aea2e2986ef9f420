"""Learned second-pass proposal: features, training targets, the MLP, its gradients
and Adam, in float64 (test infrastructure: only tests/, the smoke check and the
CPU baseline of bench.py use this package).

The paper draws pass-2 columns from the pass-1 estimate g(j) (Sec. 5) and names a
learned importance as future work; this is that extension, with every choice below
our reading:

* Features of (slice s, coarsened column c), 32 values:
   0-2 mean shading-point position of the slice   3-5 mean normal of the slice
   6-8 slice AABB min                             9-11 slice AABB max
  12-14 AABB min of node c's VPLs                15-17 AABB max
  18-20 position of the representative VPL       21-23 its normal
  24    log(I_c / I_root)
  25    mean of the pass-1 values of column c / mu_s
  26    standard deviation (population) of them / mu_s
  27    log(1 + their count)
  28    min / mu_s                               29    max / mu_s
  30    log(m'_s) / 10                           31    log(n'_s) / 10
  with mu_s the mean of all pass-1 values of the slice (1 if it is not positive) and
  the statistics of a column without pass-1 values 0.
* Target of column c: leverage l_c = squared norm of row c of an orthonormal basis
  of the dominant rank-r right subspace of the slice matrix M (m' x n', entries
  A(i, c) with I_c, Sec. 3), found by K rounds of subspace iteration on G = M^T M
  from a Philox start (counter (k, c, s, 4), u in [-1/2, 1/2)), each round
  Q <- G Q then modified Gram-Schmidt (a column whose norm falls to zero is set
  to zero).  p_c = (l_c + 1/n') / sum.  Leverage sampling is the standard importance
  for low-rank completion; the subspace-iteration form makes the target a fixed
  computation that the GPU repeats.
* Network: 32 -> 64 -> 64 -> 64 -> 1, SiLU after each hidden layer.  Weights, inputs
  and hidden activations are rounded to bfloat16 (round to nearest even) before
  every product; biases, accumulation and the logit stay float32/float64.
* Loss: mean over slices of the cross-entropy between p and the softmax of the
  logits over the slice's columns.  Adam (beta 0.9 / 0.999, eps 1e-8).
* Runtime weight of column c: mix * softmax_c + (1 - mix) * g_c / sum g (mix 0.8).
"""
from __future__ import annotations

import numpy as np

from . import philox, shading
from .tree import node_scale

N_FEAT = 32
HIDDEN = 64
TAG_LEVERAGE = 4

# flat parameter layout (float32 master copy): W1[64][32] b1 W2[64][64] b2 W3[64][64] b3 W4[64] b4
SHAPES = [("W1", (HIDDEN, N_FEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (HIDDEN, HIDDEN)), ("b3", (HIDDEN,)), ("W4", (HIDDEN,)), ("b4", (1,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    theta = np.asarray(theta, dtype=np.float64)
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = theta[o:o + k].reshape(shp)
        o += k
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed: int) -> np.ndarray:
    """Uniform(+-1/sqrt(fan_in)) weights and zero biases from Philox (counter (i, 0, 0, 5))."""
    w = philox.draw(seed, np.arange(N_PARAM), 0, 0, 5)[0].astype(np.float64) * 2.0 ** -32 - 0.5
    parts, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        fan_in = shp[1] if len(shp) == 2 else HIDDEN
        parts[name] = (2.0 * w[o:o + k] / np.sqrt(fan_in)).reshape(shp) if name[0] == "W" else np.zeros(shp)
        o += k
    return pack(parts).astype(np.float32).astype(np.float64)


# ---------------------------------------------------------------- bfloat16
def bf16(x) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even) and back, as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    nan = np.isnan(f)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def silu(h):
    return h / (1.0 + np.exp(-h))


def dsilu(h):
    s = 1.0 / (1.0 + np.exp(-h))
    return s * (1.0 + h * (1.0 - s))


# ---------------------------------------------------------------- network
def forward(theta, X, rounding=True):
    """Logits [n] of features X [n][32]; returns (z, cache).  rounding=False gives the
    plain float64 network (for finite-difference checks)."""
    P = unpack(theta)
    q = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    x0 = q(X)
    W = [q(P["W1"]), q(P["W2"]), q(P["W3"]), q(P["W4"])]
    h1 = x0 @ W[0].T + P["b1"]
    a1 = q(silu(h1))
    h2 = a1 @ W[1].T + P["b2"]
    a2 = q(silu(h2))
    h3 = a2 @ W[2].T + P["b3"]
    a3 = q(silu(h3))
    z = a3 @ W[3] + P["b4"][0]
    return z, dict(x0=x0, W=W, h=(h1, h2, h3), a=(a1, a2, a3))


def backward(theta, cache, dz) -> np.ndarray:
    """Gradient of sum(dz * z) with respect to the parameters (the rounding is taken
    as the identity, as the GPU's straight-through update does)."""
    x0, W = cache["x0"], cache["W"]
    h1, h2, h3 = cache["h"]
    a1, a2, a3 = cache["a"]
    g = {}
    g["W4"] = dz @ a3
    g["b4"] = np.array([dz.sum()])
    d3 = np.outer(dz, W[3]) * dsilu(h3)
    g["W3"] = d3.T @ a2
    g["b3"] = d3.sum(0)
    d2 = (d3 @ W[2]) * dsilu(h2)
    g["W2"] = d2.T @ a1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ W[1]) * dsilu(h1)
    g["W1"] = d1.T @ x0
    g["b1"] = d1.sum(0)
    return pack(g)


def group_softmax(z, group_off):
    p = np.empty_like(z)
    for a, b in zip(group_off[:-1], group_off[1:]):
        if b > a:
            e = np.exp(z[a:b] - z[a:b].max())
            p[a:b] = e / e.sum()
    return p


def loss_and_dz(z, target, group_off):
    """Mean over groups of -sum_c p_c log softmax(z)_c, and its gradient in z."""
    G = len(group_off) - 1
    sm = group_softmax(z, group_off)
    loss = 0.0
    for a, b in zip(group_off[:-1], group_off[1:]):
        if b > a:
            zz = z[a:b] - z[a:b].max()
            loss -= float(np.dot(target[a:b], zz - np.log(np.exp(zz).sum())))
    return loss / G, (sm - target) / G


def adam(theta, m, v, grad, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def mixture(z, g, group_off, mix=0.8):
    """Pass-2 column weights: mix * slice softmax + (1 - mix) * g / sum g."""
    sm = group_softmax(z, group_off)
    w = np.empty_like(sm)
    for a, b in zip(group_off[:-1], group_off[1:]):
        gs = float(np.sum(g[a:b]))
        w[a:b] = mix * sm[a:b] + (1 - mix) * (g[a:b] / gs if gs > 0 else 1.0 / max(b - a, 1))
    return w


# ---------------------------------------------------------------- features
def slice_features(pts_s, row0: int, m_s: int, tree, vpls, col_node, p1_cols, p1_vals) -> np.ndarray:
    """[n'][32] features of one slice (layout in the module docstring)."""
    P = np.asarray(pts_s, dtype=np.float64)
    V = np.asarray(vpls, dtype=np.float64)
    pos = P[0, row0:row0 + m_s, :3]
    nrm = P[1, row0:row0 + m_s, :3]
    n_s = len(col_node)
    F = np.zeros((n_s, N_FEAT))
    if n_s == 0:
        return F
    vals = np.asarray(p1_vals, dtype=np.float64)
    mu = vals.mean() if vals.size else 0.0
    mu = mu if mu > 0 else 1.0
    root = 0
    F[:, 0:3] = pos.mean(0)
    F[:, 3:6] = nrm.mean(0)
    F[:, 6:9] = pos.min(0)
    F[:, 9:12] = pos.max(0)
    nodes = np.asarray(col_node, dtype=np.int64)
    F[:, 12:15] = tree.lo[nodes]
    F[:, 15:18] = tree.hi[nodes]
    rep = tree.rep[nodes]
    F[:, 18:21] = V[0, rep, :3]
    F[:, 21:24] = V[1, rep, :3]
    F[:, 24] = np.log(tree.I[nodes].astype(np.float64) / float(tree.I[root]))
    for c in range(n_s):
        v = vals[np.asarray(p1_cols) == c]
        if v.size:
            F[c, 25] = v.mean() / mu
            F[c, 26] = np.sqrt(np.mean((v - v.mean()) ** 2)) / mu
            F[c, 27] = np.log1p(v.size)
            F[c, 28] = v.min() / mu
            F[c, 29] = v.max() / mu
    F[:, 30] = np.log(m_s) / 10
    F[:, 31] = np.log(n_s) / 10
    return F


# ---------------------------------------------------------------- targets
def slice_matrix(pts_s, row0: int, m_s: int, tree, vpls, boxes, col_node, d_min: float) -> np.ndarray:
    """The full slice matrix M[i][c] = A(row0 + i, c) over the coarsened columns."""
    nodes = np.asarray(col_node, dtype=np.int64)
    n_s = nodes.size
    rows = np.repeat(np.arange(row0, row0 + m_s), n_s)
    cols = np.tile(np.arange(n_s), m_s)
    vals = shading.node_entries(pts_s, vpls, rows, tree.rep[nodes][cols], node_scale(tree, vpls, nodes)[cols],
                                boxes, d_min)
    return vals.reshape(m_s, n_s)


def subspace_start(seed: int, s: int, n_s: int, r: int) -> np.ndarray:
    k, c = np.meshgrid(np.arange(r), np.arange(n_s))
    w = philox.draw(seed, k, c, s, TAG_LEVERAGE)[0].astype(np.float64)
    return w * 2.0 ** -32 - 0.5


def mgs(Q):
    """Modified Gram-Schmidt on the columns (a column whose norm is 0 becomes 0)."""
    Q = Q.copy()
    for k in range(Q.shape[1]):
        for j in range(k):
            Q[:, k] -= np.dot(Q[:, j], Q[:, k]) * Q[:, j]
        nrm = np.linalg.norm(Q[:, k])
        Q[:, k] = Q[:, k] / nrm if nrm > 0 else 0.0
    return Q


def leverage(M, r: int, iters: int, seed: int, s: int) -> np.ndarray:
    """Row norms^2 of the basis after `iters` rounds of Q <- mgs(M^T M Q)."""
    n_s = M.shape[1]
    r = min(r, n_s)
    G = M.T @ M
    Q = mgs(subspace_start(seed, s, n_s, r))
    for _ in range(iters):
        Q = mgs(G @ Q)
    return np.sum(Q * Q, axis=1)


def targets(lev) -> np.ndarray:
    n_s = lev.size
    t = lev + 1.0 / n_s
    return t / t.sum()
