"""Light tree over the VPLs (Sec. 3 step 1; Sec. 4).

The paper adopts the light tree of the lightcuts papers without giving a build.
The reading taken here is a binary radix tree over Morton codes of the VPL
positions (the linear-BVH construction of Karras, HPG 2012):

* Morton code: each coordinate is normalised to the VPL bounding box in float32,
  x = (p - lo) / (hi - lo), quantised to q = clamp(floor(x * 1024), 0, 1023) and the
  three 10-bit integers are bit-interleaved (x highest).  Float32 is used because
  the code is an integer decided by floating point; both sides decide it in the
  precision of the GPU kernel.
* The orientation class of the VPL normal (the cube face it points to,
  2 * dominant axis + (component > 0)) is placed above the 30 Morton bits, so that
  no cluster mixes lights facing different ways (the lightcuts trees cluster oriented
  lights by position and direction).
* Keys ((class << 30 | code) << 32 | vpl index) are unique; the leaves are the VPLs
  in key order.
* Internal node i (0 <= i < n-1) covers the key range found by Karras's search and
  splits it at the highest differing bit.  Node ids: internal nodes 0..n-2 (root 0),
  leaf j is node n-1+j.
* Records, bottom-up: intensity I = flux * albedo for a VPL and I_f = I_a + I_b for
  a parent (Sec. 4), in float32 with that exact operation order; the bounding box;
  the BRDF bound B = max over the node's VPLs of f_max / albedo; the representative
  rep(f) = rep of the child with the larger I, ties to the left child (Sec. 4 lets
  the parent "be the same as" one child except for intensity).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .shading import brdf_max


@dataclasses.dataclass
class LightTree:
    n: int
    order: np.ndarray      # [n] VPL index of leaf j
    child: np.ndarray      # [2n-1, 2] node ids, -1 for leaves
    parent: np.ndarray     # [2n-1], -1 for the root
    first: np.ndarray      # [2n-1] first leaf index covered
    last: np.ndarray       # [2n-1] last leaf index covered
    I: np.ndarray          # [2n-1] float32 intensity
    B: np.ndarray          # [2n-1] BRDF bound (float64)
    lo: np.ndarray         # [2n-1, 3] float32
    hi: np.ndarray         # [2n-1, 3] float32
    rep: np.ndarray        # [2n-1] representative VPL index

    @property
    def n_nodes(self) -> int:
        return 2 * self.n - 1

    def is_leaf(self, node) -> np.ndarray:
        return np.asarray(node) >= self.n - 1

    def leaf_node(self, j):
        return self.n - 1 + np.asarray(j)


def _expand10(v: np.ndarray) -> np.ndarray:
    """Spread the low 10 bits of v so that bit b moves to bit 3b."""
    v = v.astype(np.uint64)
    out = np.zeros_like(v)
    for b in range(10):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def morton_codes(pos: np.ndarray) -> np.ndarray:
    """30-bit Morton codes of float32 positions [k, 3], normalised to their bounding box."""
    pos = np.asarray(pos, dtype=np.float32)
    lo = pos.min(axis=0)
    hi = pos.max(axis=0)
    ext = (hi - lo).astype(np.float32)
    ext = np.where(ext > 0, ext, np.float32(1.0)).astype(np.float32)
    x = ((pos - lo).astype(np.float32) / ext).astype(np.float32)
    q = np.floor(x * np.float32(1024.0)).astype(np.int64)
    q = np.clip(q, 0, 1023)
    return (_expand10(q[:, 0]) << np.uint64(2)) | (_expand10(q[:, 1]) << np.uint64(1)) | _expand10(q[:, 2])


def orientation_class(nrm: np.ndarray) -> np.ndarray:
    """Cube face the normal points to: 2 * dominant axis + (component > 0), in 0..5.

    The dominant axis is the first axis of largest absolute component."""
    nrm = np.asarray(nrm, dtype=np.float32)
    ax = np.argmax(np.abs(nrm), axis=1)
    pos = nrm[np.arange(nrm.shape[0]), ax] > 0
    return (2 * ax + pos).astype(np.uint64)


def _clz64(x: int) -> int:
    return 64 - int(x).bit_length()


def build(vpls: np.ndarray) -> LightTree:
    """Build the light tree of the VPLs ``vpls[3, n, 4]``."""
    V = np.asarray(vpls, dtype=np.float32)
    n = V.shape[1]
    if n < 1:
        raise ValueError("need at least one VPL")
    codes = morton_codes(V[0, :, :3]) | (orientation_class(V[1, :, :3]) << np.uint64(30))
    keys = (codes << np.uint64(32)) | np.arange(n, dtype=np.uint64)
    order = np.argsort(keys, kind="stable")
    skeys = [int(k) for k in keys[order]]

    N = 2 * n - 1
    child = np.full((N, 2), -1, dtype=np.int64)
    parent = np.full(N, -1, dtype=np.int64)
    first = np.zeros(N, dtype=np.int64)
    last = np.zeros(N, dtype=np.int64)

    def delta(i, j):
        if j < 0 or j > n - 1:
            return -1
        return _clz64(skeys[i] ^ skeys[j])

    # Karras (2012): each internal node finds its range and split independently.
    for i in range(n - 1):
        d = 1 if delta(i, i + 1) - delta(i, i - 1) > 0 else -1
        dmin = delta(i, i - d)
        lmax = 2
        while delta(i, i + lmax * d) > dmin:
            lmax *= 2
        l = 0
        t = lmax // 2
        while t >= 1:
            if delta(i, i + (l + t) * d) > dmin:
                l += t
            t //= 2
        j = i + l * d
        dnode = delta(i, j)
        s = 0
        div = 2
        while True:
            t = (l + div - 1) // div
            if delta(i, i + (s + t) * d) > dnode:
                s += t
            if t <= 1:
                break
            div *= 2
        gamma = i + s * d + min(d, 0)
        a, b = min(i, j), max(i, j)
        left = (n - 1 + gamma) if a == gamma else gamma
        right = (n - 1 + gamma + 1) if b == gamma + 1 else gamma + 1
        child[i] = (left, right)
        parent[left] = i
        parent[right] = i
        first[i], last[i] = a, b
    for j in range(n):
        first[n - 1 + j] = last[n - 1 + j] = j

    I = np.zeros(N, dtype=np.float32)
    B = np.zeros(N, dtype=np.float64)
    lo = np.zeros((N, 3), dtype=np.float32)
    hi = np.zeros((N, 3), dtype=np.float32)
    rep = np.zeros(N, dtype=np.int64)
    leaf = n - 1 + np.arange(n)
    flux = V[2, order, 3]
    alb = V[0, order, 3]
    I[leaf] = (flux * alb).astype(np.float32)
    B[leaf] = brdf_max(alb.astype(np.float64), V[1, order, 3].astype(np.float64)) / np.maximum(
        alb.astype(np.float64), 1e-30)
    lo[leaf] = V[0, order, :3]
    hi[leaf] = V[0, order, :3]
    rep[leaf] = order
    # children always cover strictly smaller ranges: visit parents by range size
    inner = np.arange(n - 1)
    for f in inner[np.argsort(last[inner] - first[inner], kind="stable")]:
        a, b = child[f]
        I[f] = np.float32(I[a] + I[b])
        B[f] = max(B[a], B[b])
        lo[f] = np.minimum(lo[a], lo[b])
        hi[f] = np.maximum(hi[a], hi[b])
        rep[f] = rep[a] if I[a] >= I[b] else rep[b]
    return LightTree(n=n, order=order.astype(np.int64), child=child, parent=parent, first=first,
                     last=last, I=I, B=B, lo=lo, hi=hi, rep=rep)


def node_scale(tree: LightTree, vpls: np.ndarray, nodes) -> np.ndarray:
    """I_c / I_rep(c): the factor that turns A(i, rep(c)) into A(i, c)."""
    nodes = np.asarray(nodes, dtype=np.int64)
    V = np.asarray(vpls, dtype=np.float32)
    r = tree.rep[nodes]
    i_rep = (V[2, r, 3] * V[0, r, 3]).astype(np.float32).astype(np.float64)
    return tree.I[nodes].astype(np.float64) / np.maximum(i_rep, 1e-300)


def primary_child(tree: LightTree, f):
    """(p, q): p is the child whose representative the parent inherits, q the other."""
    a, b = tree.child[f]
    return (a, b) if tree.I[a] >= tree.I[b] else (b, a)
