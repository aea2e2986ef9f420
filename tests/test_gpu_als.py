"""Masked ALS (lt_complete) against the float64 oracle beyond the tiny workload.

* Slices of the full-size bench workload (256x256 points, 16384 VPLs, 64 slices,
  rank 16, about 95 entries a row and 150 a column) completed again by the oracle
  from the GPU's own samples: the first, a middle and the largest slice, whose lines
  take every group-size class and the persistent kernel's slice segments.
* Lines whose float32 Cholesky fails the pivot check: rows observed in fewer
  entries than the rank with a ridge of 1e-9 have a rank-deficient Gram (pivot
  ratio far below 1e-6); the library solves them again in float64 with their Gram
  formed in float64.  The count of such lines is read back through the C ABI and
  the factors must still match the oracle.

Tolerance (the completion row of the parity table): the completed image and each
slice's completed matrix within 1e-3 of the oracle's after the same iterations.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene
from oracle import als as o_als

pytestmark = pytest.mark.gpu

IMAGE_RTOL = 1e-3
SLICE_RTOL = 1e-3


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room256_vpl16k_2box")
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=0).setup()
    R.render()
    return cfg, sc, R


def test_als_full_size_sampled_slices(full):
    """Three slices of the bench workload completed again by the oracle from the
    GPU's entries: pixels and completed matrix within 1e-3."""
    cfg, sc, R = full
    off = R.slice_off.cpu().numpy()
    perm = R.row_perm.cpu().numpy()
    img = R.img.cpu().numpy().astype(np.float64)
    r = cfg["rank"]
    U = R.uv.U.cpu().numpy().reshape(-1, r).astype(np.float64)
    V = R.uv.V.cpu().numpy().reshape(R.frame.S, R.frame.C, r).astype(np.float64)
    sizes = np.diff(off)
    for s in sorted({0, R.frame.S // 2, int(np.argmax(sizes))}):
        rows, cols, vals, col_node, _ = R.smp.slice(s)
        m_s, n_s = int(sizes[s]), col_node.size
        Uo, Vo = o_als.complete_slice(rows, cols, vals.astype(np.float64), m_s, n_s, r, cfg["als_iters"],
                                      cfg["lam_rel"], cfg["frame_seed"], s)
        pix_o = np.maximum(Uo @ Vo.sum(axis=0), 0.0)
        pix_g = img[perm[off[s]:off[s + 1]]]
        assert np.linalg.norm(pix_g - pix_o) <= IMAGE_RTOL * np.linalg.norm(pix_o), s
        Mo = Uo @ Vo.T
        Mg = U[off[s]:off[s + 1]] @ V[s, :n_s].T
        assert np.linalg.norm(Mg - Mo) <= SLICE_RTOL * np.linalg.norm(Mo), s


class _Synthetic:
    """A frame of S slices of m_s rows and n_s columns with given observed entries
    (the completion reads only the slice layout and the entries)."""

    def __init__(self, lt, entries, m_s, n_s, r):
        S = len(entries)
        dev = torch.device("cuda", 0)
        self.slice_off = torch.arange(0, (S + 1) * m_s, m_s, dtype=torch.int32, device=dev)
        self.frame = lt.lt_frame(None, S * m_s, None, 0, lt._ptr(self.slice_off), S, m_s, lt.lt_tree(), n_s,
                                 None, None, None, 0)
        caps = [len(e[0]) for e in entries]
        off = np.concatenate([[0], np.cumsum(caps)]).astype(np.int64)
        key = np.concatenate([(rr.astype(np.uint32) << 16) | cc.astype(np.uint32) for rr, cc, _ in entries])
        val = np.concatenate([v for _, _, v in entries]).astype(np.float32)
        i32 = dict(dtype=torch.int32, device=dev)
        self.ncol = torch.full((S,), n_s, **i32)
        self.col_node = torch.zeros(S * n_s, **i32)
        self.g = torch.zeros(S * n_s, dtype=torch.float32, device=dev)
        self.off = torch.from_numpy(off).to(dev)
        self.key = torch.from_numpy(key.view(np.int32)).to(dev)
        self.val = torch.from_numpy(val).to(dev)
        self.n1 = torch.zeros(S, **i32)
        self.cnt = torch.tensor(caps, **i32)
        self.smp = lt.lt_samples(lt._ptr(self.ncol), lt._ptr(self.col_node), lt._ptr(self.g), lt._ptr(self.off),
                                 lt._ptr(self.key), lt._ptr(self.val), lt._ptr(self.n1), lt._ptr(self.cnt))
        self.U = torch.zeros(S * m_s * r, dtype=torch.float32, device=dev)
        self.V = torch.zeros(S * n_s * r, dtype=torch.float32, device=dev)
        self.uv = lt.lt_factors(r, lt._ptr(self.U), lt._ptr(self.V), None)


def _thin_row_slices(rng, S, m_s, n_s, r, thin_every, k_thin, k_full):
    """Entries of an exactly rank-r positive matrix per slice: every thin_every-th
    row observes k_thin < r columns, the others k_full >= 3r."""
    out = []
    for _ in range(S):
        X = rng.uniform(0.2, 1.0, (m_s, r))
        Y = rng.uniform(0.2, 1.0, (n_s, r))
        rows, cols = [], []
        for i in range(m_s):
            k = k_thin if i % thin_every == 0 else k_full
            c = np.sort(rng.choice(n_s, k, replace=False))
            rows.append(np.full(k, i))
            cols.append(c)
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        out.append((rows, cols, np.sum(X[rows] * Y[cols], axis=1)))
    return out


@pytest.mark.parametrize("r,form", [(8, 1), (8, 0), (16, 1), (16, 0), (18, 0), (32, 0)])
def test_als_float64_retry_on_rank_deficient_rows(r, form):
    """Rows with fewer entries than the rank and a ridge of 1e-9 fail the float32
    pivot check; the float64 pass solves them and the result matches the oracle
    (r <= 16: both forms of the half-step, tensor cores and lane-group SIMT; r = 18
    and 32: the warp-per-line kernel, with factor rows of stride 18 read by scalar
    loads and of stride 32 by 16-byte loads)."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300 import lt
    lt.load()
    ctx = lt.Context(0)
    lt.lt_set_tuning(ctx, als_form=form)
    S, m_s, n_s, iters, lam, seed = 3, 200, 3 * r + 16, 4, 1e-9, 11
    thin_every, k_thin, k_full = 5, r // 2, 3 * r + 4
    entries = _thin_row_slices(np.random.default_rng(r), S, m_s, n_s, r, thin_every, k_thin, k_full)
    syn = _Synthetic(lt, entries, m_s, n_s, r)
    ctx._check("lt_complete", ctx.lib.lt_complete(ctx.h, ctypes.byref(syn.frame), ctypes.byref(syn.smp), iters,
                                                  lam, seed, ctypes.byref(syn.uv)))
    lt.lt_sync(ctx)
    n64 = lt.lt_complete_fp64_lines(ctx)
    thin_rows = S * ((m_s + thin_every - 1) // thin_every)
    # every thin row, in every U-step, takes the float64 path
    assert n64 >= thin_rows * iters, (n64, thin_rows * iters)
    U = syn.U.cpu().numpy().reshape(S, m_s, r).astype(np.float64)
    V = syn.V.cpu().numpy().reshape(S, n_s, r).astype(np.float64)
    for s, (rows, cols, vals) in enumerate(entries):
        vals32 = vals.astype(np.float32).astype(np.float64)
        Uo, Vo = o_als.complete_slice(rows, cols, vals32, m_s, n_s, r, iters, lam, seed, s)
        Mo = Uo @ Vo.T
        Mg = U[s] @ V[s].T
        assert np.linalg.norm(Mg - Mo) <= SLICE_RTOL * np.linalg.norm(Mo), s
        thin = np.arange(0, m_s, thin_every)
        assert np.linalg.norm(U[s][thin] - Uo[thin]) <= SLICE_RTOL * np.linalg.norm(Uo[thin]), s
        pix_o, pix_g = Uo @ Vo.sum(axis=0), U[s] @ V[s].sum(axis=0)
        assert np.linalg.norm(pix_g - pix_o) <= IMAGE_RTOL * np.linalg.norm(pix_o), s
    ctx.close()


def test_fp64_lines_are_rare_on_the_bench_frame(full):
    """The bench frame (ridge 1e-2) solves at most 0.1% of its lines in float64."""
    cfg, sc, R = full
    from paper_2202_12567_gb300 import lt
    R.complete(cfg["frame_seed"])
    lines = cfg["als_iters"] * (R.frame.m + int(R.smp.ncol.sum().item()))
    n64 = lt.lt_complete_fp64_lines(R.ctx)
    print(f"float64 lines: {n64} of {lines}")
    assert n64 <= 1e-3 * lines
