"""The ADM nonnegative completion (App. A) on the GPU against the float64 oracle on
the same observed entries: same start, same iteration count, every rank path of the
kernel, per-slice ranks, empty and tiny slices, determinism, argument checks, and
sampled slices of the full-size workload.

Tolerance: the oracle run in float32 drifts from float64 by at most 5e-6 in the
image after 100 iterations on the tiny workload; the GPU form reorders the same
arithmetic (sparse residual, X step as X_k + t (A + alpha I)^-1, Gauss-Jordan
inverses), so the image must agree within 1e-4 and each slice's completed matrix
within 1e-3."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene
from oracle import adm as o_adm
from oracle import pipeline
from oracle import render as o_render

pytestmark = pytest.mark.gpu

IMAGE_RTOL = 1e-4
SLICE_RTOL = 1e-3


def _cfg(**kw):
    base = dict(completion="adm", adm_iters=100, adm_alpha_rel=0.3, adm_gamma=1.0)
    base.update(kw)
    return get_config("room64_vpl1k_2box", **base)


@pytest.fixture(scope="module")
def tiny():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    cfg = _cfg()
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    return cfg, sc, st


def _renderer(cfg, sc, st):
    from paper_2202_12567_gb300.renderer import Renderer
    return Renderer(sc, cfg, device=0).setup(cut=st["cut"], row_perm=st["row_perm"], slice_off=st["slice_off"])


def _oracle_on_gpu_samples(R, cfg, st, ranks=None):
    """The oracle's ADM on the entries the GPU sampled and evaluated."""
    factors = []
    for s in range(R.frame.S):
        rows, cols, vals, col_node, _ = R.smp.slice(s)
        m_s = int(st["slice_off"][s + 1] - st["slice_off"][s])
        r = cfg["rank"] if ranks is None else int(ranks[s])
        X, YT = o_adm.complete_slice_adm(rows, cols, vals.astype(np.float64), m_s, col_node.size, r,
                                         cfg["adm_iters"], cfg["adm_alpha_rel"], cfg["adm_gamma"],
                                         cfg["frame_seed"], s)
        factors.append((X, YT))
    return factors


def _gpu_factors(R, cfg, st):
    r = cfg["rank"]
    U = R.uv.U.cpu().numpy().reshape(-1, r).astype(np.float64)
    V = R.uv.V.cpu().numpy().reshape(R.frame.S, R.frame.C, r).astype(np.float64)
    ncol = R.smp.ncol.cpu().numpy()
    off = st["slice_off"]
    return [(U[off[s]:off[s + 1]], V[s, :ncol[s]]) for s in range(R.frame.S)]


def _compare(R, cfg, st, sc, ranks=None):
    from paper_2202_12567_gb300 import lt
    lt.lt_sync(R.ctx)
    img = R.img.cpu().numpy().astype(np.float64)
    want = _oracle_on_gpu_samples(R, cfg, st, ranks)
    ref = o_render.render_slices(want, st["row_perm"], st["slice_off"], sc.m)
    rel = np.linalg.norm(img - ref) / np.linalg.norm(ref)
    assert rel <= IMAGE_RTOL, rel
    got = _gpu_factors(R, cfg, st)
    for s, ((Xg, Yg), (Xo, Yo)) in enumerate(zip(got, want)):
        Mo = Xo @ Yo[:, :Xo.shape[1]].T
        Mg = Xg[:, :Xo.shape[1]] @ Yg[:, :Xo.shape[1]].T
        den = max(np.linalg.norm(Mo), 1e-30)
        assert np.linalg.norm(Mg - Mo) <= SLICE_RTOL * den, f"slice {s}"
    return rel


@pytest.mark.parametrize("iters", [0, 1, 2, 25, 100])
def test_adm_matches_oracle_on_the_same_samples(tiny, iters):
    cfg, sc, st = tiny
    cfg = dict(cfg, adm_iters=iters)
    R = _renderer(cfg, sc, st)
    R.render()
    _compare(R, cfg, st, sc)


@pytest.mark.parametrize("rank", [10, 16, 32])
def test_adm_rank_paths(tiny, rank):
    """rank 10: factor rows not a multiple of 4 (scalar loads); 16 and 32: the other
    register widths of the kernel."""
    cfg, sc, st = tiny
    cfg = dict(cfg, rank=rank, adm_iters=20)
    R = _renderer(cfg, sc, st)
    R.render()
    _compare(R, cfg, st, sc)


def test_adm_per_slice_ranks(tiny):
    from paper_2202_12567_gb300 import lt
    cfg, sc, st = tiny
    cfg = dict(cfg, rank=32, rank_cols=30, adm_iters=30)
    R = _renderer(cfg, sc, st)
    R.render()
    lt.lt_sync(R.ctx)
    rk = R.uv.rank.cpu().numpy()
    assert rk.min() < rk.max()
    _compare(R, cfg, st, sc, ranks=rk)
    U = R.uv.U.view(-1, cfg["rank"]).cpu().numpy()
    off = st["slice_off"]
    for s in range(len(rk)):
        assert np.all(U[off[s]:off[s + 1], rk[s]:] == 0)


def test_adm_is_deterministic(tiny):
    cfg, sc, st = tiny
    R = _renderer(cfg, sc, st)
    a = R.render().clone()
    U = R.uv.U.clone()
    b = R.render().clone()
    assert torch.equal(a, b) and torch.equal(U, R.uv.U)


def test_adm_graph_replays_the_frame(tiny):
    """The ADM completion inside the captured frame graph replays the one-call frame."""
    cfg, sc, st = tiny
    R = _renderer(cfg, sc, st)
    plain = R.render_frame(seed=5).clone()
    R.capture()
    assert torch.equal(R.render_graph(seed=5), plain)
    R.graph.close()
    R.graph = None


def test_adm_rejects_bad_arguments(tiny):
    from paper_2202_12567_gb300 import lt
    cfg, sc, st = tiny
    R = _renderer(cfg, sc, st)
    R.pass1(1)
    R.pass2(1)
    R.evaluate()
    for iters, ar, g in [(-1, 0.3, 1.0), (5, 0.0, 1.0), (5, -1.0, 1.0), (5, 0.3, 0.0), (5, 0.3, 1.7)]:
        with pytest.raises(RuntimeError):
            lt.lt_complete_adm(R.ctx, R.frame, R.smp, R.uv, iters, ar, g, 1)


def test_adm_empty_and_tiny_slices():
    """Slices with 0, 1 and 2 rows and a one-node cut run and give finite images; a
    slice without entries gets zero factors."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = _cfg(adm_iters=7)
    sc = make_scene(cfg)
    m = sc.m
    perm = np.arange(m, dtype=np.int32)
    off = np.array([0, 0, 1, 3, m // 2, m], dtype=np.int32)
    for cut in (np.array([0], dtype=np.int32), None):
        if cut is None:
            cut = pipeline.setup(sc, cfg)["cut"]
        R = Renderer(sc, dict(cfg, n_slices=5), device=0).setup(cut=cut, row_perm=perm, slice_off=off)
        img = R.render().cpu().numpy()
        assert np.all(np.isfinite(img)) and img.max() > 0


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room256_vpl16k_2box", completion="adm", adm_iters=100)
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=0).setup()
    R.render()
    return cfg, sc, R


def test_adm_full_size_sampled_slices(full):
    """The bench workload (256x256 points, 16384 VPLs, 64 slices): three slices
    completed again by the oracle from the GPU's entries."""
    cfg, sc, R = full
    off = R.slice_off.cpu().numpy()
    perm = R.row_perm.cpu().numpy()
    img = R.img.cpu().numpy().astype(np.float64)
    r = cfg["rank"]
    U = R.uv.U.cpu().numpy().reshape(-1, r).astype(np.float64)
    V = R.uv.V.cpu().numpy().reshape(R.frame.S, R.frame.C, r).astype(np.float64)
    for s in (0, R.frame.S // 2, R.frame.S - 1):
        rows, cols, vals, col_node, _ = R.smp.slice(s)
        m_s = int(off[s + 1] - off[s])
        X, YT = o_adm.complete_slice_adm(rows, cols, vals.astype(np.float64), m_s, col_node.size, r,
                                         cfg["adm_iters"], cfg["adm_alpha_rel"], cfg["adm_gamma"],
                                         cfg["frame_seed"], s)
        pix_o = np.maximum(X @ YT.sum(axis=0), 0.0)
        pix_g = img[perm[off[s]:off[s + 1]]]
        assert np.linalg.norm(pix_g - pix_o) <= 10 * IMAGE_RTOL * np.linalg.norm(pix_o), s
        Mo = X @ YT.T
        Mg = U[off[s]:off[s + 1]] @ V[s, :col_node.size].T
        assert np.linalg.norm(Mg - Mo) <= SLICE_RTOL * np.linalg.norm(Mo), s
