"""Temporal coherence across frames (lt_complete_warm) against the oracle: the start
of a frame's completion from the previous frame's factors (columns mapped by node,
copied exactly; the other columns seeded as lt_complete seeds them), and a chain of
two frames (the second started from the first with three sweeps) against the oracle
pipeline run the same way."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene
from oracle import als as o_als
from oracle import pipeline

pytestmark = pytest.mark.gpu

IMAGE_RTOL = 1e-3


@pytest.fixture(scope="module")
def tiny():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    cfg = get_config("room64_vpl1k_2box", max_cut=256)
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    return cfg, sc, st


def _renderer(cfg, sc, st):
    from paper_2202_12567_gb300.renderer import Renderer
    return Renderer(sc, cfg, device=0).setup(cut=st["cut"], row_perm=st["row_perm"], slice_off=st["slice_off"])


def test_warm_start_maps_the_previous_columns(tiny):
    from paper_2202_12567_gb300 import lt
    cfg, sc, st = tiny
    R = _renderer(cfg, sc, st)
    R.render(seed=7, warm=True)
    prev_node, prev_ncol, prev_V = (t.cpu().numpy() for t in R._prev)
    seed = 8
    R.pass1(seed)
    R.pass2(seed)
    R.evaluate()
    R.complete(seed, warm=True, iters=0)  # the start alone
    V = R.uv.V.view(R.frame.S, R.frame.C, cfg["rank"]).cpu().numpy().astype(np.float64)
    C, r = R.frame.C, cfg["rank"]
    matched = 0
    for s in range(R.frame.S):
        rows, cols, vals, col_node, g = R.smp.slice(s)
        n_s = col_node.size
        pn = prev_node[s * C:s * C + prev_ncol[s]]
        pV = prev_V.reshape(R.frame.S, C, r)[s, :prev_ncol[s]].astype(np.float64)
        want = o_als.warm_start(seed, s, col_node, vals, r, pn, pV)
        hit = np.isin(col_node, pn)
        matched += int(hit.sum())
        assert np.array_equal(V[s, :n_s][hit], want[hit]), s          # copied rows: exact
        np.testing.assert_allclose(V[s, :n_s][~hit], want[~hit], rtol=1e-5, atol=1e-7)  # seeded rows
    assert matched > 0
    lt.lt_sync(R.ctx)


def test_warm_chain_matches_oracle(tiny):
    cfg, sc, st = tiny
    R = _renderer(cfg, sc, st)
    R.render(seed=7, warm=True)
    img = R.render(seed=8, warm=True, iters=3).cpu().numpy().astype(np.float64)
    _, res7 = pipeline.render_frame(sc, cfg, st, seed=7)
    ref, _ = pipeline.render_frame(sc, dict(cfg, als_iters=3), st, seed=8, prev=res7)
    rel = np.linalg.norm(img - ref) / np.linalg.norm(ref)
    assert rel <= IMAGE_RTOL, rel


def test_warm_arguments(tiny):
    from paper_2202_12567_gb300 import lt
    cfg, sc, st = tiny
    R = _renderer(cfg, sc, st)
    R.render(seed=7, warm=True)
    node, ncol, V = R._prev
    with pytest.raises(lt.LtError):  # the previous V may not be the output V
        lt.lt_complete_warm(R.ctx, R.frame, R.smp, R.uv, 3, cfg["lam_rel"], 8, node, ncol, R.uv.V)
    lt.lt_sync(R.ctx)
