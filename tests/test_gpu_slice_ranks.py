"""Per-slice ranks (a rank 8..32 chosen from each slice's coarsened cut): the rank
rule and the completed image against the oracle pipeline with the same rule, with
slices on both ALS kernels (lane groups up to rank 16, warp groups above)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene
from oracle import pipeline

pytestmark = pytest.mark.gpu

IMAGE_RTOL = 1e-3


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    cfg = get_config("room64_vpl1k_2box", max_cut=256, rank=32, rank_cols=30)
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    return cfg, sc, st


def test_rank_rule_matches_oracle_and_mixes_paths(setup):
    from paper_2202_12567_gb300 import lt
    from paper_2202_12567_gb300.renderer import Renderer
    cfg, sc, st = setup
    R = Renderer(sc, cfg, device=0).setup(cut=st["cut"], row_perm=st["row_perm"], slice_off=st["slice_off"])
    R.pass1(cfg["frame_seed"])
    rk = lt.lt_slice_ranks(R.ctx, R.frame, R.smp, cfg["rank"], cfg["rank_cols"]).cpu().numpy()
    ncol = R.smp.ncol.cpu().numpy()
    want = np.array([pipeline.slice_rank(cfg, n) for n in ncol])
    assert np.array_equal(rk, want)
    assert rk.min() <= 16 < rk.max()  # both ALS kernels take part


def test_per_slice_rank_frame_matches_oracle(setup):
    from paper_2202_12567_gb300.renderer import Renderer
    cfg, sc, st = setup
    R = Renderer(sc, cfg, device=0).setup(cut=st["cut"], row_perm=st["row_perm"], slice_off=st["slice_off"])
    img = R.render().cpu().numpy().astype(np.float64)
    ref_img, res = pipeline.render_frame(sc, cfg, st)
    rel = np.linalg.norm(img - ref_img) / np.linalg.norm(ref_img)
    assert rel <= IMAGE_RTOL, rel
    # components beyond a slice's rank are zero
    U = R.uv.U.view(-1, cfg["rank"]).cpu().numpy()
    rk = R.uv.rank.cpu().numpy()
    off = st["slice_off"]
    for s in range(len(rk)):
        assert np.all(U[off[s]:off[s + 1], rk[s]:] == 0)


def test_per_slice_rank_graph_replays_the_frame(setup):
    from paper_2202_12567_gb300 import lt
    from paper_2202_12567_gb300.renderer import Renderer
    cfg, sc, st = setup
    R = Renderer(sc, cfg, device=0).setup()
    plain = R.render_frame(seed=3).clone()
    g = R.capture()
    assert torch.equal(R.render_graph(seed=3), plain)
    g.close()
    R.graph = None
