"""The paper's recursive 6-D binary split slicing on the GPU against the oracle:
identical permutation and slice offsets on several scenes and targets (the split is
exact integer and float32-min/max work plus a radix select, so it is bit-exact), the
one-slice and one-pixel-slice limits, and a frame on split slices against the
oracle pipeline."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene
from oracle import pipeline
from oracle import slices as o_slices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300 import lt
    return lt.Context(0)


def _check(ctx, sc, target, w=0.3):
    from paper_2202_12567_gb300 import lt
    pts = torch.from_numpy(np.ascontiguousarray(sc.points)).cuda()
    perm, off = lt.lt_make_slices_split(ctx, pts, target, w)
    want_perm, want_off = o_slices.split6d_slices(sc.points, target, w)
    assert np.array_equal(off.cpu().numpy(), want_off)
    assert np.array_equal(perm.cpu().numpy(), want_perm)
    return off.cpu().numpy()


@pytest.mark.parametrize("target", [100, 256, 800, 1000])
def test_split_matches_oracle_tiny(ctx, target):
    sc = make_scene(get_config("room64_vpl1k_2box"))
    _check(ctx, sc, target)


@pytest.mark.parametrize("name", ["room256_vpl16k_2box", "room256_vpl16k_200box"])
def test_split_matches_oracle_full_size(ctx, name):
    sc = make_scene(get_config(name))
    off = _check(ctx, sc, 800)
    assert len(off) - 1 == 128 and np.diff(off).max() <= 800


def test_split_limits(ctx):
    sc = make_scene(get_config("room64_vpl1k_2box", width=16, height=16, n_vpl=64))
    off = _check(ctx, sc, 1000)  # m <= target: one slice
    assert off.tolist() == [0, 256]
    off = _check(ctx, sc, 1)     # one pixel per slice
    assert len(off) == 257
    _check(ctx, sc, 3, w=0.0)    # normals ignored


def test_frame_on_split_slices_matches_oracle_pipeline():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room64_vpl1k_2box", slicing="split6d", slice_size=300)
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    R = Renderer(sc, cfg, device=0).setup(cut=st["cut"])
    assert np.array_equal(R.slice_off.cpu().numpy(), st["slice_off"])
    assert np.array_equal(R.row_perm.cpu().numpy(), st["row_perm"])
    img = R.render().cpu().numpy().astype(np.float64)
    ref, _ = pipeline.render_frame(sc, cfg, st)
    rel = np.linalg.norm(img - ref) / np.linalg.norm(ref)
    assert rel <= 1e-3, rel
