"""Slices held between two row counts (lt_bound_slices) against the oracle: from the
same starting slices, small slices merged into the nearest by centroid and large
ones split by the recursive 6-D median split give the identical permutation and slice
offsets (index work with float64 centroid sums in a fixed order: bit-exact), on the
tiny scene's k-means slices and on the GPU k-means slices of a full-size scene; the
renderer's frame on bounded slices equals the same frame given those slices."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene
from oracle import slices as o_slices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300 import lt
    return lt.Context(0)


def _check(ctx, sc, perm0, off0, lo, hi, w=0.3):
    from paper_2202_12567_gb300 import lt
    pts = torch.from_numpy(np.ascontiguousarray(sc.points)).cuda()
    perm, off = lt.lt_bound_slices(ctx, pts, torch.as_tensor(perm0, dtype=torch.int32).cuda(),
                                   torch.as_tensor(off0, dtype=torch.int32).cuda(), lo, hi, w)
    want_perm, want_off = o_slices.bound_slices(sc.points, np.asarray(perm0), np.asarray(off0), lo, hi, w)
    assert np.array_equal(off.cpu().numpy(), want_off)
    assert np.array_equal(perm.cpu().numpy(), want_perm)
    return off.cpu().numpy()


def test_bounds_match_oracle_tiny(ctx):
    sc = make_scene(get_config("room64_vpl1k_2box"))
    perm0, off0, _, _ = o_slices.kmeans_slices(sc.points, 16, 10, 0.3)
    off = _check(ctx, sc, perm0, off0, 200, 300)
    assert len(off) - 1 != 16  # merges and splits took place
    _check(ctx, sc, perm0, off0, 1, 4096)       # loose bounds: the slices as given
    _check(ctx, sc, perm0, off0, 4096, 4096)    # everything merged into one slice


def test_bounds_match_oracle_full_size(ctx):
    from paper_2202_12567_gb300 import lt
    cfg = get_config("room256_vpl16k_200box")
    sc = make_scene(cfg)
    pts = torch.from_numpy(np.ascontiguousarray(sc.points)).cuda()
    perm0, off0 = lt.lt_make_slices(ctx, pts, 64, 10, 0.3)
    sizes = np.diff(off0.cpu().numpy())
    lo, hi = int(np.percentile(sizes, 25)), int(np.percentile(sizes, 75))
    off = _check(ctx, sc, perm0.cpu().numpy(), off0.cpu().numpy(), lo, max(hi, 2 * lo))
    assert np.diff(off).min() >= lo and np.diff(off).max() <= max(hi, 2 * lo)


def test_bad_arguments_are_refused(ctx):
    from paper_2202_12567_gb300 import lt
    sc = make_scene(get_config("room64_vpl1k_2box", width=16, height=16, n_vpl=64))
    pts = torch.from_numpy(np.ascontiguousarray(sc.points)).cuda()
    perm = torch.arange(256, dtype=torch.int32).cuda()
    with pytest.raises(lt.LtError):
        lt.lt_bound_slices(ctx, pts, perm, torch.tensor([0, 100, 200], dtype=torch.int32).cuda(), 1, 10, 0.3)
    with pytest.raises(lt.LtError):
        lt.lt_bound_slices(ctx, pts, perm, torch.tensor([0, 256], dtype=torch.int32).cuda(), 10, 5, 0.3)
    lt.lt_sync(ctx)


def test_frame_on_bounded_slices():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room64_vpl1k_2box", slice_bounds=(200, 300))
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=0).setup()
    sizes = np.diff(R.slice_off.cpu().numpy())
    assert sizes.min() >= 150 and sizes.max() <= 300
    img = R.render().clone()
    R2 = Renderer(sc, cfg, device=0).setup(cut=R.cut.cpu().numpy(), row_perm=R.row_perm.cpu().numpy(),
                                           slice_off=R.slice_off.cpu().numpy())
    assert torch.equal(R2.render(), img)
