"""Triangle occluders on the GPU: the BVH's structure, shadow segments against the
oracle's Moller-Trumbore over every triangle, a box written as triangles against
the box, a frame of a mesh scene against the oracle pipeline, the mesh workload
against the GPU brute force, and uploads replacing the triangles."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene
from oracle import pipeline, shading

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lt():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300 import lt
    return lt


@pytest.fixture(scope="module")
def ctx(lt):
    return lt.Context(0)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _box_triangles(b):
    lo, hi = np.asarray(b[:3], float), np.asarray(b[3:], float)
    c = np.array([[lo[0] if i & 1 == 0 else hi[0], lo[1] if i & 2 == 0 else hi[1], lo[2] if i & 4 == 0 else hi[2]]
                  for i in range(8)])
    out = []
    for q0, q1, q2, q3 in [(0, 1, 3, 2), (4, 5, 7, 6), (0, 1, 5, 4), (2, 3, 7, 6), (0, 2, 6, 4), (1, 3, 7, 5)]:
        out += [[c[q0], c[q1], c[q2]], [c[q0], c[q2], c[q3]]]
    return np.array(out, dtype=np.float32)


def test_bvh_structure(lt, ctx):
    sc = make_scene(get_config("room256_vpl16k_mesh", width=8, height=8, n_vpl=8))
    tris = sc.tris
    nt = tris.shape[0]
    lt.lt_scene_upload(ctx, _cuda(sc.boxes))
    lt.lt_mesh_upload(ctx, _cuda(tris))
    aabb, child, leaf = (x.cpu().numpy() for x in lt.lt_mesh_bvh(ctx, nt, "cuda"))
    assert sorted(leaf.tolist()) == list(range(nt))
    lo, hi = tris.min(axis=1), tris.max(axis=1)
    assert np.array_equal(aabb[nt - 1:, :3], lo[leaf]) and np.array_equal(aabb[nt - 1:, 3:], hi[leaf])
    seen = np.zeros(2 * nt - 1, dtype=int)
    for i in range(nt - 1):
        for c in child[i]:
            seen[c] += 1
            assert np.all(aabb[i, :3] <= aabb[c, :3]) and np.all(aabb[i, 3:] >= aabb[c, 3:])
    assert seen[0] == 0 and np.all(seen[1:] == 1)  # a tree rooted at 0


def test_shadow_segments_match_oracle(lt, ctx):
    sc = make_scene(get_config("room256_vpl16k_mesh", width=8, height=8, n_vpl=8, mesh_subdiv=2))
    rng = np.random.default_rng(2)
    k = 50_000
    o = rng.uniform(0, 1, (k, 3)).astype(np.float32)
    e = rng.uniform(0, 1, (k, 3)).astype(np.float32)
    lt.lt_scene_upload(ctx, _cuda(sc.boxes))
    lt.lt_mesh_upload(ctx, _cuda(sc.tris))
    got = lt.lt_shadow_test(ctx, _cuda(o), _cuda(e)).cpu().numpy().astype(bool)
    exp = shading.segment_blocked(o.astype(np.float64), e.astype(np.float64), sc.occluders)
    assert np.mean(got != exp) <= 1e-4
    only_tris = exp & ~shading.segment_blocked(o.astype(np.float64), e.astype(np.float64), sc.boxes)
    assert only_tris.mean() > 0.01  # the spheres block segments the boxes do not
    # a new scene upload clears the triangles
    lt.lt_scene_upload(ctx, _cuda(sc.boxes))
    got = lt.lt_shadow_test(ctx, _cuda(o), _cuda(e)).cpu().numpy().astype(bool)
    exp = shading.segment_blocked(o.astype(np.float64), e.astype(np.float64), sc.boxes)
    assert np.mean(got != exp) <= 1e-4


def test_box_as_triangles_on_the_gpu(lt, ctx):
    box = np.array([[0.3, 0.2, 0.4, 0.6, 0.5, 0.7]], dtype=np.float32)
    rng = np.random.default_rng(4)
    o = rng.uniform(0, 1, (100_000, 3)).astype(np.float32)
    e = rng.uniform(0, 1, (100_000, 3)).astype(np.float32)
    inside = lambda x: np.all((x >= box[0, :3]) & (x <= box[0, 3:]), axis=1)
    keep = ~inside(o) & ~inside(e)
    o, e = o[keep], e[keep]
    lt.lt_scene_upload(ctx, _cuda(box))
    by_box = lt.lt_shadow_test(ctx, _cuda(o), _cuda(e)).cpu().numpy().astype(bool)
    lt.lt_scene_upload(ctx, _cuda(np.zeros((0, 6), dtype=np.float32)))
    lt.lt_mesh_upload(ctx, _cuda(_box_triangles(box[0])))
    by_tris = lt.lt_shadow_test(ctx, _cuda(o), _cuda(e)).cpu().numpy().astype(bool)
    assert by_box.mean() > 0.05
    assert np.mean(by_box != by_tris) <= 1e-4


def test_mesh_frame_matches_oracle_pipeline(lt):
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room64_vpl1k_mesh")
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    R = Renderer(sc, cfg, device=0).setup(cut=st["cut"], row_perm=st["row_perm"], slice_off=st["slice_off"])
    img = R.render().cpu().numpy().astype(np.float64)
    ref, _ = pipeline.render_frame(sc, cfg, st)
    rel = np.linalg.norm(img - ref) / np.linalg.norm(ref)
    assert rel <= 1e-3, rel


def test_mesh_workload_against_gpu_bruteforce(lt):
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room256_vpl16k_mesh")
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=0).setup()
    img = R.render().double()
    ref = R.bruteforce().double()
    rel = float(torch.linalg.norm(img - ref) / torch.linalg.norm(ref))
    print("mesh workload rel-RMSE vs brute force:", rel)
    assert rel <= 0.06, rel  # a quality bound, not parity (3.9% measured at 15% sampling)
    # the brute force sees the spheres: rows on the floor below them are darker than
    # the same render with the triangles cleared
    lt.lt_scene_upload(R.ctx, R.boxes)
    bare = R.bruteforce().double()
    assert float((bare - ref).sum()) > 0.0
