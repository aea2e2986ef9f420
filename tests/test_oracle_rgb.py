"""Pins of the colour oracle: a grey scene gives the scalar entries in every
channel, a light with one channel lights that channel only, entries are linear in
each channel's flux, node intensities add up the tree, and at full sampling and
full rank the stacked completion reproduces the RGB brute force."""
import numpy as np

from ltinputs import get_config, make_scene
from oracle import bruteforce, pipeline, rgb, shading
from oracle import tree as tree_mod


def _setup(**kw):
    cfg = get_config("room64_vpl1k_2box", width=16, height=16, n_vpl=64, n_slices=4, max_cut=64, rgb=True, **kw)
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    return cfg, sc, st


def _grey(sc):
    """The scene's own scalar albedos and flux in all three channels."""
    g = dict(point_albedo=np.repeat(sc.points[0, :, 3:4], 3, axis=1),
             vpl_albedo=np.repeat(sc.vpls[0, :, 3:4], 3, axis=1),
             vpl_flux=np.repeat(sc.vpls[2, :, 3:4], 3, axis=1))
    return g


def test_grey_scene_gives_the_scalar_entries_in_every_channel():
    cfg, sc, st = _setup()
    tr = st["tree"]
    rng = np.random.default_rng(1)
    rows = rng.integers(0, sc.m, 300)
    nodes = rng.integers(0, tr.n_nodes, 300)
    got = rgb.node_entries(st["pts_s"], sc.vpls, _grey(sc), st["row_perm"], tr, rows, nodes, sc.boxes, cfg["d_min"])
    want = shading.node_entries(st["pts_s"], sc.vpls, rows, tr.rep[nodes], tree_mod.node_scale(tr, sc.vpls, nodes),
                                sc.boxes, cfg["d_min"])
    assert np.any(want > 0)
    for k in range(3):
        np.testing.assert_allclose(got[:, k], want, rtol=1e-6, atol=1e-12)


def test_node_intensity_adds_up_the_tree():
    cfg, sc, st = _setup()
    tr = st["tree"]
    I = rgb.node_intensity(tr, sc.rgb)
    prod = sc.rgb["vpl_flux"].astype(np.float64) * sc.rgb["vpl_albedo"]
    np.testing.assert_allclose(I[0], prod.sum(axis=0), rtol=1e-12)
    internal = np.arange(tr.n - 1)
    np.testing.assert_allclose(I[internal], I[tr.child[internal, 0]] + I[tr.child[internal, 1]], rtol=1e-12)
    leaves = tr.leaf_node(np.arange(tr.n))
    np.testing.assert_allclose(I[leaves], prod[tr.order], rtol=1e-12)
    # the grey intensities are the tree's own float32 sums
    np.testing.assert_allclose(rgb.node_intensity(tr, _grey(sc))[:, 0], tr.I, rtol=1e-5)


def test_one_channel_light_and_linearity():
    cfg, sc, st = _setup()
    tr = st["tree"]
    rows = np.arange(0, sc.m, 3)
    nodes = np.full(rows.size, 0)
    red = dict(sc.rgb, vpl_flux=sc.rgb["vpl_flux"] * np.array([1.0, 0.0, 0.0], dtype=np.float32))
    e = rgb.node_entries(st["pts_s"], sc.vpls, red, st["row_perm"], tr, rows, nodes, sc.boxes)
    assert np.any(e[:, 0] > 0) and not e[:, 1:].any()
    two = dict(sc.rgb, vpl_flux=sc.rgb["vpl_flux"] * np.array([2.0, 1.0, 1.0], dtype=np.float32))
    base = rgb.node_entries(st["pts_s"], sc.vpls, sc.rgb, st["row_perm"], tr, rows, nodes, sc.boxes)
    dbl = rgb.node_entries(st["pts_s"], sc.vpls, two, st["row_perm"], tr, rows, nodes, sc.boxes)
    np.testing.assert_allclose(dbl[:, 0], 2 * base[:, 0], rtol=1e-12)
    np.testing.assert_allclose(dbl[:, 1:], base[:, 1:], rtol=1e-12)
    bf = rgb.bruteforce_rgb(sc.points, sc.vpls, red, sc.boxes)
    assert bf[:, 0].max() > 0 and not bf[:, 1:].any()


def test_full_sampling_full_rank_reproduces_rgb_bruteforce():
    """rate 100%, eps 0, tau 0 (the cut is every VPL), rank n': the stacked
    completion of each slice is exact and the image equals the RGB brute force."""
    cfg = get_config("room64_vpl1k_2box", width=8, height=8, n_vpl=12, n_slices=2, rate=1.0, rate1=1.0,
                     eps_cut=0.0, max_cut=100, tau=0.0, lam_rel=1e-13, als_iters=3, rank=12, rgb=True)
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    assert len(st["cut"]) == 12
    img, omega = rgb.render_frame(sc, cfg, st)
    for rows, cols, col_node, vals in omega:
        assert rows.size == (len(rows) // col_node.size) * col_node.size
    ref = rgb.bruteforce_rgb(sc.points, sc.vpls, sc.rgb, sc.boxes)
    np.testing.assert_allclose(img, ref, rtol=1e-8, atol=1e-9 * ref.max())
    # the channels differ (a coloured scene), and their luminance is close to the
    # scalar image of the luminance scene
    assert np.abs(ref[:, 0] - ref[:, 2]).max() > 0.05 * ref.max()
    lum = bruteforce.render(sc.points, sc.vpls, sc.boxes)
    assert np.linalg.norm(ref @ np.array([0.2126, 0.7152, 0.0722]) - lum) < 0.2 * np.linalg.norm(lum)


def test_stacking_puts_channel_k_of_pixel_i_at_row_3i_plus_k():
    r3, c3, v3 = rgb.stack([0, 2], [5, 1], [[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]])
    assert r3.tolist() == [0, 1, 2, 6, 7, 8] and c3.tolist() == [5, 5, 5, 1, 1, 1]
    assert v3.tolist() == [1.0, 2.0, 3.0, 4.0, 5.0, 6.0]
    U = np.arange(12, dtype=np.float64).reshape(6, 2)
    V = np.array([[1.0, 0.0], [0.0, 2.0]])
    img = rgb.render_stacked([(U, V)], np.array([1, 0]), np.array([0, 2]), 2)
    t = V.sum(axis=0)
    assert np.allclose(img[1], (U @ t)[:3]) and np.allclose(img[0], (U @ t)[3:])
