"""Colour on the GPU against the colour oracle: the ratio tables, every expanded
entry against the per-channel definition on the GPU's own samples, the stacked
completion and image against the oracle's on the same samples, a grey scene giving
the scalar frame in every channel, argument checks, and the full-size colour
workload against the RGB brute force."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene
from oracle import als as o_als
from oracle import pipeline, rgb
from oracle import render as o_render

pytestmark = pytest.mark.gpu

ENTRY_RTOL = 1e-5
IMAGE_RTOL = 1e-3


@pytest.fixture(scope="module")
def tiny():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room64_vpl1k_2box", rgb=True)
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    R = Renderer(sc, cfg, device=0).setup(cut=st["cut"], row_perm=st["row_perm"], slice_off=st["slice_off"])
    R.setup_rgb()
    img = R.render_rgb().cpu().numpy().astype(np.float64)
    return cfg, sc, st, R, img


def test_ratio_tables(tiny):
    cfg, sc, st, R, _ = tiny
    pr = R.rgb.pt_ratio.view(-1, 4).cpu().numpy()[:, :3]
    perm = st["row_perm"]
    want = sc.rgb["point_albedo"][perm].astype(np.float64) / st["pts_s"][0, :, 3:4].astype(np.float64)
    np.testing.assert_allclose(pr, want, rtol=1e-6)
    tr = st["tree"]
    nr = R.rgb.node_ratio.view(-1, 4).cpu().numpy()[:, :3]
    want = rgb.node_intensity(tr, sc.rgb) / tr.I.astype(np.float64)[:, None]
    np.testing.assert_allclose(nr, want, rtol=1e-5)
    assert np.array_equal(R.rgb.slice_off3.cpu().numpy(), 3 * np.asarray(st["slice_off"]))
    p3 = R.rgb.row_perm3.cpu().numpy()
    assert np.array_equal(p3[0::3], 3 * perm) and np.array_equal(p3[2::3], 3 * perm + 2)


def test_expanded_entries_match_the_per_channel_definition(tiny):
    cfg, sc, st, R, _ = tiny
    tr = st["tree"]
    for s in range(R.frame.S):
        rows, cols, vals, col_node, _ = R.smp.slice(s)
        r3, c3, v3 = R.rgb.slice(s)
        assert r3.size == 3 * rows.size
        assert np.array_equal(r3.reshape(-1, 3), 3 * rows[:, None] + np.arange(3))
        assert np.array_equal(c3.reshape(-1, 3), np.repeat(cols[:, None], 3, axis=1))
        a = int(st["slice_off"][s])
        want = rgb.node_entries(st["pts_s"], sc.vpls, sc.rgb, st["row_perm"], tr, a + rows, col_node[cols], sc.boxes,
                                cfg["d_min"])
        got = v3.reshape(-1, 3).astype(np.float64)
        assert np.all(np.abs(got - want) <= ENTRY_RTOL * np.abs(want) + 1e-12 * max(want.max(), 1e-30)), s


def test_stacked_completion_matches_oracle(tiny):
    cfg, sc, st, R, img = tiny
    factors = []
    for s in range(R.frame.S):
        r3, c3, v3 = R.rgb.slice(s)
        m_s = int(st["slice_off"][s + 1] - st["slice_off"][s])
        n_s = int(R.smp.ncol[s].item())
        factors.append(o_als.complete_slice(r3, c3, v3.astype(np.float64), 3 * m_s, n_s, cfg["rank"],
                                            cfg["als_iters"], cfg["lam_rel"], cfg["frame_seed"], s))
    ref = rgb.render_stacked(factors, st["row_perm"], st["slice_off"], sc.m)
    got = img.reshape(-1, 3)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= IMAGE_RTOL, rel
    assert np.abs(ref[:, 0] - ref[:, 2]).max() > 0.01 * ref.max()  # the channels differ


def test_adm_on_the_stacked_slices(tiny):
    from paper_2202_12567_gb300 import lt
    cfg, sc, st, R, _ = tiny
    lt.lt_complete_rgb(R.ctx, R.rgb, 0, 0.0, cfg["frame_seed"], adm=(30, 0.3, 1.0))
    lt.lt_render_rgb(R.ctx, R.rgb)
    lt.lt_sync(R.ctx)
    got = R.rgb.img.view(-1, 3).cpu().numpy().astype(np.float64)
    cfg_adm = dict(cfg, completion="adm", adm_iters=30, adm_alpha_rel=0.3, adm_gamma=1.0)
    factors = []
    for s in range(R.frame.S):
        r3, c3, v3 = R.rgb.slice(s)
        m_s = int(st["slice_off"][s + 1] - st["slice_off"][s])
        n_s = int(R.smp.ncol[s].item())
        vals = v3.astype(np.float64).reshape(-1, 3)
        factors.append(rgb.complete_stacked(r3[0::3] // 3, c3[0::3], vals, m_s, n_s, cfg["rank"], cfg_adm,
                                            cfg["frame_seed"], s))
    ref = rgb.render_stacked(factors, st["row_perm"], st["slice_off"], sc.m)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-4, rel


def test_grey_scene_gives_the_scalar_frame_in_every_channel():
    """Grey colours (the scalar albedo and flux in all three channels): the stacked
    slice repeats every row three times, ALS solves the same systems scaled by 3, and
    each channel is the scalar frame."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room64_vpl1k_2box")
    sc = make_scene(cfg)
    sc.rgb = dict(point_albedo=np.repeat(sc.points[0, :, 3:4], 3, axis=1),
                  vpl_albedo=np.repeat(sc.vpls[0, :, 3:4], 3, axis=1),
                  vpl_flux=np.repeat(sc.vpls[2, :, 3:4], 3, axis=1))
    R = Renderer(sc, cfg, device=0).setup()
    R.setup_rgb()
    scalar = R.render().cpu().numpy().astype(np.float64)
    col = R.render_rgb().cpu().numpy().astype(np.float64)
    for k in range(3):
        rel = np.linalg.norm(col[:, k] - scalar) / np.linalg.norm(scalar)
        assert rel <= 1e-4, (k, rel)


def test_rgb_rejects_oversized_slices(tiny):
    from paper_2202_12567_gb300 import lt
    cfg, sc, st, R, _ = tiny
    f = R.frame.struct()
    big = lt.lt_frame.from_buffer_copy(f)
    big.max_rows = 30000
    with pytest.raises(RuntimeError):
        R.ctx._check("lt_expand_rgb", R.ctx.lib.lt_expand_rgb(R.ctx.h, ctypes.byref(big), ctypes.byref(R.smp.struct()),
                                                              ctypes.byref(R.rgb.struct()),
                                                              ctypes.byref(R.rgb.samples3())))


def test_full_size_colour_workload():
    """256x256 points, 16384 VPLs, colour: the stacked frame against the RGB brute
    force, and sampled slices' expanded entries against the definition."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room256_vpl16k_2box_rgb")
    sc = make_scene(cfg)
    R = Renderer(sc, cfg, device=0).setup()
    R.setup_rgb()
    img = R.render_rgb().cpu().numpy().astype(np.float64)
    ref = R.bruteforce_rgb().cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(img - ref) / np.linalg.norm(ref)
    print("colour rel-RMSE vs RGB brute force:", rel)
    assert rel <= 0.03, rel
    off = R.slice_off.cpu().numpy()
    perm = R.row_perm.cpu().numpy()
    pts_s = sc.points[:, perm]
    from oracle import tree as tree_mod
    tr = tree_mod.build(sc.vpls)
    for s in (0, R.frame.S - 1):
        rows, cols, vals, col_node, _ = R.smp.slice(s)
        pick = np.random.default_rng(s).choice(rows.size, size=min(2000, rows.size), replace=False)
        r3, c3, v3 = R.rgb.slice(s)
        want = rgb.node_entries(pts_s, sc.vpls, sc.rgb, perm, tr, int(off[s]) + rows[pick], col_node[cols[pick]],
                                sc.boxes, cfg["d_min"])
        got = v3.reshape(-1, 3)[pick].astype(np.float64)
        assert np.all(np.abs(got - want) <= ENTRY_RTOL * np.abs(want) + 1e-12 * max(want.max(), 1e-30)), s
