"""Parity of the learned-proposal kernels (through the C ABI) with the oracle.

Features and leverage targets are compared on the oracle's cut and slices (pass-1
entry sets are identical there); the network is compared on seeded synthetic
features and parameters: logits, the loss, the gradient against float64 backprop
(normwise 1e-2, the bfloat16 bound) and one Adam step.  The frame with the
proposal must replay identically as a CUDA graph and draw as many entries as the
frame without it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from ltinputs import get_config, make_scene
from oracle import pipeline, proposal as P

pytestmark = pytest.mark.gpu

FEAT_RTOL, FEAT_ATOL = 1e-4, 1e-5
GRAD_NORMWISE = 1e-2


@pytest.fixture(scope="module")
def lt():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2202_12567_gb300 import lt as _lt
    _lt.load()
    return _lt


@pytest.fixture(scope="module")
def ctx(lt):
    return lt.Context(0)


@pytest.fixture(scope="module")
def tiny(lt):
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room64_vpl1k_2box", max_cut=256)
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    R = Renderer(sc, cfg, device=0).setup(cut=st["cut"], row_perm=st["row_perm"], slice_off=st["slice_off"])
    seed = cfg["frame_seed"]
    R.pass1(seed)
    lt.lt_sync(R.ctx)
    ores = {s: pipeline.run_slice(st, sc, cfg, s, seed) for s in range(R.frame.S)}
    same = [s for s in range(R.frame.S)
            if np.array_equal(R.smp.col_node[s * R.frame.C:s * R.frame.C + int(R.smp.ncol[s])].cpu().numpy(),
                              ores[s].p1.col_node)]
    assert len(same) >= R.frame.S - 1
    return cfg, sc, st, R, ores, same


def _synthetic(n, seed, groups):
    rng = np.random.default_rng(seed)
    X = (rng.normal(size=(n, P.N_FEAT)) * rng.uniform(0.2, 2.0, size=P.N_FEAT)).astype(np.float32)
    theta = (P.init_params(seed) + rng.normal(size=P.N_PARAM) * 0.02).astype(np.float32)
    go = np.asarray(groups, dtype=np.int32)
    t = rng.random(n)
    for a, b in zip(go[:-1], go[1:]):
        t[a:b] /= t[a:b].sum()
    return X, theta.astype(np.float64), go, t.astype(np.float32)


def test_features_match_oracle(lt, tiny):
    cfg, sc, st, R, ores, same = tiny
    feat, goff = lt.lt_proposal_features(R.ctx, R.frame, R.smp)
    F = feat.cpu().numpy()
    go = goff.cpu().numpy()
    ncol = R.smp.ncol.cpu().numpy()
    assert go[0] == 0 and np.array_equal(np.diff(go), ncol)
    for s in same:
        o = ores[s].p1
        a, b = int(st["slice_off"][s]), int(st["slice_off"][s + 1])
        want = P.slice_features(st["pts_s"], a, b - a, st["tree"], sc.vpls, o.col_node, o.cols, o.vals)
        got = F[go[s]:go[s + 1]]
        np.testing.assert_allclose(got, want, rtol=FEAT_RTOL, atol=FEAT_ATOL, err_msg=f"slice {s}")


@pytest.mark.parametrize("n", [1, 63, 64, 1000])
def test_forward_matches_oracle(lt, ctx, n):
    X, theta, go, _ = _synthetic(n, 7 + n, [0, n])
    z = lt.lt_proposal_forward(ctx, torch.from_numpy(theta.astype(np.float32)).cuda(), torch.from_numpy(X).cuda())
    got = z.cpu().numpy().astype(np.float64)
    want, _ = P.forward(theta, X)
    err = np.abs(got - want)
    assert np.all(err <= 1e-2 * (1 + np.abs(want))), err.max()
    assert np.median(err) <= 2e-3 * (1 + np.median(np.abs(want)))


def test_forward_reads_the_device_row_count(lt, ctx):
    X, theta, _, _ = _synthetic(300, 3, [0, 300])
    n_dev = torch.tensor([130], dtype=torch.int32, device="cuda")
    z = torch.full((300,), -7.0, device="cuda")
    lt.lt_proposal_forward(ctx, torch.from_numpy(theta.astype(np.float32)).cuda(), torch.from_numpy(X).cuda(), 300,
                           n_dev, z)
    zz = z.cpu().numpy()
    assert np.all(zz[130:] == -7.0) and np.all(zz[:130] != -7.0)


def test_init_matches_oracle(lt, ctx):
    th = lt.lt_proposal_init(ctx, 12345).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(th, P.init_params(12345), rtol=1e-6, atol=1e-9)


def test_gradient_and_loss_match_float64_backprop(lt, ctx):
    groups = [0, 200, 201, 333, 333, 700, 777]  # a one-row group and an empty one
    n = groups[-1]
    X, theta, go, t = _synthetic(n, 21, groups)
    grad, loss = lt.lt_proposal_grad(ctx, torch.from_numpy(theta.astype(np.float32)).cuda(), torch.from_numpy(X).cuda(),
                                     torch.from_numpy(t).cuda(), torch.from_numpy(go).cuda(), len(go) - 1, n)
    g = grad.cpu().numpy().astype(np.float64)
    z, cache = P.forward(theta, X)
    L, dz = P.loss_and_dz(z, t.astype(np.float64), go)
    want = P.backward(theta, cache, dz)
    assert np.linalg.norm(g - want) <= GRAD_NORMWISE * np.linalg.norm(want)
    o = 0
    for name, shp in P.SHAPES:
        k = int(np.prod(shp))
        gb, wb = g[o:o + k], want[o:o + k]
        assert np.linalg.norm(gb - wb) <= 3e-2 * np.linalg.norm(wb) + 1e-7, name
        o += k
    assert abs(float(loss.item()) - L) <= 1e-3 * abs(L)
    # deterministic: the same call twice gives the same bits
    grad2, _ = lt.lt_proposal_grad(ctx, torch.from_numpy(theta.astype(np.float32)).cuda(),
                                   torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(),
                                   torch.from_numpy(go).cuda(), len(go) - 1, n)
    assert torch.equal(grad, grad2)


def test_adam_matches_oracle(lt, ctx):
    rng = np.random.default_rng(5)
    th, m, v, g = (rng.normal(size=P.N_PARAM).astype(np.float32) for _ in range(4))
    v = np.abs(v)
    ct = [torch.from_numpy(a.copy()).cuda() for a in (th, m, v, g)]
    lt.lt_proposal_adam(ctx, ct[0], ct[1], ct[2], ct[3], 3, 1e-3)
    want_t, want_m, want_v = P.adam(th.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                                    g.astype(np.float64), 3, 1e-3)
    np.testing.assert_allclose(ct[1].cpu().numpy(), want_m, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(ct[2].cpu().numpy(), want_v, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(ct[0].cpu().numpy(), want_t, rtol=1e-5, atol=1e-6)


def test_slice_matrices_and_leverage_targets_match_oracle(lt, tiny):
    cfg, sc, st, R, ores, same = tiny
    ctx = R.ctx
    feat, goff = lt.lt_proposal_features(ctx, R.frame, R.smp)
    ncol = R.smp.ncol.cpu().numpy().astype(np.int64)
    cap = int(np.sum(R.frame.sizes * ncol))
    M, moff = lt.lt_slice_matrices(ctx, R.frame, R.smp, cfg["d_min"], cap)
    r, iters, seed = cfg["rank"], 30, 99
    tgt = lt.lt_leverage_targets(ctx, R.frame, R.smp, M, moff, goff, r, iters, seed).cpu().numpy()
    Mh, mo, go = M.cpu().numpy(), moff.cpu().numpy(), goff.cpu().numpy()
    assert mo[-1] == cap
    for s in same[:6]:
        o = ores[s].p1
        a, b = int(st["slice_off"][s]), int(st["slice_off"][s + 1])
        Mo = P.slice_matrix(st["pts_s"], a, b - a, st["tree"], sc.vpls, sc.boxes, o.col_node, cfg["d_min"])
        Mg = Mh[mo[s]:mo[s + 1]].reshape(b - a, len(o.col_node))
        assert np.all(np.abs(Mg - Mo) <= 1e-5 * np.abs(Mo) + 1e-12), f"slice {s}"
        want = P.targets(P.leverage(Mo, r, iters, seed, s))
        got = tgt[go[s]:go[s + 1]]
        assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want), f"slice {s}"
        assert abs(got.sum() - 1) < 1e-4


def test_mixture_weights_match_oracle(lt, tiny):
    cfg, sc, st, R, ores, same = tiny
    ctx = R.ctx
    rng = np.random.default_rng(8)
    theta = (P.init_params(3) + rng.normal(size=P.N_PARAM) * 0.05).astype(np.float32)
    feat, goff = lt.lt_proposal_features(ctx, R.frame, R.smp)
    th = torch.from_numpy(theta).cuda()
    z = lt.lt_proposal_forward(ctx, th, feat, R.frame.S * R.frame.C, goff[R.frame.S:])
    w = lt.lt_proposal_weights(ctx, R.frame, R.smp, goff, z, 0.8).cpu().numpy()
    C = R.frame.C
    for s in same[:6]:
        o = ores[s].p1
        a, b = int(st["slice_off"][s]), int(st["slice_off"][s + 1])
        Fo = P.slice_features(st["pts_s"], a, b - a, st["tree"], sc.vpls, o.col_node, o.cols, o.vals)
        zo, _ = P.forward(theta.astype(np.float64), Fo)
        wo = P.mixture(zo, o.g, np.array([0, len(zo)]))
        got = w[s * C:s * C + len(zo)]
        assert abs(got.sum() - 1) < 1e-5
        assert np.all(np.abs(got - wo) <= 2e-2 * wo + 1e-7), f"slice {s}"


def test_training_lowers_the_loss(lt, ctx):
    from paper_2202_12567_gb300 import proposal
    cfg = get_config("room64_vpl1k_2box", max_cut=256)
    batches = [proposal.scene_batch(ctx, cfg, 1000 + k) for k in range(6)]
    theta0 = lt.lt_proposal_init(ctx, 1)
    l0 = proposal.loss_of(ctx, theta0, batches)
    theta, hist = proposal.train(ctx, cfg, None, epochs=60, lr=3e-3, batches=batches)
    l1 = proposal.loss_of(ctx, theta, batches)
    assert np.all(np.isfinite(hist)) and l1 < l0 - 0.02, (l0, l1)


def test_frame_with_proposal_replays_and_keeps_the_sample_count(lt):
    from paper_2202_12567_gb300.renderer import Renderer
    cfg = get_config("room64_vpl1k_2box", max_cut=256)
    R = Renderer(make_scene(cfg), cfg, device=0).setup()
    R.render_frame(seed=9)
    cnt_g = R.smp.cnt.clone()
    theta = lt.lt_proposal_init(R.ctx, 4)
    prm = lt.params(cfg, proposal=theta, mix=0.8)
    lt.lt_render_frame(R.ctx, R.frame, prm, 9, R.smp, R.uv, R.row_perm, R.img)
    lt.lt_sync(R.ctx)
    img = R.img.clone()
    assert torch.equal(R.smp.cnt, cnt_g) and torch.isfinite(img).all() and float(img.sum()) > 0
    g = lt.lt_frame_graph_capture(R.ctx, R.frame, prm, R.smp, R.uv, R.row_perm, R.img, keep=(theta,))
    lt.lt_frame_graph_launch(g, 9)
    lt.lt_sync(R.ctx)
    assert torch.equal(R.img, img)
    g.close()


def test_shipped_proposal_beats_g_at_equal_sample_count(lt):
    """The network trained by `python -m paper_2202_12567_gb300.proposal` (200 scenes
    1000..1199) against the paper's pdf g on held-out scenes of the same generator."""
    import os
    from paper_2202_12567_gb300 import proposal
    if not os.path.exists(proposal.DEFAULT_THETA):
        pytest.skip("no trained proposal shipped")
    cfg = get_config("room256_vpl16k_2box")
    ctx = lt.Context(0)
    theta = proposal.load_theta()
    res = proposal.ab_compare(ctx, cfg, theta, [5001, 5002, 5003])
    assert all(r["entries_g"] == r["entries_learned"] for r in res)
    g = np.mean([r["rel_g"] for r in res])
    p = np.mean([r["rel_learned"] for r in res])
    assert p < g, res
