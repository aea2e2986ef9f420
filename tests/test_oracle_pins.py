"""Pins of the CPU oracle against facts fixed outside it (no GPU needed).

Each test checks a part of the oracle against something other than its own code:
published known-answer vectors, closed forms, a second independent algorithm,
invariants stated by the paper, or brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

from ltinputs import get_config, make_scene
from ltinputs.scenes import single_quad_scene
from oracle import als, bruteforce, cut as cut_mod, pass1, pass2, philox, pipeline, render, shading
from oracle import slices as slices_mod, tree as tree_mod

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_philox_uniformity():
    w = philox.draw(123, np.arange(200000, dtype=np.uint64), 5, 2, philox.TAG_PASS1)[0]
    idx = philox.uniform_index(w, 10)
    counts = np.bincount(idx, minlength=10)
    chi2 = np.sum((counts - 20000.0) ** 2 / 20000.0)
    assert chi2 < 30.0  # 9 dof, p ~ 4e-4


# --------------------------------------------------------------------------- shading
def _quad_case(res=256, h=0.5, side=1.0):
    flux, rho_v, rho_x = 0.7, 0.6, 0.4
    pts, vpls = single_quad_scene([side / 2, h, side / 2], [0, -1, 0], flux, rho_v, 0.0, res, rho_x, side)
    return pts, vpls, flux, rho_v, rho_x


def test_entry_closed_form_one_vpl_one_quad():
    """A point at horizontal distance r below a downward VPL at height h receives
    Phi (rho_v/pi)(rho_x/pi) h^2 / (h^2 + r^2)^2 (both cosines equal h/d)."""
    pts, vpls, flux, rho_v, rho_x = _quad_case(res=32)
    m = pts.shape[1]
    val = shading.vpl_entries(pts, vpls, np.arange(m), np.zeros(m, dtype=int), np.zeros((0, 6)))
    x = pts[0, :, 0].astype(np.float64) - 0.5
    z = pts[0, :, 2].astype(np.float64) - 0.5
    h = 0.5
    r2 = x * x + z * z
    expect = flux * (rho_v / math.pi) * (rho_x / math.pi) * h * h / (h * h + r2) ** 2
    np.testing.assert_allclose(val, expect, rtol=1e-6)


def _corner_form_factor(X, Y):
    """Differential element to a parallel rectangle whose corner lies on the element's
    normal (standard radiative-transfer catalogue form)."""
    a = X / math.sqrt(1 + X * X) * math.atan(Y / math.sqrt(1 + X * X))
    b = Y / math.sqrt(1 + Y * Y) * math.atan(X / math.sqrt(1 + Y * Y))
    return (a + b) / (2 * math.pi)


def test_bruteforce_integral_matches_form_factor():
    """Sum of the image times pixel area = Phi rho_v rho_x / pi^2 * pi * F(VPL->quad)."""
    res, h, side = 256, 0.5, 1.0
    pts, vpls, flux, rho_v, rho_x = _quad_case(res=res, h=h, side=side)
    img = bruteforce.render(pts, vpls, np.zeros((0, 6)))
    integral = img.sum() * (side / res) ** 2
    F = 4 * _corner_form_factor(side / 2 / h, side / 2 / h)
    expect = flux * rho_v * rho_x / math.pi ** 2 * math.pi * F
    assert abs(integral / expect - 1) < 2e-5


def test_glossy_brdf_peak_and_energy():
    """Phong lobe: peak value at the mirror direction; f_max bounds it; diffuse case."""
    n = np.array([[0.0, 1.0, 0.0]])
    w_in = np.array([[0.6, 0.8, 0.0]])
    mirror = np.array([[-0.6, 0.8, 0.0]])
    e = 40.0
    f = shading.brdf(np.array([0.5]), np.array([e]), n, w_in, mirror)
    assert abs(f[0] - (0.5 * 0.5 / math.pi + 0.5 * 0.5 * (e + 2) / (2 * math.pi))) < 1e-12
    assert f[0] <= shading.brdf_max(0.5, e) + 1e-15
    # cos^e lobe integrated against cos over the hemisphere around the mirror direction
    # equals 1 for the normalised modified Phong lobe (e + 2)/(2 pi) cos^e a cos(theta)
    # when the mirror direction is the normal: check by quadrature
    th = np.linspace(0, math.pi / 2, 20001)
    lobe = (e + 2) / (2 * math.pi) * np.cos(th) ** e * np.cos(th) * np.sin(th) * 2 * math.pi
    assert abs(np.trapezoid(lobe, th) - 1.0) < 1e-6
    fd = shading.brdf(np.array([0.3]), np.array([0.0]), n, w_in, mirror)
    assert abs(fd[0] - 0.3 / math.pi) < 1e-15


# --------------------------------------------------------------------------- visibility
BOX = np.array([[0.4, 0.4, 0.4, 0.6, 0.6, 0.6]])


@pytest.mark.parametrize("o,e,blocked", [
    ((0.5, 0.5, 0.0), (0.5, 0.5, 1.0), True),      # through the centre
    ((0.5, 0.7, 0.0), (0.5, 0.7, 1.0), False),     # passes above
    ((0.5, 0.6, 0.0), (0.5, 0.6, 1.0), True),      # runs along the top face (closed box)
    ((0.5, 0.5, 0.0), (0.5, 0.5, 0.3), False),     # ends before the box
    ((0.5, 0.5, 0.7), (0.5, 0.5, 1.0), False),     # starts after the box
    ((0.3, 0.3, 0.3), (0.7, 0.7, 0.7), True),      # diagonal through two corners
    ((0.3, 0.7, 0.5), (0.7, 0.3001, 0.5), True),   # cuts a corner region
    ((0.2, 0.8, 0.5), (0.55, 0.8, 0.5), False),    # parallel to x, outside the y slab
    ((0.5, 0.5, 0.5), (0.5, 0.5, 0.9), True),      # starts inside the box
])
def test_segment_blocked_cases(o, e, blocked):
    assert bool(shading.segment_blocked(np.array([o]), np.array([e]), BOX)[0]) == blocked


def test_segment_blocked_matches_point_sampling():
    """Random segments: the slab test agrees with dense point-in-box sampling except
    in a thin band around the boxes' surfaces."""
    rng = np.random.default_rng(5)
    boxes = np.sort(rng.uniform(0.1, 0.9, size=(12, 2, 3)), axis=1).reshape(12, 6)
    boxes = np.concatenate([boxes[:, [0, 2, 4]], boxes[:, [1, 3, 5]]], axis=1)  # fix order
    boxes = np.stack([np.minimum(boxes[:, :3], boxes[:, 3:]), np.maximum(boxes[:, :3], boxes[:, 3:])], 1).reshape(12, 6)
    o = rng.uniform(0, 1, size=(3000, 3))
    e = rng.uniform(0, 1, size=(3000, 3))
    got = shading.segment_blocked(o, e, boxes)
    t = np.linspace(shading.T_MIN, shading.T_MAX, 4001)
    pts = o[:, None, :] + t[None, :, None] * (e - o)[:, None, :]
    lo, hi = boxes[:, :3], boxes[:, 3:]
    margin = 1e-3
    inside_deep = np.zeros(3000, dtype=bool)
    near = np.zeros(3000, dtype=bool)
    for b in range(boxes.shape[0]):
        d_in = np.minimum(pts - lo[b], hi[b] - pts).min(axis=-1)   # >0 inside
        inside_deep |= (d_in > margin).any(axis=1)
        near |= (np.abs(d_in) <= margin).any(axis=1) | ((d_in > -margin) & (d_in <= margin)).any(axis=1)
    sure = ~near | inside_deep
    assert np.all(got[inside_deep])
    assert np.all(~got[sure & ~inside_deep])
    assert sure.mean() > 0.9


# --------------------------------------------------------------------------- tree
def _top_down_ranges(keys):
    """Binary radix tree by recursive splitting at the highest differing bit."""
    out = {}
    stack = [(0, len(keys) - 1)]
    while stack:
        a, b = stack.pop()
        if a == b:
            continue
        bit = (keys[a] ^ keys[b]).bit_length() - 1
        g = a
        while not (keys[g + 1] >> bit) & 1:
            g += 1
        out[(a, b)] = ((a, g), (g + 1, b))
        stack.append((a, g))
        stack.append((g + 1, b))
    return out


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (300, 3), (1024, 4)])
def test_tree_equals_top_down_radix_tree(n, seed):
    sc = make_scene(get_config("room64_vpl1k_2box", n_vpl=max(n, 1)), seed=seed)
    tr = tree_mod.build(sc.vpls)
    V = sc.vpls
    keys = ((tree_mod.morton_codes(V[0, :, :3]) | (tree_mod.orientation_class(V[1, :, :3]) << np.uint64(30)))
            << np.uint64(32)) | np.arange(n, dtype=np.uint64)
    skeys = sorted(int(k) for k in keys)
    assert [int(keys[i]) for i in tr.order] == skeys
    ref = _top_down_ranges(skeys)
    got = {}
    for f in range(n - 1):
        a, b = tr.child[f]
        got[(int(tr.first[f]), int(tr.last[f]))] = ((int(tr.first[a]), int(tr.last[a])),
                                                       (int(tr.first[b]), int(tr.last[b])))
    assert got == ref
    # I_f = I_a + I_b down to the leaves: the root carries the total intensity
    total = float(np.sum(V[2, :, 3].astype(np.float64) * V[0, :, 3]))
    assert abs(float(tr.I[0]) / total - 1) < 1e-5
    # the representative is a VPL inside the node
    pos_in = np.searchsorted(np.asarray(tr.order), 0)
    for f in range(tr.n_nodes):
        j = int(np.nonzero(tr.order == tr.rep[f])[0][0])
        assert tr.first[f] <= j <= tr.last[f]


# --------------------------------------------------------------------------- global cut
@pytest.fixture(scope="module")
def tiny():
    cfg = get_config("room64_vpl1k_2box")
    sc = make_scene(cfg)
    tr = tree_mod.build(sc.vpls)
    return cfg, sc, tr


def _covers_each_leaf_once(tr, cut):
    cover = np.zeros(tr.n, dtype=int)
    for c in cut:
        cover[tr.first[c]:tr.last[c] + 1] += 1
    return np.all(cover == 1)


def test_cut_partitions_leaves_and_is_in_leaf_order(tiny):
    cfg, sc, tr = tiny
    cut = cut_mod.build_global_cut(tr, sc.points, sc.vpls, sc.width, sc.height, 0.05, 300)
    assert len(cut) == 300
    assert _covers_each_leaf_once(tr, cut)
    assert np.all(np.diff(tr.first[cut]) > 0)


def test_cut_zero_eps_gives_all_leaves():
    cfg = get_config("room64_vpl1k_2box", n_vpl=64, width=16, height=16)
    sc = make_scene(cfg)
    tr = tree_mod.build(sc.vpls)
    cut = cut_mod.build_global_cut(tr, sc.points, sc.vpls, sc.width, sc.height, 0.0, 10_000)
    assert sorted(cut.tolist()) == list(range(tr.n - 1, 2 * tr.n - 1))


def test_cut_bound_is_conservative(tiny):
    """b_c(x) bounds the true unoccluded sum of the node's VPLs (brute force)."""
    cfg, sc, tr = tiny
    cut = cut_mod.build_global_cut(tr, sc.points, sc.vpls, sc.width, sc.height, 0.05, 200)
    rows = cut_mod.test_rows(sc.width, sc.height)[::3]
    b = cut_mod.node_bound(tr, sc.points, rows, cut)
    for k, c in enumerate(cut[::7]):
        vp = tr.order[tr.first[c]:tr.last[c] + 1]
        rr = np.repeat(rows, vp.size)
        cc = np.tile(vp, rows.size)
        true = shading.unoccluded(sc.points, sc.vpls, rr, cc).reshape(rows.size, vp.size).sum(1)
        assert np.all(b[:, 7 * k] >= true * (1 - 1e-9))


# --------------------------------------------------------------------------- slicing
def test_kmeans_recovers_separated_blobs():
    rng = np.random.default_rng(0)
    centres = np.array([[0.1, 0.1, 0.1], [0.9, 0.1, 0.1], [0.1, 0.9, 0.9], [0.9, 0.9, 0.9]])
    lab = rng.integers(0, 4, size=400)
    pts = np.zeros((3, 400, 4), dtype=np.float32)
    pts[0, :, :3] = centres[lab] + rng.normal(0, 0.01, size=(400, 3))
    pts[1, :, 1] = 1.0
    perm, off, got, C = slices_mod.kmeans_slices(pts, 4, 10)
    # the partition equals the blobs (labels up to renaming)
    pairs = set(zip(lab.tolist(), got.tolist()))
    assert len(pairs) == 4
    # nearest-centroid invariant and slice-contiguous permutation
    X = slices_mod.features(pts)
    d2 = ((X[:, None, :] - C[None]) ** 2).sum(-1)
    assert np.all(d2[np.arange(400), got] <= d2.min(1) + 1e-15)
    assert np.all(np.diff(got[perm]) >= 0) and off[-1] == 400


# --------------------------------------------------------------------------- pass 1
@pytest.fixture(scope="module")
def tiny_setup(tiny):
    cfg, sc, tr = tiny
    cfg = dict(cfg, max_cut=256)
    st = pipeline.setup(sc, cfg)
    return cfg, sc, st


def _run_p1(cfg, sc, st, s, tau=None, order_rng=None):
    a, b = int(st["slice_off"][s]), int(st["slice_off"][s + 1])
    return pass1.coarsen_slice(st["tree"], st["forest"], st["pts_s"], sc.vpls, sc.boxes, s, a, b - a,
                               cfg["rate1"], cfg["tau"] if tau is None else tau, 7, cfg["d_min"],
                               order_rng)


def test_pass1_eps_identity_and_cost_recursion(tiny_setup):
    """eps(L_f) in its first form ||(V_a + V_b) - V_a I_f / I_a|| equals the second form
    used by the oracle (Sec. 4); cost(f) = eps(f) + cost(q) (Eq. 2); merge iff cost < thr."""
    cfg, sc, st = tiny_setup
    tr, fo = st["tree"], st["forest"]
    res = _run_p1(cfg, sc, st, 3)
    assert len(res.log) > 10
    cost = {}
    n_merged = 0
    for (f, eps, cf, thr, merged, p, q, rf, vp, vq) in res.log:
        Ip, Iq, If = (float(tr.I[fo.node[x]]) for x in (p, q, f))
        first_form = np.max(np.abs((vp + vq) - vp * If / Ip))
        assert abs(first_form - eps) <= 1e-6 * max(1e-30, np.max(np.abs(vp)) + np.max(np.abs(vq)))
        # V_p, V_q are the entries of p and q on zeta_f, recomputed independently here
        for x, vx in ((p, vp), (q, vq)):
            t = fo.node[x]
            ref = shading.node_entries(st["pts_s"], sc.vpls, int(st["slice_off"][3]) + rf,
                                       np.full(rf.size, tr.rep[t]),
                                       np.full(rf.size, tree_mod.node_scale(tr, sc.vpls, [t])[0]), sc.boxes)
            np.testing.assert_allclose(vx, ref, rtol=1e-12, atol=0)
        assert abs(cf - (eps + cost.get(q, 0.0))) <= 1e-15 + 1e-12 * cf
        assert thr > 0 and merged == (cf < thr)
        if merged:
            cost[f] = cf
            n_merged += 1
    assert n_merged > 0


@pytest.mark.parametrize("tau", [None, 0.0])
def test_pass1_dark_slice_coarsens_to_the_root(tiny_setup, tau):
    """A slice whose shading points have zero albedo: every entry is zero, so S_hat = 0
    and every pair's cost is zero; the zero bound is read as met by a zero cost, so
    every pair merges (with any tau) and the coarsened cut is the forest's root."""
    cfg, sc, st = tiny_setup
    s = 3
    a, b = int(st["slice_off"][s]), int(st["slice_off"][s + 1])
    dark = dict(st, pts_s=st["pts_s"].copy())
    dark["pts_s"][0, a:b, 3] = 0.0
    res = _run_p1(cfg, sc, dark, s, tau=tau)
    fo = st["forest"]
    assert res.s_hat == 0.0 and len(res.log) == fo.C - 1
    assert all(merged for (_, _, _, _, merged, *_rest) in res.log)
    assert np.array_equal(res.col_node, fo.node[fo.parent == -1])
    assert np.all(res.vals == 0.0) and np.all(res.g == 0.0)
    # the same slice lit keeps columns apart
    assert _run_p1(cfg, sc, st, s).col_node.size > 1


def test_pass1_tau_zero_never_merges(tiny_setup):
    cfg, sc, st = tiny_setup
    res = _run_p1(cfg, sc, st, 2, tau=0.0)
    assert np.array_equal(res.col_node, st["cut"])


def test_pass1_tau_infinite_merges_to_forest_root(tiny_setup):
    cfg, sc, st = tiny_setup
    res = _run_p1(cfg, sc, st, 2, tau=np.inf)
    assert res.col_node.tolist() == [0]
    # every observed entry of the root column is a row of the slice, without repeats
    assert np.unique(res.rows).size == res.rows.size


def test_pass1_rows_per_node_rule(tiny_setup):
    cfg, sc, st = tiny_setup
    tr = st["tree"]
    cut = st["cut"]
    m_s = 200
    k = pass1.rows_per_node(tr, cut, m_s, cfg["rate1"])
    assert np.all((k >= 2) & (k <= 64))
    # proportional to intensity where the clamp is inactive (Sec. 4)
    kappa = max(2.0, cfg["rate1"] * m_s)
    x = kappa * len(cut) * tr.I[cut].astype(np.float64) / float(tr.I[0])
    free = (x > 2.5) & (x < 63.5)
    assert np.all(np.abs(k[free] - x[free]) <= 0.5 + 1e-4)
    for c in range(0, len(cut), 37):
        r = pass1.draw_rows(7, 1, c, int(k[c]), m_s)
        assert r.size == k[c] and np.unique(r).size == r.size and r.min() >= 0 and r.max() < m_s


def test_pass1_order_independent(tiny_setup):
    cfg, sc, st = tiny_setup
    a = _run_p1(cfg, sc, st, 5)
    b = _run_p1(cfg, sc, st, 5, order_rng=np.random.default_rng(11))
    assert np.array_equal(a.col_node, b.col_node)
    assert np.array_equal(a.rows, b.rows) and np.array_equal(a.cols, b.cols)
    np.testing.assert_array_equal(a.vals, b.vals)


# --------------------------------------------------------------------------- pass 2
def test_pass2_column_law_and_uniform_rows():
    """Raw draws follow q_c / sum q (chi-square) and rows are uniform."""
    w = np.array([0.0, 1.0, 3.0, 0.5, 2.0, 0.0, 7.0, 0.25])
    q = pass2.quantised_weights(w)
    assert q[0] == 0 and q[5] == 0 and q[6] == 1 << 24
    cdf = np.cumsum(q)
    N = 200_000
    row, col = pass2.raw_draws(99, 4, 13, cdf, np.arange(N))
    counts = np.bincount(col, minlength=w.size)
    assert counts[0] == 0 and counts[5] == 0
    p = q.astype(np.float64) / q.sum()
    nz = p > 0
    chi2 = np.sum((counts[nz] - N * p[nz]) ** 2 / (N * p[nz]))
    assert chi2 < 25.0     # 5 dof
    rc = np.bincount(row, minlength=13)
    chi2r = np.sum((rc - N / 13) ** 2 / (N / 13))
    assert chi2r < 40.0    # 12 dof


def test_pass2_exact_count_no_duplicates():
    rng = np.random.default_rng(1)
    m_s, n_s, rate = 50, 40, 0.3
    obs = rng.choice(m_s * n_s, 100, replace=False)
    g = rng.uniform(0, 1, n_s)
    r, c, nd, cap = pass2.draw_pass2(5, 0, m_s, g, obs, rate)
    T = pass2.target_count(rate, m_s, n_s)
    keys = r * n_s + c
    assert not cap
    assert keys.size == T - obs.size
    assert np.unique(np.concatenate([keys, obs])).size == T


def test_pass2_nothing_when_pass1_suffices():
    r, c, nd, cap = pass2.draw_pass2(5, 0, 10, np.ones(10), np.arange(60), 0.5)
    assert r.size == 0 and nd == 0


# --------------------------------------------------------------------------- ALS
def test_als_exact_recovery_of_rank_r():
    """Rank-r matrix from >= 3 r (m + n) uniform samples: rel. Frobenius <= 1e-5."""
    rng = np.random.default_rng(3)
    m, n, r = 120, 90, 6
    X = rng.uniform(0.1, 1.0, (m, r))
    Y = rng.uniform(0.1, 1.0, (n, r))
    M = X @ Y.T
    k = 3 * r * (m + n)
    idx = rng.choice(m * n, k, replace=False)
    rows, cols = idx // n, idx % n
    U, V = als.complete_slice(rows, cols, M[rows, cols], m, n, r, 300, 1e-10, 1, 0)
    err = np.linalg.norm(U @ V.T - M) / np.linalg.norm(M)
    assert err <= 1e-5


def test_als_fully_observed_reaches_truncated_svd():
    rng = np.random.default_rng(4)
    m, n, r = 60, 40, 5
    Q1, _ = np.linalg.qr(rng.normal(size=(m, m)))
    Q2, _ = np.linalg.qr(rng.normal(size=(n, n)))
    sv = np.concatenate([np.linspace(10, 6, r), np.linspace(0.5, 0.01, n - r)])
    M = (Q1[:, :n] * sv) @ Q2.T
    rows, cols = np.divmod(np.arange(m * n), n)
    U, V = als.complete_slice(rows, cols, M.ravel(), m, n, r, 200, 1e-13, 2, 0)
    err = np.linalg.norm(U @ V.T - M)
    best = np.sqrt(np.sum(sv[r:] ** 2))
    assert abs(err - best) / best < 1e-6


def test_warm_start_maps_columns_by_node():
    """Columns whose node was a previous column start from its V row (first r
    components, zero beyond the previous rank); the others from the seeded start."""
    rng = np.random.default_rng(6)
    prev_nodes = np.array([40, 7, 19, 3])
    prev_V = rng.uniform(0.1, 1.0, (4, 5))
    nodes = np.array([3, 11, 40, 19])             # 11 is new
    vals = rng.uniform(0.0, 2.0, 50)
    V0 = als.warm_start(9, 2, nodes, vals, 8, prev_nodes, prev_V)
    cold = als.init_v(9, 2, 4, 8, float(vals.mean()))
    for c, i in ((0, 3), (2, 0), (3, 2)):
        assert np.array_equal(V0[c, :5], prev_V[i]) and np.all(V0[c, 5:] == 0.0)
    assert np.array_equal(V0[1], cold[1])
    # a lower rank keeps the first components
    assert np.array_equal(als.warm_start(9, 2, nodes, vals, 3, prev_nodes, prev_V)[0], prev_V[3, :3])


def test_warm_start_from_the_answer_needs_one_sweep():
    """Started at the true V of an exactly rank-r matrix, one sweep recovers it; the
    seeded start does not (a start that ignored the previous factors fails this)."""
    rng = np.random.default_rng(8)
    m, n, r = 80, 60, 4
    X = rng.uniform(0.1, 1.0, (m, r))
    Y = rng.uniform(0.1, 1.0, (n, r))
    M = X @ Y.T
    idx = rng.choice(m * n, 3 * r * (m + n), replace=False)
    rows, cols = idx // n, idx % n
    nodes = np.arange(100, 100 + n)
    V0 = als.warm_start(1, 0, nodes, M[rows, cols], r, nodes, Y)
    U, V = als.complete_slice(rows, cols, M[rows, cols], m, n, r, 1, 1e-12, 1, 0, V0=V0)
    assert np.linalg.norm(U @ V.T - M) / np.linalg.norm(M) <= 1e-6
    U, V = als.complete_slice(rows, cols, M[rows, cols], m, n, r, 1, 1e-12, 1, 0)
    assert np.linalg.norm(U @ V.T - M) / np.linalg.norm(M) > 1e-3


@pytest.mark.parametrize("n_s,R,cols,want", [
    # values worked out by hand from r_s = min(R, max(8, 8 * ceil(n' / cols)))
    (0, 32, 512, 8), (1, 32, 512, 8), (511, 32, 512, 8), (512, 32, 512, 8), (513, 32, 512, 16),
    (1024, 32, 512, 16), (1025, 32, 512, 24), (1536, 32, 512, 24), (1537, 32, 512, 32),
    (2049, 32, 512, 32), (4 * 512 + 1, 32, 512, 32), (100000, 32, 512, 32),
    (513, 16, 512, 16), (2000, 16, 512, 16), (1, 8, 512, 8), (5000, 8, 512, 8),
    (100, 32, 100, 8), (101, 32, 100, 16), (301, 32, 100, 32)])
def test_slice_rank_rule(n_s, R, cols, want):
    """The per-slice rank rule (configuration 3: rank 8-32 chosen per slice) against
    hand-computed values at and one past every multiple of the column quantum."""
    assert pipeline.slice_rank({"rank": R, "rank_cols": cols}, n_s) == want


def test_slice_rank_fixed_without_columns():
    assert pipeline.slice_rank({"rank": 16, "rank_cols": 0}, 5000) == 16
    assert pipeline.slice_rank({"rank": 24}, 3) == 24


# --------------------------------------------------------------------------- render
def test_render_factorised_sum_equals_explicit_sum():
    rng = np.random.default_rng(6)
    U = rng.normal(size=(30, 4))
    V = rng.normal(size=(25, 4))
    img = render.render_slices([(U, V)], np.arange(30), np.array([0, 30]), 30, clamp=False)
    assert abs(img.sum() - (U @ V.T).sum()) < 1e-12 * np.abs(U @ V.T).sum()
    np.testing.assert_allclose(img, (U @ V.T).sum(1), rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------- end to end
def test_full_sampling_full_rank_reproduces_bruteforce():
    """rate 100%, eps 0, tau 0, r = min(m', n'): the pipeline equals brute force."""
    cfg = get_config("room64_vpl1k_2box", width=8, height=8, n_vpl=12, n_slices=2, rate=1.0,
                     eps_cut=0.0, max_cut=100, tau=0.0, lam_rel=1e-13, als_iters=2)
    sc = make_scene(cfg)
    ref = bruteforce.render(sc.points, sc.vpls, sc.boxes)
    st = pipeline.setup(sc, cfg)
    assert len(st["cut"]) == 12
    factors = []
    for s in range(2):
        a, b = int(st["slice_off"][s]), int(st["slice_off"][s + 1])
        m_s = b - a
        p1 = pass1.coarsen_slice(st["tree"], st["forest"], st["pts_s"], sc.vpls, sc.boxes, s, a, m_s,
                                 1.0, 0.0, 7)
        n_s = p1.col_node.size
        r2, c2, _, cap = pass2.draw_pass2(7, s, m_s, np.ones(n_s), p1.rows * n_s + p1.cols, 1.0)
        assert not cap
        nodes = p1.col_node[c2]
        v2 = shading.node_entries(st["pts_s"], sc.vpls, a + r2, st["tree"].rep[nodes],
                                  tree_mod.node_scale(st["tree"], sc.vpls, nodes), sc.boxes)
        rows = np.concatenate([p1.rows, r2]); cols = np.concatenate([p1.cols, c2])
        vals = np.concatenate([p1.vals, v2])
        assert rows.size == m_s * n_s
        U, V = als.complete_slice(rows, cols, vals, m_s, n_s, min(m_s, n_s), 2, 1e-13, 7, s)
        factors.append((U, V))
    img = render.render_slices(factors, st["row_perm"], st["slice_off"], sc.m, clamp=False)
    np.testing.assert_allclose(img, ref, rtol=1e-9, atol=1e-9 * ref.max())


def test_rel_rmse_definition():
    ref = np.array([3.0, 4.0])
    assert bruteforce.rel_rmse(np.array([3.0, 4.0]), ref) == 0.0
    assert abs(bruteforce.rel_rmse(np.array([0.0, 0.0]), ref) - 1.0) < 1e-15


# ---------------------------------------------------------------- 6-D recursive split slicing
def _line_points(xs, normal=(0.0, 1.0, 0.0)):
    P = np.zeros((3, len(xs), 4), dtype=np.float32)
    P[0, :, 0] = xs
    P[1, :, :3] = normal
    return P


def test_split_slices_of_points_on_a_line_are_runs_of_x():
    rng = np.random.default_rng(3)
    xs = rng.permutation(1000).astype(np.float32) / 1000
    perm, off = slices_mod.split6d_slices(_line_points(xs), 100)
    assert sorted(perm.tolist()) == list(range(1000))
    assert np.diff(off).tolist() == slices_mod.split_sizes(1000, 100)
    rank = np.argsort(np.argsort(xs))  # position of each pixel in x order
    for s in range(len(off) - 1):
        r = np.sort(rank[perm[off[s]:off[s + 1]]])
        assert r[-1] - r[0] == r.size - 1  # a contiguous run of the x order
        assert np.all(np.diff(perm[off[s]:off[s + 1]]) > 0)  # ascending pixels inside a slice
    starts = [rank[perm[off[s]:off[s + 1]]].min() for s in range(len(off) - 1)]
    assert starts == sorted(starts)  # left to right


def test_split_sizes_and_ties():
    assert slices_mod.split_sizes(1000, 100) == [62, 63, 62, 63, 62, 63, 62, 63, 62, 63, 62, 63, 62, 63, 62, 63]
    assert slices_mod.split_sizes(50, 100) == [50]
    assert slices_mod.split_sizes(7, 2) == [1, 2, 2, 2]
    # identical features: the split falls back to the pixel index
    perm, off = slices_mod.split6d_slices(_line_points(np.zeros(10, dtype=np.float32)), 3)
    assert perm.tolist() == list(range(10)) and off.tolist() == [0, 2, 5, 7, 10]


def test_split_takes_the_dimension_of_largest_extent():
    # x spans 1, the normal's z spans 2 w = 0.6 < 1 < ... ; with w = 1 the normal wins
    xs = np.linspace(0, 1, 8, dtype=np.float32)
    P = _line_points(xs)
    P[1, :, :3] = 0.0
    P[1, :4, 2] = 1.0
    P[1, 4:, 2] = -1.0
    P[1, ::2, 2] *= -1.0  # normal z alternates against x
    perm, off = slices_mod.split6d_slices(P, 4, w=0.3)
    assert sorted(perm[:4].tolist()) == [0, 1, 2, 3]  # split on x
    perm, off = slices_mod.split6d_slices(P, 4, w=1.0)
    nz = P[1, :, 2]
    assert np.all(nz[perm[:4]] < 0) and np.all(nz[perm[4:]] > 0)  # split on the normal


# ---------------------------------------------------------------- slice bounds (uneven slices)
def _cluster_points(centres_sizes, rng):
    """Points on three well separated clusters of given sizes (x positions), normal +y."""
    xs = np.concatenate([c + 0.001 * rng.standard_normal(n) for c, n in centres_sizes]).astype(np.float32)
    return _line_points(xs)


def test_bounds_merge_the_small_slice_into_the_nearest():
    rng = np.random.default_rng(11)
    P = _cluster_points([(0.0, 100), (0.1, 5), (1.0, 100)], rng)
    perm = np.arange(205)
    off = np.array([0, 100, 105, 205])
    p2, o2 = slices_mod.bound_slices(P, perm, off, 10, 1000)
    assert o2.tolist() == [0, 105, 205]                        # the 5 points join the cluster at 0.0
    assert p2[:105].tolist() == list(range(105))
    # placed nearer the far cluster, it joins that one (a wrong sign or index in the
    # distance, or the largest instead of the nearest, fails one of the two)
    P = _cluster_points([(0.0, 100), (0.9, 5), (1.0, 100)], rng)
    p2, o2 = slices_mod.bound_slices(P, perm, off, 10, 1000)
    assert o2.tolist() == [0, 100, 205] and p2[100:].tolist() == list(range(100, 205))


def test_bounds_split_like_the_recursive_split_and_keep_slices_in_bounds():
    rng = np.random.default_rng(12)
    xs = rng.permutation(1000).astype(np.float32) / 1000
    P = _line_points(xs)
    # one slice of all points above max_rows: the same parts as the recursive split
    p2, o2 = slices_mod.bound_slices(P, np.arange(1000), np.array([0, 1000]), 1, 100)
    q, oq = slices_mod.split6d_slices(P, 100)
    assert np.array_equal(p2, q) and np.array_equal(o2, oq)
    # loose bounds leave given slices as they are (pixels sorted inside each)
    perm = rng.permutation(1000)
    off = np.array([0, 300, 310, 700, 1000])
    p3, o3 = slices_mod.bound_slices(P, perm, off, 1, 1000)
    assert np.array_equal(o3, off)
    for s in range(4):
        assert p3[off[s]:off[s + 1]].tolist() == sorted(perm[off[s]:off[s + 1]].tolist())
    # tight bounds on a real scene's k-means slices: a partition, every slice in bounds
    cfg = get_config("room64_vpl1k_2box")
    sc = make_scene(cfg)
    rp, so, _, _ = slices_mod.kmeans_slices(sc.points, 16, 10, 0.3)
    p4, o4 = slices_mod.bound_slices(sc.points, rp, so, 200, 300)
    sizes = np.diff(o4)
    assert sorted(p4.tolist()) == list(range(sc.m))
    assert sizes.min() >= 150 and sizes.max() <= 300         # a split halves a slice of > 300
    assert np.diff(so).min() < 200 and np.diff(so).max() > 300  # both rules were exercised


# ---------------------------------------------------------------- coarsening to a target cut size
def _target_setup():
    cfg = get_config("room64_vpl1k_2box")
    sc = make_scene(cfg)
    st = pipeline.setup(sc, cfg)
    a, b = int(st["slice_off"][3]), int(st["slice_off"][4])
    run = lambda **kw: pass1.coarsen_slice(st["tree"], st["forest"], st["pts_s"], sc.vpls, sc.boxes, 3, a, b - a,
                                           cfg["rate1"], kw.pop("tau", cfg["tau"]), 7, cfg["d_min"], **kw)
    return st, run


def _same(x, y):
    return (np.array_equal(x.col_node, y.col_node) and np.array_equal(x.rows, y.rows)
            and np.array_equal(x.cols, y.cols) and np.array_equal(x.vals, y.vals) and np.array_equal(x.g, y.g))


def test_target_limits_equal_the_threshold_limits():
    st, run = _target_setup()
    C = st["forest"].C
    assert _same(run(target=C), run(tau=0.0))             # nothing merges
    assert _same(run(target=1), run(tau=float("inf")))    # everything merges


def test_target_sizes_are_met_and_nested():
    st, run = _target_setup()
    prev = None
    for T in (600, 300, 100, 20):
        r = run(target=T)
        assert r.col_node.size == T
        merged = {e[0] for e in r.log}
        if prev is not None:
            assert prev <= merged  # a smaller target merges a superset
        prev = merged


def test_target_order_is_the_effective_cost_order():
    """Greedy by cost among testable pairs merges the K pairs of smallest effective cost
    eff(f) = max(cost(f), eff(children)) (ties: lower height, lower id): the order the
    GPU selects by."""
    st, run = _target_setup()
    forest = st["forest"]
    C = forest.C
    full = run(tau=float("inf"))
    cost = {e[0]: e[2] for e in full.log}
    height = pass1.forest_heights(forest)
    eff = {}

    def get(f):
        if f < C:
            return 0.0
        if f not in eff:
            eff[f] = max(cost[f], get(int(forest.child[f, 0])), get(int(forest.child[f, 1])))
        return eff[f]

    order = sorted(cost, key=lambda f: (get(f), height[f], f))
    for T in (700, 400, 150, 30):
        r = run(target=T)
        assert {e[0] for e in r.log} == set(order[:C - T])


# ---------------------------------------------------------------- triangle occluders
def _box_triangles(b):
    """The 12 triangles of the closed box b = [lo xyz, hi xyz]."""
    lo, hi = np.asarray(b[:3], float), np.asarray(b[3:], float)
    c = np.array([[lo[0] if i & 1 == 0 else hi[0], lo[1] if i & 2 == 0 else hi[1], lo[2] if i & 4 == 0 else hi[2]]
                  for i in range(8)])
    quads = [(0, 1, 3, 2), (4, 5, 7, 6), (0, 1, 5, 4), (2, 3, 7, 6), (0, 2, 6, 4), (1, 3, 7, 5)]
    out = []
    for q0, q1, q2, q3 in quads:
        out.append([c[q0], c[q1], c[q2]])
        out.append([c[q0], c[q2], c[q3]])
    return np.array(out)


def test_box_as_triangles_blocks_the_same_segments():
    rng = np.random.default_rng(5)
    box = np.array([[0.3, 0.2, 0.4, 0.6, 0.5, 0.7]])
    o = rng.uniform(0, 1, (20000, 3))
    e = rng.uniform(0, 1, (20000, 3))
    inside = lambda x: np.all((x >= box[0, :3]) & (x <= box[0, 3:]), axis=1)
    keep = ~inside(o) & ~inside(e)  # a solid box also blocks a segment inside it, a surface does not
    o, e = o[keep], e[keep]
    by_box = shading.segment_blocked(o, e, box)
    by_tris = shading.segment_hits_triangles(o, e, _box_triangles(box[0]))
    assert by_box.sum() > 1000
    assert np.array_equal(by_box, by_tris)
    # the pair form tests both
    assert np.array_equal(shading.segment_blocked(o, e, (np.zeros((0, 6)), _box_triangles(box[0]))), by_box)


def test_single_triangle_cases():
    tri = np.array([[[0.0, 0.0, 0.5], [1.0, 0.0, 0.5], [0.0, 1.0, 0.5]]])
    o = np.array([[0.2, 0.2, 0.0], [0.8, 0.8, 0.0], [0.2, 0.2, 0.0], [0.2, 0.2, 0.5], [0.2, 0.2, 0.6]])
    e = np.array([[0.2, 0.2, 1.0], [0.8, 0.8, 1.0], [0.2, 0.2, 0.4], [0.9, 0.0, 0.5], [0.2, 0.2, 1.0]])
    # through the inside; outside the hypotenuse; ends before the plane; in the plane; starts behind it
    assert shading.segment_hits_triangles(o, e, tri).tolist() == [True, False, False, False, False]


def test_mesh_scene_full_sampling_reproduces_bruteforce():
    """The triangle occluders enter every shadow ray of the pipeline: at full sampling
    and full rank the frame equals the brute force over the mesh scene."""
    cfg = get_config("room64_vpl1k_mesh", width=8, height=8, n_vpl=12, n_slices=2, rate=1.0, eps_cut=0.0,
                     max_cut=100, tau=0.0, lam_rel=1e-13, als_iters=2, rank=12, rate1=1.0, mesh_subdiv=1)
    sc = make_scene(cfg)
    assert sc.tris is not None and sc.tris.shape[0] == 160
    ref = bruteforce.render(sc.points, sc.vpls, sc.occluders)
    nobox = bruteforce.render(sc.points, sc.vpls, sc.boxes)
    assert not np.allclose(ref, nobox)  # the spheres cast shadows
    img, _ = pipeline.render_frame(sc, cfg)
    # full-rank ALS on 32 x 12 slices with a 1e-13 ridge: exact up to its conditioning
    np.testing.assert_allclose(img, ref, rtol=1e-6, atol=1e-6 * ref.max())
