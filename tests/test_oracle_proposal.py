"""Pins of the learned-proposal oracle (oracle/proposal.py) against things that do
not come from the oracle itself: torch's bfloat16 conversion, finite differences,
numpy's SVD, closed-form feature values and a memorisation run."""
import numpy as np
import pytest

from oracle import proposal as P


def test_bf16_matches_torch_round_to_nearest_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-8, 8, size=20000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 3.4e38, -1e-40]])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = P.bf16(x)
    assert np.array_equal(got, want)


def _tiny_batch(seed=0, n=37, groups=(0, 11, 20, 37)):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, P.N_FEAT))
    theta = P.init_params(seed + 1) + rng.normal(size=P.N_PARAM) * 0.05
    go = np.array(groups)
    t = rng.random(n)
    for a, b in zip(go[:-1], go[1:]):
        t[a:b] /= t[a:b].sum()
    return X, theta, go, t


def test_backward_matches_central_differences():
    X, theta, go, t = _tiny_batch()

    def loss(th):
        z, _ = P.forward(th, X, rounding=False)
        return P.loss_and_dz(z, t, go)[0]

    z, cache = P.forward(theta, X, rounding=False)
    _, dz = P.loss_and_dz(z, t, go)
    g = P.backward(theta, cache, dz)
    rng = np.random.default_rng(9)
    idx = rng.choice(P.N_PARAM, 60, replace=False)
    idx = np.concatenate([idx, [P.N_PARAM - 1, 0, 2048, 10432]])  # b4, W1[0][0], b1[0], W4[0]
    h = 1e-6
    for i in idx:
        e = np.zeros(P.N_PARAM)
        e[i] = h
        fd = (loss(theta + e) - loss(theta - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_dz_of_the_group_cross_entropy():
    rng = np.random.default_rng(4)
    go = np.array([0, 5, 5, 12])  # an empty group too
    z = rng.normal(size=12)
    t = rng.random(12)
    t[:5] /= t[:5].sum()
    t[5:] /= t[5:].sum()
    L, dz = P.loss_and_dz(z, t, go)
    assert abs(dz[:5].sum()) < 1e-15 and abs(dz[5:].sum()) < 1e-15
    h = 1e-6
    for i in range(12):
        e = np.zeros(12)
        e[i] = h
        fd = (P.loss_and_dz(z + e, t, go)[0] - P.loss_and_dz(z - e, t, go)[0]) / (2 * h)
        assert abs(fd - dz[i]) < 1e-8
    # softmax equal to the target: zero gradient and loss = entropy of the target
    zz = np.log(t)
    L2, dz2 = P.loss_and_dz(zz, t, go)
    ent = -(np.sum(t[:5] * np.log(t[:5])) + np.sum(t[5:] * np.log(t[5:]))) / 3
    assert np.allclose(dz2, 0, atol=1e-15) and abs(L2 - ent) < 1e-12


def test_adam_memorises_a_one_hot_target():
    X, theta, go, _ = _tiny_batch(seed=5)
    t = np.zeros(X.shape[0])
    for a, b in zip(go[:-1], go[1:]):
        t[a + 1] = 1.0
    m = np.zeros(P.N_PARAM)
    v = np.zeros(P.N_PARAM)
    z, c = P.forward(theta, X)
    L0 = P.loss_and_dz(z, t, go)[0]
    for step in range(1, 301):
        z, c = P.forward(theta, X)
        L, dz = P.loss_and_dz(z, t, go)
        theta, m, v = P.adam(theta, m, v, P.backward(theta, c, dz), step, 3e-3)
    assert L0 > 1.5 and L < 0.05


def test_leverage_equals_svd_with_a_spectral_gap():
    rng = np.random.default_rng(11)
    m, n, r = 90, 40, 6
    U, _ = np.linalg.qr(rng.normal(size=(m, m)))
    V, _ = np.linalg.qr(rng.normal(size=(n, n)))
    sig = np.concatenate([np.geomspace(50, 20, r), np.geomspace(2, 0.1, n - r)])
    M = U[:, :n] * sig @ V.T
    lev = P.leverage(M, r, 30, seed=7, s=3)
    _, _, Vt = np.linalg.svd(M)
    want = np.sum(Vt[:r].T ** 2, axis=1)
    assert np.allclose(lev, want, atol=1e-9)
    assert abs(lev.sum() - r) < 1e-9
    t = P.targets(lev)
    assert abs(t.sum() - 1) < 1e-12 and np.all(t > 0)


def test_leverage_of_a_rank_one_matrix_is_the_column_energy():
    rng = np.random.default_rng(2)
    u, w = rng.random(30), rng.random(12) + 0.1
    lev = P.leverage(np.outer(u, w), 1, 5, seed=1, s=0)
    assert np.allclose(lev, w * w / np.dot(w, w), atol=1e-12)


class _Tree:
    def __init__(self):
        self.lo = np.array([[0, 0, 0], [0.1, 0.2, 0.3], [0.5, 0.5, 0.5]], dtype=np.float32)
        self.hi = np.array([[1, 1, 1], [0.2, 0.3, 0.4], [0.9, 0.8, 0.7]], dtype=np.float32)
        self.rep = np.array([0, 1, 0])
        self.I = np.array([4.0, 1.0, 3.0], dtype=np.float32)


def test_features_closed_form():
    pts = np.zeros((3, 5, 4), dtype=np.float32)
    pts[0, :, :3] = [[0.1, 0.2, 0.3], [0.3, 0.2, 0.1], [0.2, 0.5, 0.8], [9, 9, 9], [9, 9, 9]]
    pts[1, :, :3] = [[0, 1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 0], [0, 0, 0]]
    vpls = np.zeros((3, 2, 4), dtype=np.float32)
    vpls[0, :, :3] = [[0.4, 0.9, 0.4], [0.6, 0.99, 0.5]]
    vpls[1, :, :3] = [[0, -1, 0], [1, 0, 0]]
    cols = np.array([0, 0, 0, 1])
    vals = np.array([2.0, 2.0, 2.0, 6.0])
    F = P.slice_features(pts, 0, 3, _Tree(), vpls, np.array([1, 2]), cols, vals)
    mu = 3.0
    assert np.allclose(F[0, 0:3], [0.2, 0.3, 0.4]) and np.allclose(F[0, 3:6], [0, 2 / 3, -1 / 3])
    assert np.allclose(F[:, 6:9], [0.1, 0.2, 0.1]) and np.allclose(F[:, 9:12], [0.3, 0.5, 0.8])
    assert np.allclose(F[1, 12:18], [0.5, 0.5, 0.5, 0.9, 0.8, 0.7])
    assert np.allclose(F[0, 18:24], [0.6, 0.99, 0.5, 1, 0, 0]) and np.allclose(F[1, 18:24], [0.4, 0.9, 0.4, 0, -1, 0])
    assert np.allclose(F[:, 24], [np.log(0.25), np.log(0.75)])
    assert np.allclose(F[0, 25:30], [2 / mu, 0, np.log(4), 2 / mu, 2 / mu])  # equal values: no spread
    assert np.allclose(F[1, 25:30], [6 / mu, 0, np.log(2), 6 / mu, 6 / mu])
    assert np.allclose(F[:, 30], np.log(3) / 10) and np.allclose(F[:, 31], np.log(2) / 10)
    # a column without pass-1 values has zero statistics
    F2 = P.slice_features(pts, 0, 3, _Tree(), vpls, np.array([1, 2]), np.array([1]), np.array([5.0]))
    assert np.all(F2[0, 25:30] == 0)


def test_mixture_is_a_distribution_per_slice():
    rng = np.random.default_rng(1)
    go = np.array([0, 7, 19])
    w = P.mixture(rng.normal(size=19), rng.random(19), go)
    assert abs(w[:7].sum() - 1) < 1e-12 and abs(w[7:].sum() - 1) < 1e-12 and np.all(w > 0)
    # g all zero: the g part becomes uniform
    w2 = P.mixture(np.zeros(19), np.zeros(19), go)
    assert np.allclose(w2[:7], 1 / 7)
