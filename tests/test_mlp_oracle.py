"""Pins of the learned-weight oracle (no GPU): finite differences for every gradient, GELU's
known values, brute-force kNN against a k-d tree, and Adam's first step."""
import numpy as np
import pytest

from oracle import mlp_oracle as L


def test_gelu_known_values():
    z = np.array([0.0, 10.0, -10.0])
    g = L.gelu(z)
    assert g[0] == 0.0 and abs(g[1] - 10.0) < 1e-12 and abs(g[2]) < 1e-12
    assert abs(L.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    zz = np.linspace(-4, 4, 101)
    fd = (L.gelu(zz + 1e-6) - L.gelu(zz - 1e-6)) / 2e-6
    assert np.max(np.abs(fd - L.gelu_grad(zz))) < 1e-8


def test_gradients_finite_differences():
    rng = np.random.default_rng(0)
    P = L.init_params(rng)
    P["w4"] = rng.standard_normal(L.HID) * 0.3
    X = rng.standard_normal((13, L.D_IN))
    t = rng.standard_normal(13)
    y, cache = L.forward(P, X)
    g = L.backward(P, cache, y, t)
    for k in P:
        flat = P[k].reshape(-1)
        for i in rng.choice(flat.size, min(6, flat.size), replace=False):
            old = flat[i]
            flat[i] = old + 1e-6
            lp = L.loss(L.forward(P, X)[0], t)
            flat[i] = old - 1e-6
            lm = L.loss(L.forward(P, X)[0], t)
            flat[i] = old
            fd = (lp - lm) / 2e-6
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, i, fd, an)


def test_knn_matches_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(1)
    lam = rng.random((400, 2)) * 20
    X, idx = L.knn_features(lam, np.zeros(400))
    tree = spatial.cKDTree(lam)
    d, j = tree.query(lam, k=L.K_NN + 1)
    assert np.array_equal(np.sort(j[:, 1:], axis=1), np.sort(idx, axis=1))
    off = X[:, :2 * L.K_NN].reshape(400, L.K_NN, 2)
    dist = np.hypot(off[..., 0], off[..., 1])
    assert np.all(np.diff(dist, axis=1) >= 0)
    assert np.allclose(dist, d[:, 1:], rtol=0, atol=1e-12)


def test_knn_ties_by_index():
    g = np.arange(5.0)
    X, Y = np.meshgrid(g, g)
    lam = np.stack([X.ravel(), Y.ravel()], 1)
    _, idx = L.knn_features(lam, np.zeros(25), k=4)
    # the centre (2, 2) = index 12 has four neighbours at distance 1: indices 7, 11, 13, 17
    assert idx[12].tolist() == [7, 11, 13, 17]


def test_adam_first_step_is_signed_lr():
    P = {"a": np.array([1.0, -2.0, 3.0])}
    g = {"a": np.array([0.5, -4.0, 0.0])}
    L.adam_step(P, g, {}, lr=0.01)
    # after bias correction m/sqrt(v) = sign(g) on the first step (0 where g = 0)
    assert np.allclose(P["a"], [0.99, -1.99, 3.0], atol=1e-6)


def test_training_reduces_loss():
    rng = np.random.default_rng(2)
    P = L.init_params(rng)
    X = rng.standard_normal((256, L.D_IN)) * 0.5
    t = np.tanh(X[:, 0] - 0.5 * X[:, 3])
    st = {}
    l0 = L.loss(L.forward(P, X)[0], t)
    for _ in range(200):
        y, c = L.forward(P, X)
        L.adam_step(P, L.backward(P, c, y, t), st, lr=3e-3)
    assert L.loss(L.forward(P, X)[0], t) < 0.2 * l0


# ---- planted mistakes: each must make one of the pins above fail --------------------------------

_ORIG = {k: getattr(L, k) for k in ("gelu_grad", "backward", "adam_step", "knn_features")}


def _gelu_grad_no_cubic(z):
    u = L._C * (z + 0.044715 * z ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * L._C


def _backward_transposed(P, cache, y, t):
    """W3 used untransposed when the error flows back through it (square, so no shape error)."""
    Q = dict(P)
    Q["W3"] = P["W3"].T
    return _ORIG["backward"](Q, cache, y, t)


def _adam_no_bias_correction(P, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    for k in P:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] * g[k]
        P[k] = P[k] - lr * m / (np.sqrt(v) + eps)
    return P


def _knn_ties_reversed(lam, aux, k=L.K_NN):
    """Neighbours at equal distance taken by larger index first."""
    M = np.asarray(lam).shape[0]
    X, idx = _ORIG["knn_features"](np.asarray(lam)[::-1], np.asarray(aux)[::-1], k)
    return X[::-1], (M - 1 - idx)[::-1]


@pytest.mark.parametrize("name,mutant,pin", [
    ("gelu_grad", _gelu_grad_no_cubic, "test_gelu_known_values"),
    ("backward", _backward_transposed, "test_gradients_finite_differences"),
    ("adam_step", _adam_no_bias_correction, "test_adam_first_step_is_signed_lr"),
    ("knn_features", _knn_ties_reversed, "test_knn_ties_by_index"),
])
def test_planted_mistake_is_caught(monkeypatch, name, mutant, pin):
    monkeypatch.setattr(L, name, mutant)
    with pytest.raises(AssertionError):
        globals()[pin]()
