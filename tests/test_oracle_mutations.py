"""Plant a plausible mistake in the oracle (on the CPU) and check that some pin fails.

Each mutation replaces one oracle function for the duration of the test; the pins call the
module's functions through the module, so the mistake propagates to every caller."""
import numpy as np
import pytest

from oracle import ftcg_oracle as O
from tests.oracle_pins import PINS

_orig = {k: getattr(O, k) for k in dir(O) if callable(getattr(O, k))}


def _sign_flip_direct(lam, c, N):
    """exp(-2 pi i ...) in place of exp(+2 pi i ...)."""
    return _orig["direct_adjoint"](-np.asarray(lam), c, N)


def _drop_last_tap(u, c, w, beta, kind):
    out = _orig["tap_weights"](u, c, w, beta, kind)
    out[:, -1] = 0.0
    return out


def _floor_origin(lam, N, sigma, w):
    u = float(sigma) * np.asarray(lam, dtype=np.float64)
    return np.floor(u - 0.5 * w).astype(np.int64), u


def _deapod_wrong_scale(N, sigma, w, kind=O.ES, beta=None):
    if beta is None:
        beta = O.kernel_beta(w, sigma, kind)
    return 1.0 / O.phi_hat(O.pixel_range(N) / N, w, beta, kind)


def _fejer_no_norm(delta, N):
    return _orig["fejer"](delta, N) * N * N


def _lag_weights_wrong(N):
    d = np.arange(-N, N)
    c1 = (N - np.abs(d)) / float(N)
    return np.multiply.outer(c1, c1) / (N * N * N)


def _transposed_origins(lam, N, sigma, w):
    c, u = _orig["tap_origins"](lam, N, sigma, w)
    return c[:, ::-1].copy(), u[:, ::-1].copy()


def _phi_hat_no_jacobian(xi, w, beta, kind=O.ES, n=200):
    x, wt = np.polynomial.legendre.leggauss(n)
    th = 0.25 * np.pi * (x + 1.0)
    t = 0.5 * w * np.sin(th)
    f = O.phi(t, w, beta, kind) * wt * 0.25 * np.pi * 0.5 * w
    return 2.0 * np.cos(2.0 * np.pi * np.multiply.outer(np.asarray(xi, float), t)) @ f


def _beta_off(w, sigma, kind=O.ES):
    return _orig["kernel_beta"](w, sigma, kind) * 0.7


def _spread_clipped(lam, c, N, sigma, w, kind=O.ES, beta=None):
    """Taps past the grid edge clipped to the edge instead of wrapped mod G."""
    G = O.grid_side(N, sigma)
    if beta is None:
        beta = O.kernel_beta(w, sigma, kind)
    org, u = O.tap_origins(lam, N, sigma, w)
    wx = O.tap_weights(u[:, 0], org[:, 0], w, beta, kind)
    wy = O.tap_weights(u[:, 1], org[:, 1], w, beta, kind)
    grid = np.zeros((G, G), np.complex128)
    for ty in range(w):
        iy = np.clip(org[:, 1] + ty, 0, G - 1)
        for tx in range(w):
            ix = np.clip(org[:, 0] + tx, 0, G - 1)
            np.add.at(grid, (iy, ix), np.asarray(c, np.complex128) * wy[:, ty] * wx[:, tx])
    return grid


def _forward_sign(lam, img, N, sigma, w, kind=O.ES, beta=None):
    """The gridded forward transform with the exponent's sign flipped."""
    return _orig["forward"](-np.asarray(lam), img, N, sigma, w, kind, beta)


def _fejer_unsquared(delta, N):
    """The Dirichlet magnitude where the squared (Fejer) kernel belongs."""
    return np.sqrt(_orig["fejer"](delta, N))


def _pixels_shifted(lam, c, N, sigma, w, pix, kind=O.ES, beta=None):
    return _orig["adjoint_pixels"](lam, c, N, sigma, w, np.asarray(pix) + np.array([1, 0]), kind,
                                   beta)


MUTATIONS = {
    "spread_clip": ("spread", _spread_clipped),
    "forward_sign": ("forward", _forward_sign),
    "fejer_unsquared": ("fejer", _fejer_unsquared),
    "pixels_shift": ("adjoint_pixels", _pixels_shifted),
    "direct_sign": ("direct_adjoint", _sign_flip_direct),
    "drop_tap": ("tap_weights", _drop_last_tap),
    "floor_origin": ("tap_origins", _floor_origin),
    "deapod_scale": ("deapod_factors", _deapod_wrong_scale),
    "fejer_norm": ("fejer", _fejer_no_norm),
    "lag_weights": ("fejer_lag_weights", _lag_weights_wrong),
    "xy_swap": ("tap_origins", _transposed_origins),
    "no_jacobian": ("phi_hat", _phi_hat_no_jacobian),
    "beta_off": ("kernel_beta", _beta_off),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(O, attr, fn)
    failed = []
    for pin in PINS:
        try:
            ok, _ = pin(O)
        except Exception:
            ok = False
        if not ok:
            failed.append(pin.__name__)
    assert failed, f"mutation {name} passed every pin"
