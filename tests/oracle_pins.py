"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each pin returns (ok, detail). They are collected in PINS so that the mutation test can plant a
mistake in the oracle and check that at least one pin catches it.
"""
from __future__ import annotations

import numpy as np

import sasgen


def _rng(seed=1):
    return np.random.default_rng(seed)


def pin_phi_hat_closed_forms(O):
    """Quadrature of the window transform vs the KB and truncated-Gaussian closed forms."""
    worst = 0.0
    for kind in (O.KB, O.GAUSS):
        for w in (6, 8, 12):
            b = O.kernel_beta(w, 2.0, kind)
            xi = np.linspace(-0.3, 0.3, 31)
            q = O.phi_hat(xi, w, b, kind)
            cf = O.phi_hat_closed(xi, w, b, kind)
            worst = max(worst, float(np.max(np.abs(q - cf) / np.abs(cf))))
    return worst < 1e-11, f"max rel err {worst:.2e}"


def pin_phi_hat_es_simpson(O):
    """ES transform at a few frequencies vs a composite Simpson rule on 200001 points in t."""
    w, sigma = 8, 2.0
    b = O.kernel_beta(w, sigma)
    t = np.linspace(-w / 2, w / 2, 200001)
    f = O.phi(t, w, b)
    worst = 0.0
    for xi in (0.0, 0.1, 0.25):
        g = f * np.cos(2 * np.pi * xi * t)
        h = t[1] - t[0]
        simpson = h / 3 * (g[0] + g[-1] + 4 * g[1:-1:2].sum() + 2 * g[2:-1:2].sum())
        worst = max(worst, abs(O.phi_hat(xi, w, b) - simpson) / abs(simpson))
    return worst < 1e-8, f"max rel err {worst:.2e}"


def pin_uniform_grid_is_fft(O):
    """Integer raster lambda = {-N/2..N/2-1}^2: the direct sum is N^2 ifft2 of the samples placed
    at lambda mod N (the data frame is an orthonormal basis there)."""
    N = 16
    g = np.arange(-N // 2, N // 2)
    X, Y = np.meshgrid(g, g)
    lam = np.stack([X.ravel(), Y.ravel()], 1).astype(np.float64)
    rng = _rng(2)
    c = rng.standard_normal(N * N) + 1j * rng.standard_normal(N * N)
    C = np.zeros((N, N), np.complex128)
    C[np.mod(Y.ravel(), N), np.mod(X.ravel(), N)] = c
    ref = np.fft.ifft2(C) * N * N
    p = np.mod(np.arange(-N // 2, N // 2), N)
    ref = ref[np.ix_(p, p)]
    I1 = O.direct_adjoint(lam, c, N)
    e1 = O.rel_l2(I1, ref)
    I2 = O.adjoint(lam, c, N, 2.0, 8)
    e2 = O.rel_l2(I2, ref)
    return e1 < 1e-13 and e2 < 1e-6, f"direct {e1:.2e} gridded {e2:.2e}"


def pin_gridder_vs_direct(O):
    """O2 (gridding) vs O1 (direct sum) on the tiny raster: the ES window's aliasing bound at
    sigma = 2 (w=6: 8.5e-6 measured, bound 1.2e-5; w=8: 1.3e-7, bound 2e-7)."""
    p = sasgen.tiny()
    v = sasgen.values_for(p)
    I1 = O.direct_adjoint(p.lam, v, p.N)
    e6 = O.rel_l2(O.adjoint(p.lam, v, p.N, 2.0, 6), I1)
    e8 = O.rel_l2(O.adjoint(p.lam, v, p.N, 2.0, 8), I1)
    return e6 < 1.2e-5 and e8 < 2e-7, f"w6 {e6:.2e} w8 {e8:.2e}"


def pin_gridder_random_wrap(O):
    """Random samples spread over three periods (wrap mod G) and a non-square sigma = 1.5 case."""
    ok = True
    msgs = []
    for (M, N, sigma, w, spread, bound) in ((700, 32, 2.0, 8, 96, 2e-7), (500, 24, 1.5, 10, 24, 1e-5)):
        lam, v = sasgen.random_case(5, M, N, sigma, w, spread)
        e = O.rel_l2(O.adjoint(lam, v, N, sigma, w), O.direct_adjoint(lam, v, N))
        ok &= e < bound
        msgs.append(f"{e:.2e}")
    return ok, " ".join(msgs)


def pin_forward_vs_direct(O):
    """Gridded type-2 transform vs the exact sum over pixels."""
    lam, _ = sasgen.random_case(6, 400, 32, spread=40)
    rng = _rng(7)
    img = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    e = O.rel_l2(O.forward(lam, img, 32, 2.0, 8), O.direct_forward(lam, img, 32))
    return e < 2e-7, f"{e:.2e}"


def pin_adjointness(O):
    """<A c, I> = <c, A^H I> for the gridded pair, to FP64 rounding."""
    lam, c = sasgen.random_case(8, 300, 24, spread=30)
    rng = _rng(9)
    img = rng.standard_normal((24, 24)) + 1j * rng.standard_normal((24, 24))
    lhs = np.vdot(img, O.adjoint(lam, c, 24, 2.0, 7))
    rhs = np.vdot(O.forward(lam, img, 24, 2.0, 7), c)
    e = abs(lhs - rhs) / abs(lhs)
    return e < 1e-12, f"{e:.2e}"


def pin_pixels_vs_direct(O):
    """Pixel-at-a-time O2 vs the direct sum at the same pixels (and vs full O2)."""
    lam, c = sasgen.random_case(10, 500, 32, spread=32)
    pix = np.array([[-16, -16], [0, 0], [15, -3], [7, 11]])
    got = O.adjoint_pixels(lam, c, 32, 2.0, 8, pix)
    full = O.adjoint(lam, c, 32, 2.0, 8)[pix[:, 1] + 16, pix[:, 0] + 16]
    d = O.direct_adjoint(lam, c, 32)[pix[:, 1] + 16, pix[:, 0] + 16]
    e1 = float(np.max(np.abs(got - full)) / np.max(np.abs(full)))
    e2 = float(np.max(np.abs(got - d)) / np.max(np.abs(d)))
    return e1 < 1e-12 and e2 < 1e-6, f"vs full {e1:.2e} vs direct {e2:.2e}"


def pin_point_scatterer(O):
    """A scatterer at a pixel centre peaks at that pixel; one off the lattice peaks within 1 px."""
    rng = _rng(11)
    kx, ky = sasgen.polar_raster(rng, 48, 48, 30.0)
    L, N = 0.3, 32          # the raster spans about 13 x 27 cycles: inside one period
    lam = sasgen.baseband(kx, ky, L)
    ok = True
    msg = []
    for px, py, off in ((5, -7, 0.0), (-9, 4, 0.37)):
        pos = np.array([[(px + off) * L / N, (py - off) * L / N]])
        scene = sasgen.Scene(pos, np.array([1.0 + 0j]), L)
        v = sasgen.sample_values(lam, scene)
        I = O.adjoint(lam, v, N, 2.0, 8)
        iy, ix = np.unravel_index(np.argmax(np.abs(I)), I.shape)
        gy, gx = iy - N // 2, ix - N // 2
        if off == 0.0:
            ok &= (gx, gy) == (px, py)
        else:
            ok &= abs(gx - (px + off)) <= 1 and abs(gy - (py - off)) <= 1
        msg.append(f"({gx},{gy})")
    return ok, " ".join(msg)


def pin_tie_rule(O):
    """u - w/2 on an integer: the first tap is at distance exactly w/2 to the left."""
    lam = np.array([[3.0, -2.5], [0.25, 7.0]])
    c, u = O.tap_origins(lam, 16, 2.0, 8)
    ok = bool(np.all(c == np.array([[2, -9], [-3, 10]])))
    return ok, str(c.tolist())


def pin_weights_uniform(O):
    """Full integer raster: alpha = 1; an s-times oversampled full period: alpha = 1/s^2."""
    N = 12
    g = np.arange(-N // 2, N // 2)
    X, Y = np.meshgrid(g, g)
    lam = np.stack([X.ravel(), Y.ravel()], 1).astype(np.float64)
    a, _ = O.weights_brute(lam, N)
    e0 = float(np.max(np.abs(a - 1)))
    an, _ = O.weights_nufft(lam, N, w_alpha=12)
    e1 = float(np.max(np.abs(an - 1)))
    worst = 0.0
    for s in (2, 3):
        gg = np.arange(s * N) / s - N / 2 + 0.3
        X, Y = np.meshgrid(gg, gg)
        lam = np.stack([X.ravel(), Y.ravel()], 1)
        a, _ = O.weights_brute(lam, N)
        worst = max(worst, float(np.max(np.abs(a * s * s - 1))))
    return e0 < 1e-13 and e1 < 1e-9 and worst < 1e-12, f"{e0:.1e} {e1:.1e} {worst:.1e}"


def pin_weights_gram(O):
    """S_k equals sum_j |T_jk|^2 with T summed explicitly over the pixel lattice, and the
    diagonal LS optimum: the residual || T_{:,k} a - e_k || is smallest at a = alpha_k."""
    p = sasgen.tiny()
    lam = p.lam[::4]
    ks = [0, 77, 500]
    a, S = O.weights_brute(lam, p.N, ks)
    worst = 0.0
    opt = True
    for i, k in enumerate(ks):
        T = O.gram_column(lam, p.N, k)
        worst = max(worst, abs(np.sum(np.abs(T) ** 2) - S[i]) / S[i])
        e = np.zeros(lam.shape[0])
        e[k] = 1
        r0 = np.linalg.norm(T * a[i] - e)
        for f in (1 - 1e-3, 1 + 1e-3):
            opt &= r0 < np.linalg.norm(T * a[i] * f - e)
    return worst < 1e-12 and opt, f"{worst:.1e} optimal={opt}"


def pin_weights_route(O):
    """Fast NUFFT route of the weights vs the O(M^2) Fejer sum on the tiny raster."""
    p = sasgen.tiny()
    ab, _ = O.weights_brute(p.lam, p.N)
    an, S = O.weights_nufft(p.lam, p.N, w_alpha=12)
    e = float(np.max(np.abs(an - ab) / ab))
    im = float(np.max(np.abs(S.imag) / S.real))
    return e < 1e-10 and im < 1e-12, f"{e:.2e} imag {im:.1e}"


PINS = [
    pin_phi_hat_closed_forms,
    pin_phi_hat_es_simpson,
    pin_uniform_grid_is_fft,
    pin_gridder_vs_direct,
    pin_gridder_random_wrap,
    pin_forward_vs_direct,
    pin_adjointness,
    pin_pixels_vs_direct,
    pin_point_scatterer,
    pin_tie_rule,
    pin_weights_uniform,
    pin_weights_gram,
    pin_weights_route,
]
