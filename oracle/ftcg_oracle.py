"""FP64 CPU oracle for the weighted 2-D adjoint NUFFT of frame theoretic convolutional gridding.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this module: only the tests, the
smoke check and the CPU-baseline leg of the benchmark do. It shares no code with the CUDA
library; it is plain numpy in float64 / complex128, written to be read against the paper.

Notation (McKay, Gelb, Monga, Raj, "Using Frame Theoretic Convolutional Gridding for Robust
Synthetic Aperture Sonar Imaging", Sec. III-IV):
  lambda_j in R^2   sample positions (cycles per field of view), j = 0..M-1
  v_j               sample values f^(lambda_j)
  alpha_j           diagonal quadrature weights, D_2 = diag(alpha) (Eq. twodcgmatrix)
  N                 output image side, pixels p in {-N/2 .. N/2-1}^2
  sigma, G=sigma N  oversampling and fine-grid side (the index set I_L of Eq. twodcg)
  w                 kernel width in fine-grid cells (support of w^ in Eq. twodcg)

Every function cites the passage it follows. Readings where the paper is silent:
  R1 reconstruction uses exp(+2 pi i lambda.p/N) on a centred unit FOV (Eq. twodcg's sign).
  R2 the fine grid has spacing 1/sigma cycles per FOV and is periodic with G cells.
  R3 the window is the exponential of semicircle (ES) kernel; Kaiser-Bessel and truncated
     Gaussian are options (Sec. III-A names the Gaussian and 'several other options').
  R4 taps are the w cells starting at ceil(u - w/2); indices wrap mod G.
  R5 FTCG diagonal weights: alpha_k = 1 / sum_j F_N(lambda_j - lambda_k) (Eq. difopt with
     T = Psi Omega read as the data-frame Gram matrix on the N x N pixel lattice).
"""
from __future__ import annotations

import numpy as np

try:  # complex erf for the truncated-Gaussian closed form (pins only)
    from scipy.special import erf as _erf
    from scipy.special import i0 as _i0
except Exception:  # pragma: no cover
    _erf = None
    _i0 = None

ES, KB, GAUSS = 0, 1, 2


# --------------------------------------------------------------------------------------------
# The window (Sec. III-A: w positive, essentially compactly supported; w^ analytic)
# --------------------------------------------------------------------------------------------

def kernel_beta(w, sigma, kind=ES):
    """Shape parameter of the window for width w and oversampling sigma (reading R3).

    ES: beta = 0.97 pi (1 - 1/(2 sigma)) w (Barnett, Magland, af Klinteberg 2019).
    KB: beta = pi sqrt((w/sigma)^2 (sigma - 1/2)^2 - 0.8) (Beatty, Nishimura, Pauly 2005).
    Gaussian: phi(w/2) = exp(-beta) with beta = pi w (1 - 1/(2 sigma)) / 2."""
    if kind == ES:
        return 0.97 * np.pi * (1.0 - 0.5 / sigma) * w
    if kind == KB:
        return np.pi * np.sqrt((w / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8)
    if kind == GAUSS:
        return 0.5 * np.pi * w * (1.0 - 0.5 / sigma)
    raise ValueError(kind)


def phi(t, w, beta, kind=ES):
    """The spreading window evaluated at offset t (fine-grid cells), zero for |t| > w/2."""
    t = np.asarray(t, dtype=np.float64)
    z = 2.0 * t / w
    inside = np.abs(z) <= 1.0
    zz = np.where(inside, z, 0.0)
    if kind == ES:
        val = np.exp(beta * (np.sqrt(1.0 - zz * zz) - 1.0))
    elif kind == KB:
        val = _i0(beta * np.sqrt(1.0 - zz * zz)) / _i0(beta)
    elif kind == GAUSS:
        val = np.exp(-beta * zz * zz)
    else:
        raise ValueError(kind)
    return np.where(inside, val, 0.0)


def phi_hat(xi, w, beta, kind=ES, n=200):
    """Fourier transform of the window, phi^(xi) = int phi(t) exp(-2 pi i xi t) dt (real, even).

    The window divided out in zeta_n = psi_n / w(x) (Eq. newadm) is, on the fine grid, this
    transform at xi = p / G (Poisson summation of Eq. twodcg). Computed by Gauss-Legendre
    quadrature after t = (w/2) sin(theta), which removes the square-root edge of ES/KB."""
    xi = np.asarray(xi, dtype=np.float64)
    x, wt = np.polynomial.legendre.leggauss(n)
    th = 0.25 * np.pi * (x + 1.0)          # [0, pi/2]
    wt = wt * 0.25 * np.pi
    t = 0.5 * w * np.sin(th)
    jac = 0.5 * w * np.cos(th)
    f = phi(t, w, beta, kind) * jac * wt      # (n,)
    return 2.0 * np.cos(2.0 * np.pi * np.multiply.outer(xi, t)) @ f


def phi_hat_closed(xi, w, beta, kind):
    """Closed forms used to pin phi_hat: KB (Jackson et al. 1991 form) and truncated Gaussian."""
    xi = np.asarray(xi, dtype=np.float64)
    if kind == KB:
        a = np.sqrt(np.asarray(beta ** 2 - (np.pi * w * xi) ** 2, dtype=np.complex128))
        return (w * np.sinh(a) / a).real / _i0(beta)
    if kind == GAUSS:
        # phi(t) = exp(-t^2 / (2 s^2)) on |t| <= w/2 with s^2 = (w/2)^2 / (2 beta)
        s = 0.5 * w / np.sqrt(2.0 * beta)
        a = 0.5 * w
        z = (a + 1j * 2 * np.pi * s * s * xi) / (s * np.sqrt(2.0))
        return (s * np.sqrt(2 * np.pi) * np.exp(-2 * np.pi ** 2 * s * s * xi * xi) * _erf(z)).real
    raise ValueError(kind)


# --------------------------------------------------------------------------------------------
# O1: the target result, written out (Eq. twodcg with the window removed and I_L = Z^2)
# --------------------------------------------------------------------------------------------

def pixel_range(N):
    return np.arange(-(N // 2), N - N // 2)


def direct_adjoint(lam, c, N):
    """I_p = sum_j c_j exp(+2 pi i lambda_j . p / N), p in {-N/2..N/2-1}^2 (reading R1).

    Returned as an N x N complex128 array indexed [p_y + N/2, p_x + N/2]. The exponential
    factorises over the two axes, so the sum is the matrix product Ey^T diag(c) Ex."""
    p = pixel_range(N).astype(np.float64)
    ex = np.exp(2j * np.pi * np.multiply.outer(lam[:, 0], p) / N)
    ey = np.exp(2j * np.pi * np.multiply.outer(lam[:, 1], p) / N)
    return ey.T @ (np.asarray(c, np.complex128)[:, None] * ex)


def direct_forward(lam, img, N):
    """f_k = sum_p I_p exp(-2 pi i lambda_k . p / N): the data frame of Eq. (twoddataframe)
    applied to an image, i.e. the exact adjoint of direct_adjoint."""
    p = pixel_range(N).astype(np.float64)
    ex = np.exp(-2j * np.pi * np.multiply.outer(lam[:, 0], p) / N)
    ey = np.exp(-2j * np.pi * np.multiply.outer(lam[:, 1], p) / N)
    return np.einsum("jy,yx,jx->j", ey, img, ex)


# --------------------------------------------------------------------------------------------
# O2: convolutional gridding step by step (Eq. twodcg / twodcgmatrix), FP64
# --------------------------------------------------------------------------------------------

def grid_side(N, sigma):
    G = sigma * N
    if abs(G - round(G)) > 1e-9 or int(round(G)) % 2:
        raise ValueError("sigma * N must be an even integer")
    return int(round(G))


def tap_origins(lam, N, sigma, w):
    """u_j = sigma lambda_j (fine-grid units); the first tap c_j = ceil(u_j - w/2) (reading R4).
    Returns (c as int64 M x 2, u as float64 M x 2). Rows of Omega_2 are nonzero exactly at
    l = c_j + t, t in {0..w-1}^2 (Eq. twodcgmatrix)."""
    u = float(sigma) * np.asarray(lam, dtype=np.float64)
    c = np.ceil(u - 0.5 * w).astype(np.int64)
    return c, u


def tap_weights(u, c, w, beta, kind):
    """phi(u - c - t) for t = 0..w-1 along one axis: M x w."""
    t = np.arange(w, dtype=np.float64)
    return phi((u - c)[:, None] - t[None, :], w, beta, kind)


def spread(lam, c, N, sigma, w, kind=ES, beta=None):
    """g_l = sum_j c_j phi(u_jx - l_x) phi(u_jy - l_y) over the w x w taps of each sample, l mod G.

    This is gamma = Omega_2 (D_2 f^) of Eq. (twodcgmatrix) with c = D_2 f^ already formed.
    Returns the G x G complex128 grid indexed [l_y, l_x]."""
    G = grid_side(N, sigma)
    if beta is None:
        beta = kernel_beta(w, sigma, kind)
    org, u = tap_origins(lam, N, sigma, w)
    wx = tap_weights(u[:, 0], org[:, 0], w, beta, kind)
    wy = tap_weights(u[:, 1], org[:, 1], w, beta, kind)
    c = np.asarray(c, np.complex128)
    grid = np.zeros(G * G, np.complex128)
    ix = np.mod(org[:, 0:1] + np.arange(w)[None, :], G)          # M x w columns of the taps
    for ty in range(w):                                          # one row of taps at a time
        iy = np.mod(org[:, 1] + ty, G)
        idx = (iy[:, None] * G + ix).ravel()
        val = ((c * wy[:, ty])[:, None] * wx).ravel()
        grid += np.bincount(idx, weights=val.real, minlength=G * G)
        grid += 1j * np.bincount(idx, weights=val.imag, minlength=G * G)
    return grid.reshape(G, G)


def deapod_factors(N, sigma, w, kind=ES, beta=None):
    """1 / phi^(p / G) for p = -N/2..N/2-1: division by the window (Eq. newadm)."""
    G = grid_side(N, sigma)
    if beta is None:
        beta = kernel_beta(w, sigma, kind)
    return 1.0 / phi_hat(pixel_range(N) / G, w, beta, kind)


def adjoint(lam, c, N, sigma, w, kind=ES, beta=None):
    """O2: A^2_cg applied to c = D_2 f^ (Eq. twodcg): spread onto the periodic fine grid,
    unnormalised inverse DFT sum_l g_l exp(+2 pi i l.q/G), keep q = p mod G, divide by the
    window transform. Returns N x N complex128 indexed [p_y + N/2, p_x + N/2]."""
    G = grid_side(N, sigma)
    if beta is None:
        beta = kernel_beta(w, sigma, kind)
    g = spread(lam, c, N, sigma, w, kind, beta)
    h = np.fft.ifft2(g) * (G * G)
    p = pixel_range(N)
    q = np.mod(p, G)
    r = deapod_factors(N, sigma, w, kind, beta)
    return h[np.ix_(q, q)] * r[:, None] * r[None, :]


def forward(lam, img, N, sigma, w, kind=ES, beta=None):
    """The conjugate transpose of `adjoint` (the gridded type-2 transform): place
    I_p / (phi^ phi^) at q = p mod G, forward DFT sum_q g_q exp(-2 pi i l.q/G), then interpolate
    f_k = sum_taps phi phi h_l. Approximates direct_forward."""
    G = grid_side(N, sigma)
    if beta is None:
        beta = kernel_beta(w, sigma, kind)
    p = pixel_range(N)
    q = np.mod(p, G)
    r = deapod_factors(N, sigma, w, kind, beta)
    g = np.zeros((G, G), np.complex128)
    g[np.ix_(q, q)] = np.asarray(img, np.complex128) * r[:, None] * r[None, :]
    h = np.fft.fft2(g)
    org, u = tap_origins(lam, N, sigma, w)
    wx = tap_weights(u[:, 0], org[:, 0], w, beta, kind)
    wy = tap_weights(u[:, 1], org[:, 1], w, beta, kind)
    out = np.zeros(lam.shape[0], np.complex128)
    for ty in range(w):
        iy = np.mod(org[:, 1] + ty, G)
        for tx in range(w):
            ix = np.mod(org[:, 0] + tx, G)
            out += wy[:, ty] * wx[:, tx] * h[iy, ix]
    return out


def adjoint_pixels(lam, c, N, sigma, w, pix, kind=ES, beta=None):
    """O2 at selected pixels only, one by one: the inverse DFT of the spread grid evaluated at a
    single q = p mod G is sum_j c_j (sum_tx phi e^{2 pi i l_x p_x / G})(sum_ty phi e^{...}),
    divided by phi^(p_x/G) phi^(p_y/G). `pix` is K x 2 integer (p_x, p_y). Equals `adjoint`
    at those pixels up to rounding, at O(M w) per pixel."""
    G = grid_side(N, sigma)
    if beta is None:
        beta = kernel_beta(w, sigma, kind)
    org, u = tap_origins(lam, N, sigma, w)
    wx = tap_weights(u[:, 0], org[:, 0], w, beta, kind)
    wy = tap_weights(u[:, 1], org[:, 1], w, beta, kind)
    t = np.arange(w)
    c = np.asarray(c, np.complex128)
    # the cell l = c_j + t: exp(2 pi i l p / G) = exp(2 pi i c_j p / G) exp(2 pi i t p / G), and
    # the wrap l mod G does not change it (p and l are integers)
    ox = np.mod(org[:, 0], G)
    oy = np.mod(org[:, 1], G)
    out = np.empty(len(pix), np.complex128)
    for i, (px, py) in enumerate(np.asarray(pix)):
        sx = (wx @ np.exp(2j * np.pi * t * px / G)) * np.exp(2j * np.pi * np.mod(ox * px, G) / G)
        sy = (wy @ np.exp(2j * np.pi * t * py / G)) * np.exp(2j * np.pi * np.mod(oy * py, G) / G)
        den = phi_hat(px / G, w, beta, kind) * phi_hat(py / G, w, beta, kind)
        out[i] = np.sum(c * sx * sy) / den
    return out


# --------------------------------------------------------------------------------------------
# FTCG diagonal weights (Eq. difopt, reading R5)
# --------------------------------------------------------------------------------------------

def fejer(delta, N):
    """Normalised Fejer kernel F_N(d) = sin^2(pi d) / (N^2 sin^2(pi d / N)), = 1 on d in N Z.

    |T_jk|^2 per axis where T_jk = (1/N^2) sum_p exp(2 pi i (lambda_k - lambda_j).p / N) is the
    data-frame Gram matrix sampled on the N x N pixel lattice."""
    d = np.asarray(delta, dtype=np.float64)
    den = np.sin(np.pi * d / N)
    small = np.abs(den) < 1e-12
    num = np.sin(np.pi * d)
    safe = np.where(small, 1.0, den)
    return np.where(small, 1.0, (num * num) / (N * N * safe * safe))


def weights_brute(lam, N, idx=None, chunk=2048):
    """alpha_k = argmin_a || T e_k a - e_k ||^2 = conj(T_kk) / sum_j |T_jk|^2 = 1 / S_k with
    S_k = sum_j F_N(lambda_jx - lambda_kx) F_N(lambda_jy - lambda_ky) (Eq. difopt, column-separable
    least squares over a diagonal D). Direct O(M K) evaluation for the rows in idx."""
    lam = np.asarray(lam, np.float64)
    if idx is None:
        idx = np.arange(lam.shape[0])
    idx = np.asarray(idx)
    S = np.empty(idx.shape[0], np.float64)
    for s in range(0, idx.shape[0], chunk):
        k = idx[s:s + chunk]
        dx = lam[None, :, 0] - lam[k, None, 0]
        dy = lam[None, :, 1] - lam[k, None, 1]
        S[s:s + chunk] = np.sum(fejer(dx, N) * fejer(dy, N), axis=1)
    return 1.0 / S, S


def gram_column(lam, N, k):
    """T_{:,k} = (1/N^2) sum_p exp(2 pi i (lambda_k - lambda_j).p / N) on the pixel lattice."""
    p = pixel_range(N).astype(np.float64)
    d = lam[k][None, :] - lam
    tx = np.exp(2j * np.pi * np.multiply.outer(d[:, 0], p) / N).sum(axis=1) / N
    ty = np.exp(2j * np.pi * np.multiply.outer(d[:, 1], p) / N).sum(axis=1) / N
    return tx * ty


def fejer_lag_weights(N):
    """c(d) = prod_i (N - |d_i|) / N^2 on lags d in {-N..N-1}^2 (c(-N) = 0), so that
    F_N(dx) F_N(dy) = sum_d c(d) exp(2 pi i (dx, dy).d / N)."""
    d = np.arange(-N, N)
    c1 = (N - np.abs(d)) / float(N * N)
    return np.multiply.outer(c1, c1)


def weights_nufft(lam, N, sigma=2.0, w_alpha=16, kind=ES):
    """The same S_k by the fast route: S_k = sum_d c(d) e^{-2 pi i lambda_k.d/N} H(d) with
    H(d) = sum_j e^{+2 pi i lambda_j.d/N}. H is the gridded adjoint of unit strengths at 2 lambda
    on the 2N x 2N lattice (W1); multiply by c (W2); S is the gridded forward transform at 2 lambda
    (W3); alpha = 1 / Re S (W4). Returns (alpha, S complex)."""
    lam2 = 2.0 * np.asarray(lam, np.float64)
    H = adjoint(lam2, np.ones(lam.shape[0]), 2 * N, sigma, w_alpha, kind)
    X = H * fejer_lag_weights(N)
    S = forward(lam2, X, 2 * N, sigma, w_alpha, kind)
    return 1.0 / S.real, S


# --------------------------------------------------------------------------------------------
# Error metrics
# --------------------------------------------------------------------------------------------

def rel_l2(a, ref):
    a = np.asarray(a, np.complex128)
    ref = np.asarray(ref, np.complex128)
    return float(np.linalg.norm((a - ref).ravel()) / np.linalg.norm(ref.ravel()))
