"""The banded FTCG coefficient matrix C (ftcg_band, Sec. III-C Eq. ftcg / Eq. cr, reading (i):
banded least squares) against the FP64 oracle (oracle/ftcg_banded.py) through the C ABI.

Bars: the coefficients are FP64 on the device, from normal equations whose condition is the
square of the band columns' condition; on these rasters that leaves the coefficients within
1e-9 (max abs error over the max coefficient) of the oracle's QR-based least squares. The image
is the FP32 gridding of tau = C v: rel-L2 1e-5 against the oracle's FTCG image."""
import numpy as np
import pytest

import sasgen
from oracle import ftcg_banded as B
from oracle import ftcg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    import paper_1706_08575_gb300 as pkg
    return pkg


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def lattice(seed, n, N, spacing=1.2, jitter=0.25):
    rng = np.random.default_rng(seed)
    g = (np.arange(n) - (n - 1) / 2) * spacing
    X, Y = np.meshgrid(g, g)
    lam = np.stack([X.ravel(), Y.ravel()], 1) + rng.uniform(-jitter, jitter, (n * n, 2))
    v = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    return lam, v.astype(np.complex64)


def dense_c(band, r):
    """The device's band rows (row k: column k at rows k-r+1..k+r-1) as a dense M x M matrix."""
    M = band.shape[0]
    C = np.zeros((M, M), np.complex128)
    for k in range(M):
        for o in range(-(r - 1), r):
            j = k + o
            if 0 <= j < M:
                C[j, k] = band[k, o + r - 1]
    return C


def polar(seed, n_kr, n_th, N):
    """A small jittered polar raster in acquisition order (range fastest), spanning about 70%
    of N cycles."""
    rng = np.random.default_rng(seed)
    kx, ky = sasgen.polar_raster(rng, n_kr, n_th, 12.0, theta_jitter_deg=0.02)
    span = max(kx.max() - kx.min(), ky.max() - ky.min())
    lam = sasgen.baseband(kx, ky, 0.7 * 2 * np.pi * N / span)
    v = rng.standard_normal(lam.shape[0]) + 1j * rng.standard_normal(lam.shape[0])
    return lam, v.astype(np.complex64)


@pytest.mark.parametrize("case,r", [("lattice", 2), ("lattice", 5), ("polar", 3), ("polar", 8)])
def test_band_against_the_oracle(F, case, r):
    if case == "lattice":
        lam, v = lattice(1, 6, 8)
        N = 8
    else:
        lam, v = polar(2, 24, 20, 32)
        N = 32
    T = B.gram_matrix(lam, N)
    ref = B.banded_c(T, r)
    with F.Plan(dev(lam), N, 2.0, 8) as p:
        band = p.band(r).cpu().numpy()
        img = p.adjoint(dev(v)).cpu().numpy()
    C = dense_c(band, r)
    assert np.max(np.abs(C - ref)) < 1e-9 * np.max(np.abs(ref))
    ref_img = B.ftcg_image(lam, v.astype(np.complex128), N, 2.0, 8, ref)
    assert O.rel_l2(img, ref_img) < 1e-5


def test_band_one_is_the_diagonal_weights(F):
    lam, v = polar(3, 30, 24, 32)
    with F.Plan(dev(lam), 32, 2.0, 8) as p:
        band = p.band(1).cpu().numpy()[:, 0]
        img_band = p.adjoint(dev(v)).cpu().numpy()
        alpha = p.weights().cpu().numpy()
        img_w = p.adjoint(dev(v)).cpu().numpy()
    assert np.max(np.abs(band.imag)) < 1e-12 * np.max(np.abs(band))
    assert np.max(np.abs(band.real - alpha) / alpha) < 1e-9
    assert O.rel_l2(img_band, img_w) < 1e-5


def test_full_band_is_the_pseudo_inverse_and_the_frame_image(F):
    """12 samples with a band covering every index (r = 12): C = T^+ (Eq. dif3) and the FTCG
    image is N^2 times the minimum-norm least-squares image (Eq. insert)."""
    rng = np.random.default_rng(5)
    lam = rng.uniform(-3.5, 3.5, (12, 2))
    v = (rng.standard_normal(12) + 1j * rng.standard_normal(12)).astype(np.complex64)
    N = 8
    T = B.gram_matrix(lam, N)
    P = np.linalg.pinv(T)
    with F.Plan(dev(lam), N, 2.0, 8) as p:
        C = dense_c(p.band(12).cpu().numpy(), 12)
        img = p.adjoint(dev(v)).cpu().numpy()
    assert np.max(np.abs(C - P)) < 1e-9 * np.max(np.abs(P))
    ls = B.ls_image(lam, v.astype(np.complex128), N) * N ** 2
    assert O.rel_l2(img, ls) < 1e-5


def test_band_limits_and_weights_replace_the_band(F):
    lam, v = lattice(6, 6, 8)
    with F.Plan(dev(lam), 8, 2.0, 8) as p:
        for r in (0, 13):
            with pytest.raises(F.FtcgError) as ei:
                p.band(r)
            assert ei.value.status == 1
        p.band(3)
        p.set_weights(None)                        # back to plain gridding (alpha = 1)
        img = p.adjoint(dev(v)).cpu().numpy()
    ref = O.adjoint(lam, v.astype(np.complex128), 8, 2.0, 8)
    assert O.rel_l2(img, ref) < 1e-5
    big = np.random.default_rng(7).uniform(-30, 30, (8193, 2))
    with F.Plan(dev(big), 64, 2.0, 8) as p:
        with pytest.raises(F.FtcgError) as ei:
            p.band(2)
        assert ei.value.status == 4


def test_band_at_the_tiny_configuration(F):
    """The tiny configuration (4096 polar samples, N = 64) at r = ceil(log(2N + 1)) = 5, the band
    the paper suggests: coefficients against the oracle's banded least squares, and the image."""
    p = sasgen.tiny()
    v = sasgen.values_for(p).astype(np.complex64)
    r = int(np.ceil(np.log(2 * p.N + 1)))
    assert r == 5
    with F.Plan(dev(p.lam), p.N, p.sigma, p.w) as pl:
        band = pl.band(r).cpu().numpy()
        img = pl.adjoint(dev(v)).cpu().numpy()
    T = B.gram_matrix(p.lam, p.N)
    ref = B.banded_c(T, r)
    C = dense_c(band, r)
    assert np.max(np.abs(C - ref)) < 1e-9 * np.max(np.abs(ref))
    ref_img = B.ftcg_image(p.lam, v.astype(np.complex128), p.N, p.sigma, p.w, ref)
    assert O.rel_l2(img, ref_img) < 1e-5
