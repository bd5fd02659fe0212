"""Pins of the banded FTCG oracle (oracle/ftcg_banded.py) against what the method fixes without
it: the pixel-lattice Gram sum, the diagonal weights at r = 1 (Eq. difopt), the pseudo-inverse and
the frame approximation at a full band (Eq. dif3, Eq. insert), the monotone residual of nested
least-squares problems; and planted mistakes that a pin catches."""
import numpy as np
import pytest

from oracle import ftcg_banded as B
from oracle import ftcg_oracle as O

N = 8


def case(seed=0):
    """A jittered 6 x 6 lattice of spacing 1.2 cycles (jitter +-0.25) inside one period of N = 8,
    in acquisition order (x fastest), and random complex values."""
    rng = np.random.default_rng(seed)
    g = (np.arange(6) - 2.5) * 1.2
    X, Y = np.meshgrid(g, g)
    lam = np.stack([X.ravel(), Y.ravel()], 1) + rng.uniform(-0.25, 0.25, (36, 2))
    v = rng.standard_normal(36) + 1j * rng.standard_normal(36)
    return lam, v


def pin_gram(lam):
    T = B.gram_matrix(lam, N)
    p = O.pixel_range(N)
    PX, PY = np.meshgrid(p, p)
    E = np.exp(-2j * np.pi * (np.outer(lam[:, 0], PX.ravel()) + np.outer(lam[:, 1], PY.ravel())) / N)
    assert np.max(np.abs(T - E @ E.conj().T / N ** 2)) < 1e-12
    for k in (0, 17, 35):
        assert np.max(np.abs(T[:, k] - O.gram_column(lam, N, k))) < 1e-12


def pin_r1(lam):
    T = B.gram_matrix(lam, N)
    C = B.banded_c(T, 1)
    alpha, _ = O.weights_brute(lam, N)
    assert np.max(np.abs(C - np.diag(np.diag(C)))) == 0.0
    assert np.max(np.abs(np.diag(C) - alpha) / alpha) < 1e-12
    assert np.max(np.abs(B.banded_c_literal(T, 1) - np.eye(lam.shape[0]))) < 1e-12


def pin_full_band(lam, v):
    T = B.gram_matrix(lam, N)
    M = lam.shape[0]
    C = B.banded_c(T, M)
    P = np.linalg.pinv(T)
    assert np.linalg.norm(C - P) / np.linalg.norm(P) < 1e-9
    assert np.linalg.norm(B.banded_c_literal(T, M) - P) / np.linalg.norm(P) < 1e-9
    ls = B.ls_image(lam, v, N) * N ** 2
    assert O.rel_l2(O.direct_adjoint(lam, C @ v, N), ls) < 1e-9


def test_gram_matrix_against_lattice_sum():
    pin_gram(case()[0])


def test_r1_gives_the_diagonal_weights_and_the_literal_identity():
    pin_r1(case()[0])


def test_full_band_gives_pinv_and_the_frame_image():
    lam, v = case()
    pin_full_band(lam, v)


def test_gridded_full_band_image_within_kernel_bound():
    lam, v = case(1)
    T = B.gram_matrix(lam, N)
    C = B.banded_c(T, lam.shape[0])
    img = B.ftcg_image(lam, v, N, 2.0, 8, C)
    assert O.rel_l2(img, B.ls_image(lam, v, N) * N ** 2) < 2e-7


def test_residual_does_not_grow_with_the_band():
    """Column k's band rows for r are a subset of those for r + 1, so each column's least-squares
    residual, and the Frobenius residual, cannot grow; on a jittered raster the band helps."""
    lam, _ = case(2)
    T = B.gram_matrix(lam, N)
    res = [B.residual(T, B.banded_c(T, r)) for r in range(1, 7)]
    assert all(b <= a + 1e-12 for a, b in zip(res, res[1:]))
    assert res[2] < 0.9 * res[0]
    for r in (2, 4):
        C = B.banded_c(T, r)
        assert np.max(np.abs(C[~B.band_mask(36, r)])) == 0.0


def test_literal_reading_is_dense():
    """Eq. cr's C = (T (.) B_r)^+ inverts the banded matrix, so C itself is not banded (the
    disagreement with the text next to Eq. ftcg that reading (i) resolves)."""
    lam, _ = case(3)
    T = B.gram_matrix(lam, N)
    C = B.banded_c_literal(T, 2)
    Tb = T * B.band_mask(36, 2)
    assert np.max(np.abs(Tb @ C - np.eye(36))) < 1e-9
    assert np.max(np.abs(C[~B.band_mask(36, 4)])) > 1e-3


def _band_off_by_one(M, k, r):
    return np.arange(max(0, k - r), min(M, k + r + 1))


def _gram_transposed(lam, N_):
    return _ORIG_GRAM(lam, N_).T


_ORIG_GRAM = B.gram_matrix


@pytest.mark.parametrize("name,mutant", [("band_rows", _band_off_by_one),
                                         ("gram_matrix", _gram_transposed)])
def test_planted_mistakes_fail_a_pin(monkeypatch, name, mutant):
    lam, v = case()
    monkeypatch.setattr(B, name, mutant)
    failed = 0
    for pin in (lambda: pin_gram(lam), lambda: pin_r1(lam), lambda: pin_full_band(lam, v)):
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed > 0


def test_gram_squared_by_the_lag_route():
    """The entries of the banded normal equations, (T^2)_ab, by the lag route against the matrix
    product T T; on the diagonal they are the weight sums S_k = 1 / alpha_k."""
    lam, _ = case(4)
    T = B.gram_matrix(lam, N)
    T2 = T @ T
    for a, b in ((10, 10), (10, 11), (10, 16), (3, 0), (35, 29)):
        assert abs(B.gram2_entry_lag(lam, N, a, b) - T2[a, b]) < 1e-12 * max(1.0, abs(T2[a, a]))
    alpha, _ = O.weights_brute(lam, N)
    assert abs(B.gram2_entry_lag(lam, N, 7, 7).real * alpha[7] - 1.0) < 1e-12
    assert B.overlap_sum(3, 0.0, N) == N - 3
