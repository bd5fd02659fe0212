"""FP64 CPU oracle for the banded FTCG coefficient matrix C (r > 1), Sec. III-C.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this module: only the tests do.
It shares no code with the CUDA library; plain numpy in float64 / complex128.

FTCG replaces the diagonal quadrature weights D of convolutional gridding by a coefficient matrix
C: the image is the gridded adjoint of tau = C f^ (Eq. ftcg). The paper gives C two ways that do
not agree: next to Eq. ftcg C itself is (2r - 1)-banded, while Eq. cr sets C = (Psi Omega (.) B_r)^+
with B_r a band mask, and the pseudo-inverse of a banded matrix is dense in general. With
T = Psi Omega read as the M x M data-frame Gram matrix on the N x N pixel lattice (as for the
diagonal weights, reading R5) and the band taken over the acquisition order of the samples
(|j - k| <= r - 1, 2r - 1 diagonals), this module implements both readings:

  (i)  banded least squares: C minimises || T C - I ||_F over matrices with C_jk = 0 outside the
       band. This is the minimisation of Eq. difopt with its diagonal constraint widened to the
       band; r = 1 gives the diagonal FTCG weights, a full band gives T^+ (Eq. dif3), whose
       image is the frame approximation (Eq. insert).
  (ii) literal: C = (T (.) B_r)^+ as printed in Eq. cr (at r = 1 it is the identity, since
       T_kk = 1).
"""
from __future__ import annotations

import numpy as np

from . import ftcg_oracle as O


def gram_matrix(lam, N):
    """T_jk = N^-2 sum_p exp(2 pi i (lambda_k - lambda_j).p / N) for all j, k, p over the pixel
    lattice {-N/2..N/2-1}^2 (the matrix whose columns the diagonal weights use). The lattice sum
    factorises over the axes, T = Tx (.) Ty."""
    lam = np.asarray(lam, np.float64)
    p = O.pixel_range(N).astype(np.float64)
    ex = np.exp(2j * np.pi * np.multiply.outer(lam[:, 0], p) / N)
    ey = np.exp(2j * np.pi * np.multiply.outer(lam[:, 1], p) / N)
    return (ex.conj() @ ex.T) * (ey.conj() @ ey.T) / float(N * N)


def band_rows(M, k, r):
    """Rows of column k inside the band: {j : |j - k| <= r - 1}, clipped to 0..M-1."""
    return np.arange(max(0, k - r + 1), min(M, k + r))


def band_mask(M, r):
    j, k = np.indices((M, M))
    return np.abs(j - k) <= r - 1


def banded_c(T, r):
    """Reading (i). || T C - I ||_F separates over the columns of C, so column k is the
    minimum-norm least-squares solution of T[:, S_k] c = e_k over its band rows S_k.
    Returns C as a dense M x M complex128 array (zero outside the band)."""
    T = np.asarray(T, np.complex128)
    M = T.shape[0]
    C = np.zeros((M, M), np.complex128)
    for k in range(M):
        S = band_rows(M, k, r)
        e = np.zeros(M, np.complex128)
        e[k] = 1.0
        c, *_ = np.linalg.lstsq(T[:, S], e, rcond=None)
        C[S, k] = c
    return C


def banded_c_literal(T, r):
    """Reading (ii): C = (T (.) B_r)^+ (Eq. cr as printed)."""
    T = np.asarray(T, np.complex128)
    return np.linalg.pinv(T * band_mask(T.shape[0], r))


def residual(T, C):
    """|| T C - I ||_F, the quantity Eq. difopt minimises."""
    return float(np.linalg.norm(T @ C - np.eye(T.shape[0])))


def ftcg_image(lam, v, N, sigma, w, C):
    """The FTCG image of values v with coefficient matrix C: the gridding algorithm (O2) applied
    to tau = C v (Eq. ftcg, tau = Omega C f^)."""
    return O.adjoint(lam, np.asarray(C) @ np.asarray(v, np.complex128), N, sigma, w)


def ls_image(lam, v, N):
    """The frame approximation in its least-squares form: the minimum-norm x minimising
    || E x - v ||_2 with E_jp = exp(-2 pi i lambda_j.p / N) (the forward model of reading R1).
    Returned N x N indexed [p_y + N/2, p_x + N/2]."""
    lam = np.asarray(lam, np.float64)
    p = O.pixel_range(N).astype(np.float64)
    PX, PY = np.meshgrid(p, p)
    E = np.exp(-2j * np.pi * (np.multiply.outer(lam[:, 0], PX.ravel()) +
                              np.multiply.outer(lam[:, 1], PY.ravel())) / N)
    x, *_ = np.linalg.lstsq(E, np.asarray(v, np.complex128), rcond=None)
    return x.reshape(N, N)


def overlap_sum(d, delta, N):
    """K(d, delta) = sum of exp(2 pi i delta q / N) over the q of {-N/2..N/2-1} for which q + d
    is also in that set (one axis): the weight a lag d carries in a product of two Gram entries
    whose samples are delta apart. K(d, 0) = N - |d|, the Fejer lag weight of the diagonal route."""
    p = O.pixel_range(N)
    q = p[(p + d >= p[0]) & (p + d <= p[-1])]
    return np.exp(2j * np.pi * delta * q / N).sum()


def gram2_entry_lag(lam, N, a, b):
    """(T^2)_ab by the lag route: with H(d) = sum_j exp(2 pi i lambda_j.d / N) on the lags
    d in {-N+1..N-1}^2 (the gridded adjoint of unit strengths that the diagonal weights use),
    (T^2)_ab = N^-4 sum_d H(d) exp(-2 pi i lambda_a.d / N) K(d_x, delta_x) K(d_y, delta_y),
    delta = lambda_b - lambda_a. At a = b this is S_a of the diagonal weights. Direct O(M N^2)
    evaluation of the lag sum, for checking a device route."""
    lam = np.asarray(lam, np.float64)
    d = np.arange(-N + 1, N).astype(np.float64)
    ex = np.exp(2j * np.pi * np.multiply.outer(lam[:, 0], d) / N)
    ey = np.exp(2j * np.pi * np.multiply.outer(lam[:, 1], d) / N)
    H = ex.T @ ey                                   # H[d_x, d_y]
    delta = lam[b] - lam[a]
    kx = np.array([overlap_sum(t, delta[0], N) for t in range(-N + 1, N)])
    ky = np.array([overlap_sum(t, delta[1], N) for t in range(-N + 1, N)])
    ph = np.multiply.outer(np.exp(-2j * np.pi * lam[a, 0] * d / N),
                           np.exp(-2j * np.pi * lam[a, 1] * d / N))
    return complex(np.sum(H * ph * np.multiply.outer(kx, ky)) / float(N) ** 4)
