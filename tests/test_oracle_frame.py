"""Pins of the iterative frame-approximation oracle (oracle/ftcg_frame.py): CGLS reaches the
minimum-norm least-squares image computed by a dense solver, with and without the FTCG row
weights; its first weighted iterate is the FTCG image up to a scale; with the gridded operators
it stays within the kernel's accuracy."""
import numpy as np

from oracle import ftcg_banded as B
from oracle import ftcg_frame as Fr
from oracle import ftcg_oracle as O

N = 8


def case(seed=0, M=36):
    rng = np.random.default_rng(seed)
    g = (np.arange(6) - 2.5) * 1.2
    X, Y = np.meshgrid(g, g)
    lam = np.stack([X.ravel(), Y.ravel()], 1) + rng.uniform(-0.25, 0.25, (36, 2))
    v = rng.standard_normal(36) + 1j * rng.standard_normal(36)
    return lam[:M], v[:M]


def test_cgls_reaches_the_least_squares_image():
    lam, v = case()
    ref = B.ls_image(lam, v, N)
    x, hist = Fr.cgls(lam, v, N, iters=200)
    assert O.rel_l2(x, ref) < 1e-9
    assert hist[-1] < 1e-9 * hist[0]


def test_weighted_cgls_reaches_the_same_image():
    """36 samples and 64 pixels: E x = v is solvable, so the FTCG row weights change the path but
    not the minimum-norm limit."""
    lam, v = case(1)
    alpha, _ = O.weights_brute(lam, N)
    x, _ = Fr.cgls(lam, v, N, weights=alpha, iters=200)
    assert O.rel_l2(x, B.ls_image(lam, v, N)) < 1e-9


def test_first_weighted_iterate_is_the_ftcg_image():
    lam, v = case(2)
    alpha, _ = O.weights_brute(lam, N)
    x1, _ = Fr.cgls(lam, v, N, weights=alpha, iters=1)
    ftcg = O.direct_adjoint(lam, alpha * v, N)
    scale = np.vdot(ftcg, x1) / np.vdot(ftcg, ftcg)
    assert O.rel_l2(x1, scale * ftcg) < 1e-12
    assert scale.real > 0 and abs(scale.imag) < 1e-12 * abs(scale)


def test_gridded_operators_within_kernel_accuracy():
    lam, v = case(3)
    x, _ = Fr.cgls(lam, v, N, iters=200, gridded=True)
    assert O.rel_l2(x, B.ls_image(lam, v, N)) < 1e-5
