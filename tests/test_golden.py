"""The stored small case (tests/golden/ftcg_polar_n32.txt, written by make_golden.py from the
FP64 oracle): the oracle still reproduces it, its values satisfy what the method fixes
independently of the oracle, and the CUDA path matches it."""
import os
import sys

import numpy as np
import pytest

from oracle import ftcg_oracle as O

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402


@pytest.fixture(scope="module")
def case():
    return make_golden.read()


def test_oracle_reproduces_stored_case(case):
    meta, lam, v, alpha, pix, o2, o1 = case
    N, sigma, w = int(meta["N"]), meta["sigma"], int(meta["w"])
    a, _ = O.weights_brute(lam, N)
    assert np.max(np.abs(a - alpha) / alpha) < 1e-12
    iy, ix = pix[:, 1] + N // 2, pix[:, 0] + N // 2
    assert O.rel_l2(O.adjoint(lam, alpha * v, N, sigma, w)[iy, ix], o2) < 1e-12
    assert O.rel_l2(O.direct_adjoint(lam, alpha * v, N)[iy, ix], o1) < 1e-12


def test_stored_weights_from_the_pixel_lattice(case):
    """alpha_k = 1 / sum_j |T_jk|^2 with T_jk = N^-2 sum_p exp(2 pi i (lambda_k - lambda_j).p / N)
    summed over the N x N pixel lattice (Eq. difopt with a diagonal D), not through the Fejer
    closed form the oracle uses."""
    meta, lam, v, alpha, pix, o2, o1 = case
    N = int(meta["N"])
    p = np.arange(-N // 2, N // 2)
    PX, PY = np.meshgrid(p, p)
    E = np.exp(2j * np.pi * (np.outer(lam[:, 0], PX.ravel()) + np.outer(lam[:, 1], PY.ravel())) / N)
    T = (E.conj() @ E.T) / N ** 2            # T[j, k]
    S = np.sum(np.abs(T) ** 2, axis=0)
    assert np.max(np.abs(1.0 / S - alpha) / alpha) < 1e-12


def test_stored_gridding_within_kernel_bound_and_peaks(case):
    """The gridded image agrees with the direct sum within the ES kernel's accuracy at sigma = 2,
    w = 8, and each point scatterer peaks at its own pixel (stored first, each with its eight
    neighbours)."""
    meta, lam, v, alpha, pix, o2, o1 = case
    assert O.rel_l2(o2, o1) < 2e-7
    for s in range(2):
        block = np.abs(o1[9 * s:9 * s + 9])
        assert np.argmax(block) == 4
    assert tuple(pix[4]) == (5, -7) and tuple(pix[13]) == (-9, 4)


@pytest.mark.gpu
def test_cuda_path_matches_stored_case(case):
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_1706_08575_gb300 as F
    meta, lam, v, alpha, pix, o2, o1 = case
    N, sigma, w = int(meta["N"]), meta["sigma"], int(meta["w"])
    with F.Plan(torch.from_numpy(lam).cuda(), N, sigma, w) as pl:
        a = pl.weights().cpu().numpy()
        img = pl.adjoint(torch.from_numpy(v.astype(np.complex64)).cuda()).cpu().numpy()
    assert np.max(np.abs(a - alpha) / alpha) < 1e-9
    iy, ix = pix[:, 1] + N // 2, pix[:, 0] + N // 2
    assert O.rel_l2(img[iy, ix], o2) < 1e-5
