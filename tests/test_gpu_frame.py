"""The frame approximation on the device (ftcg_cgls, Sec. III-B Eq. afr / afrm, Eq. twodframe)
against the FP64 oracle (oracle/ftcg_frame.py) through the C ABI.

Bars, from the arithmetic: the device operators are the FP32 gridding kernels, within about 1e-6
(rel-L2) of the FP64 gridded operators at sigma = 2, w = 8. CGLS is a smooth function of the
operator outputs for a well-conditioned problem, so k iterations keep the iterate within about
k times that per operator application, times the growth of the recursion: iterates up to k = 10
are held to 1e-4 of the FP64 oracle's iterates with the same (gridded) operators, and the
converged image to 1e-4 of the dense minimum-norm least-squares image (cases whose kernel error
is ~1e-7 and whose condition keeps the FP32 recursion stable).
"""
import numpy as np
import pytest

import sasgen
from oracle import ftcg_banded as B
from oracle import ftcg_frame as Fr
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


def lattice(seed, n=6, spacing=1.2, jitter=0.25):
    rng = np.random.default_rng(seed)
    g = (np.arange(n) - (n - 1) / 2) * spacing
    X, Y = np.meshgrid(g, g)
    lam = np.stack([X.ravel(), Y.ravel()], 1) + rng.uniform(-jitter, jitter, (n * n, 2))
    v = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    return lam, v.astype(np.complex64)


@pytest.mark.parametrize("weighted", [False, True], ids=["plain", "ftcg-weights"])
def test_cgls_reaches_the_least_squares_image(F, weighted):
    """36 jittered samples, N = 8 (64 pixels): CGLS converges to the minimum-norm least-squares
    image of the dense solver, with and without the FTCG row weights."""
    lam, v = lattice(1)
    N = 8
    with F.Plan(dev(lam), N, 2.0, 8) as p:
        w = p.weights() if weighted else None
        x, hist, done = p.cgls(dev(v), weights=w, iters=150)
        x = x.cpu().numpy()
    ref = B.ls_image(lam, v.astype(np.complex128), N)
    assert O.rel_l2(x, ref) < 1e-4
    assert hist[-1] < 1e-3 * hist[0]


@pytest.mark.parametrize("k", [1, 3, 10])
def test_cgls_iterates_match_the_oracle(F, k):
    """A polar ping of the batch recipe (N = 256) with its FTCG weights: the device's k-th
    iterate against the FP64 oracle's k-th iterate with the gridded operators (same weights)."""
    q = sasgen.batch_ping(2)
    rng = np.random.default_rng(4)
    v = (rng.standard_normal(q.M) + 1j * rng.standard_normal(q.M)).astype(np.complex64)
    with F.Plan(dev(q.lam), q.N, 2.0, 8) as p:
        a = p.weights()
        x, hist, _ = p.cgls(dev(v), weights=a, iters=k)
        x = x.cpu().numpy()
        a = a.cpu().numpy()
    ref, rh = Fr.cgls(q.lam, v.astype(np.complex128), q.N, weights=a.astype(np.float32),
                      iters=k, gridded=True)
    assert O.rel_l2(x, ref) < 1e-4
    assert np.max(np.abs(hist - np.asarray(rh)) / np.asarray(rh)[0]) < 1e-4


def test_first_weighted_iterate_is_the_ftcg_image(F):
    """Started from zero, the first iterate is a positive multiple of E^H W v: the FTCG image of
    ftcg_adjoint with the same weights installed. The plan's weights are restored afterwards."""
    lam, v = sasgen.random_case(90, 3000, 48, 2.0, 8, 48)
    v = v.astype(np.complex64)
    with F.Plan(dev(lam), 48, 2.0, 8) as p:
        a = p.weights()
        img = p.adjoint(dev(v)).cpu().numpy().astype(np.complex128)
        x1, _, _ = p.cgls(dev(v), weights=a, iters=1)
        x1 = x1.cpu().numpy().astype(np.complex128)
        again = p.adjoint(dev(v)).cpu().numpy()
    scale = np.vdot(img, x1) / np.vdot(img, img)
    assert O.rel_l2(x1, scale * img) < 1e-5
    assert scale.real > 0 and abs(scale.imag) < 1e-5 * abs(scale)
    assert O.rel_l2(again, img) < 1e-6           # the same weights (atomics reorder sums)


def test_cgls_tolerance_and_history(F):
    """The residual history starts at ||E^H W v|| and a tolerance freezes the iterate: the
    reported count is the first iteration at or below tol times the initial residual."""
    lam, v = lattice(3)
    with F.Plan(dev(lam), 8, 2.0, 8) as p:
        x, hist, done = p.cgls(dev(v), iters=40, tol=1e-2)
        img = p.adjoint(dev(v)).cpu().numpy()
    assert abs(hist[0] - np.linalg.norm(img)) / np.linalg.norm(img) < 1e-5
    assert 0 < done < 40
    assert hist[done] <= 1e-2 * hist[0] < hist[done - 1]
    assert np.all(hist[done:] == hist[done])


def test_cgls_refuses_bf16_plans(F):
    lam, v = lattice(4)
    with F.Plan(dev(lam), 8, 2.0, 8, precision=F.PREC_BF16) as p:
        with pytest.raises(F.FtcgError) as ei:
            p.cgls(dev(v), iters=3)
    assert ei.value.status == 4
