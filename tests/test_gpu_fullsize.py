"""Parity at the full benchmark sizes, in the launch configuration the benchmark times (default
plan options): sampled pixels and sampled weights that the oracle computes one by one, plus
properties that hold at any size (adjointness, peaks at the bright targets)."""
import numpy as np
import pytest

import sasgen
from oracle import ftcg_oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    import paper_1706_08575_gb300 as pkg
    return pkg


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def sample_pixels(rng, N, bright, k=40):
    pix = rng.integers(-N // 2, N // 2, size=(k, 2))
    edge = np.array([[-N // 2, -N // 2], [N // 2 - 1, N // 2 - 1], [0, 0], [-N // 2, N // 2 - 1]])
    return np.concatenate([pix, edge, bright])


@pytest.fixture(scope="module")
def large(F):
    p = sasgen.large_ping()
    v = sasgen.values_for(p, device="cuda").astype(np.complex64)
    return p, v


def test_large_ping_sampled_pixels(F, large):
    p, v = large
    rng = np.random.default_rng(5)
    alpha = rng.uniform(0.5, 1.5, p.M)      # seeded weights (the weighted path, not the CUDA ones)
    with F.Plan(dev(p.lam), p.N, p.sigma, p.w) as pl:
        pl.set_weights(dev(alpha))
        img = pl.adjoint(dev(v)).cpu().numpy()
        pl.check()
    pix = sample_pixels(rng, p.N, p.bright_pixels)
    ref = O.adjoint_pixels(p.lam, alpha.astype(np.float32) * v.astype(np.complex128), p.N,
                           p.sigma, p.w, pix)
    got = img[pix[:, 1] + p.N // 2, pix[:, 0] + p.N // 2]
    assert O.rel_l2(got, ref) < TOL


def test_large_ping_weights_sampled(F, large):
    p, v = large
    with F.Plan(dev(p.lam), p.N, p.sigma, p.w) as pl:
        a = pl.weights().cpu().numpy()
        img = pl.adjoint(dev(v)).cpu().numpy()
        pl.check()
    rng = np.random.default_rng(6)
    ks = rng.choice(p.M, 24, replace=False)
    ab, _ = O.weights_brute(p.lam, p.N, ks, chunk=1)
    assert np.max(np.abs(a[ks] - ab) / ab) < 1e-9
    # every bright target is a local maximum of |I| within its 3 x 3 neighbourhood
    mag = np.abs(img)
    for px, py in p.bright_pixels:
        iy, ix = py + p.N // 2, px + p.N // 2
        win = mag[max(iy - 1, 0):iy + 2, max(ix - 1, 0):ix + 2]
        assert mag[iy, ix] == win.max()


def test_large_ping_adjointness(F, large):
    p, v = large
    rng = np.random.default_rng(7)
    img = (rng.standard_normal((p.N, p.N)) + 1j * rng.standard_normal((p.N, p.N))).astype(np.complex64)
    with F.Plan(dev(p.lam), p.N, p.sigma, p.w) as pl:
        f = pl.forward(dev(img)).cpu().numpy().astype(np.complex128)
        a = pl.adjoint(dev(v)).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(img.astype(np.complex128), a)
    rhs = np.vdot(f, v.astype(np.complex128))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_precision_sweep_fp32_sampled(F):
    p = sasgen.precision_sweep()
    v = sasgen.values_for(p, device="cuda").astype(np.complex64)
    with F.Plan(dev(p.lam), p.N, p.sigma, p.w) as pl:
        img = pl.adjoint(dev(v)).cpu().numpy()
        pl.check()
    rng = np.random.default_rng(8)
    pix = sample_pixels(rng, p.N, p.bright_pixels, k=24)
    ref = O.adjoint_pixels(p.lam, v.astype(np.complex128), p.N, p.sigma, p.w, pix)
    got = img[pix[:, 1] + p.N // 2, pix[:, 0] + p.N // 2]
    assert O.rel_l2(got, ref) < TOL
