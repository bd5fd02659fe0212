"""Precision modes: BF16 storage of values and weights, FP32 arithmetic.

Two bars per case:
  * parity: the BF16-storage path against the FP64 oracle fed the same bf16-rounded values and
    weights: rel-L2 <= 1e-5 (the arithmetic is FP32 as in the FP32 mode);
  * precision: the same image against the oracle on the unrounded FP64 inputs. BF16 keeps 8
    significand bits (unit roundoff 2^-9 ~ 2e-3); independent rounding of re, im and alpha gives
    about 2^-9 relative per sample, averaged over many samples per pixel: the stated bound is
    5e-3 rel-L2.
"""
import numpy as np
import pytest

import sasgen
from oracle import ftcg_oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-5
BF16_BOUND = 5e-3


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    import paper_1706_08575_gb300 as pkg
    return pkg


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def bf16_pair(v):
    """complex -> (M, 2) bfloat16 tensor (round to nearest even, by torch on the host)."""
    import torch
    t = torch.view_as_real(torch.from_numpy(np.asarray(v, np.complex64)))
    return t.to(torch.bfloat16)


def bf16_round(x):
    import torch
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("M,N,w,spread", [(4000, 64, 8, 64), (3000, 48, 6, 120)])
def test_bf16_storage_parity_and_error(F, M, N, w, spread):
    lam, v = sasgen.random_case(70 + M, M, N, 2.0, w, spread)
    alpha = np.random.default_rng(71).uniform(0.3, 1.7, M)
    vb = bf16_pair(v)
    with F.Plan(dev(lam), N, 2.0, w, precision=F.PREC_BF16) as p:
        p.set_weights(dev(alpha))
        img = p.adjoint(vb.cuda()).cpu().numpy()
        p.check()
    v_r = vb.to(dtype=__import__("torch").float64).numpy()
    v_r = v_r[:, 0] + 1j * v_r[:, 1]
    a_r = bf16_round(alpha)
    ref_same = O.adjoint(lam, a_r * v_r, N, 2.0, w)
    assert O.rel_l2(img, ref_same) < TOL
    ref_exact = O.adjoint(lam, alpha * v, N, 2.0, w)
    e = O.rel_l2(img, ref_exact)
    assert e < BF16_BOUND, e


def test_bf16_plan_default_weights(F):
    """A BF16 plan without installed weights grids with alpha = 1."""
    lam, v = sasgen.random_case(75, 2000, 32, 2.0, 8, 32)
    vc = v.astype(np.complex64)
    with F.Plan(dev(lam), 32, 2.0, 8, precision=F.PREC_BF16) as p:
        img = p.adjoint(dev(vc)).cpu().numpy()
    assert O.rel_l2(img, O.adjoint(lam, vc.astype(np.complex128), 32, 2.0, 8)) < TOL


def test_mixed_storage_modes(F):
    """BF16 values with FP32 weights, and FP32 values with BF16 weights."""
    lam, v = sasgen.random_case(80, 3000, 64, 2.0, 8, 64)
    alpha = np.random.default_rng(81).uniform(0.3, 1.7, 3000)
    vb = bf16_pair(v)
    import torch
    v_r = vb.to(torch.float64).numpy()
    v_r = v_r[:, 0] + 1j * v_r[:, 1]
    a32 = alpha.astype(np.float32).astype(np.float64)
    with F.Plan(dev(lam), 64, 2.0, 8) as p:
        p.set_weights(dev(alpha))
        img = p.adjoint(vb.cuda()).cpu().numpy()
    assert O.rel_l2(img, O.adjoint(lam, a32 * v_r, 64, 2.0, 8)) < TOL
    with F.Plan(dev(lam), 64, 2.0, 8, precision=F.PREC_BF16) as p:
        p.set_weights(dev(alpha))
        img = p.adjoint(dev(v.astype(np.complex64))).cpu().numpy()
    vc = v.astype(np.complex64).astype(np.complex128)
    assert O.rel_l2(img, O.adjoint(lam, bf16_round(alpha) * vc, 64, 2.0, 8)) < TOL


def test_precision_sweep_bf16_sampled(F):
    """The 4.2M-sample, N = 2048 raster in BF16 storage: sampled pixels against the oracle on the
    same rounded inputs (parity) and on the FP64 inputs (precision), plus peak positions."""
    import torch
    p = sasgen.precision_sweep()
    v = sasgen.values_for(p, device="cuda")
    vb = bf16_pair(v)
    with F.Plan(dev(p.lam), p.N, p.sigma, p.w, precision=F.PREC_BF16) as pl:
        img = pl.adjoint(vb.cuda()).cpu().numpy()
        pl.check()
    rng = np.random.default_rng(9)
    pix = np.concatenate([rng.integers(-p.N // 2, p.N // 2, size=(16, 2)), p.bright_pixels])
    v_r = vb.to(torch.float64).numpy()
    v_r = v_r[:, 0] + 1j * v_r[:, 1]
    got = img[pix[:, 1] + p.N // 2, pix[:, 0] + p.N // 2]
    ref_same = O.adjoint_pixels(p.lam, v_r, p.N, p.sigma, p.w, pix)
    assert O.rel_l2(got, ref_same) < TOL
    ref_exact = O.adjoint_pixels(p.lam, v, p.N, p.sigma, p.w, pix)
    assert O.rel_l2(got, ref_exact) < BF16_BOUND
    mag = np.abs(img)
    for px, py in p.bright_pixels:
        iy, ix = py + p.N // 2, px + p.N // 2
        assert mag[iy, ix] == mag[max(iy - 1, 0):iy + 2, max(ix - 1, 0):ix + 2].max()
