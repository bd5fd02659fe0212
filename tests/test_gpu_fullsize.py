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


# ---- whole images at full size, element by element against the FP64 gridding oracle ------------

def test_large_ping_whole_image(F, large):
    """The benchmark's ping and launch configuration (default plan: autotuned tile and kernel),
    seeded weights: every one of the 1,048,576 pixels against O.adjoint."""
    p, v = large
    alpha = np.random.default_rng(15).uniform(0.5, 1.5, p.M)
    with F.Plan(dev(p.lam), p.N, p.sigma, p.w) as pl:
        pl.set_weights(dev(alpha))
        img = pl.adjoint(dev(v)).cpu().numpy()
        pl.check()
    ref = O.adjoint(p.lam, alpha.astype(np.float32) * v.astype(np.complex128), p.N, p.sigma, p.w)
    assert O.rel_l2(img, ref) < TOL


@pytest.fixture(scope="module")
def precision(F):
    p = sasgen.precision_sweep()
    v = sasgen.values_for(p, device="cuda").astype(np.complex64)
    alpha = np.random.default_rng(16).uniform(0.5, 1.5, p.M)
    return p, v, alpha


def test_precision_sweep_whole_image_fp32(F, precision):
    p, v, alpha = precision
    with F.Plan(dev(p.lam), p.N, p.sigma, p.w) as pl:
        pl.set_weights(dev(alpha))
        img = pl.adjoint(dev(v)).cpu().numpy()
    ref = O.adjoint(p.lam, alpha.astype(np.float32) * v.astype(np.complex128), p.N, p.sigma, p.w)
    assert O.rel_l2(img, ref) < TOL


def test_precision_sweep_whole_image_bf16(F, precision):
    """BF16 storage at full size: parity (1e-5) against the oracle on the same bf16-rounded values
    and weights, and the precision bound (5e-3) against the unrounded FP64 inputs."""
    import torch
    p, v, alpha = precision
    vb = torch.view_as_real(torch.from_numpy(v)).to(torch.bfloat16)
    with F.Plan(dev(p.lam), p.N, p.sigma, p.w, precision=F.PREC_BF16) as pl:
        pl.set_weights(dev(alpha))
        img = pl.adjoint(vb.cuda()).cpu().numpy()
    vr = vb.to(torch.float64).numpy()
    vr = vr[:, 0] + 1j * vr[:, 1]
    ar = torch.from_numpy(alpha.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert O.rel_l2(img, O.adjoint(p.lam, ar * vr, p.N, p.sigma, p.w)) < TOL
    e = O.rel_l2(img, O.adjoint(p.lam, alpha * v.astype(np.complex128), p.N, p.sigma, p.w))
    assert e < 5e-3, e


def test_batch_pings_whole_images(F):
    """Four full-size pings of the uneven batch recipe with image sides 256, 512 and 1024 in one
    batched plan (persistent spreading launch, per-size-class transforms), each whole image
    against O.adjoint."""
    picks = []
    b = 0
    while len(picks) < 4:
        q = sasgen.batch_ping(b)
        if q.N not in [x.N for x in picks] or len(picks) == 3:
            picks.append(q)
        b += 1
    assert len({q.N for q in picks}) >= 3
    rng = np.random.default_rng(17)
    vals = [(rng.standard_normal(q.M) + 1j * rng.standard_normal(q.M)).astype(np.complex64)
            for q in picks]
    alphas = [rng.uniform(0.5, 1.5, q.M) for q in picks]
    with F.Batch([dev(q.lam) for q in picks], [q.N for q in picks], 2.0, 8) as bt:
        bt.set_weights([dev(a) for a in alphas])
        imgs = [i.cpu().numpy() for i in bt.adjoint([dev(x) for x in vals])]
    for q, x, a, img in zip(picks, vals, alphas, imgs):
        ref = O.adjoint(q.lam, a.astype(np.float32) * x.astype(np.complex128), q.N, 2.0, 8)
        assert O.rel_l2(img, ref) < TOL, q.N


def test_largest_grid_cufft_path_sampled(F):
    """The largest image of the test set, N = 4096 (G = 8192: beyond the shared-memory transforms,
    the pruned cuFFT path): 400,000 samples over a jittered polar wedge spanning the band, with
    random weights; 96 pixels (random, the centre row and column ends, the corners) against the
    oracle's pixel-by-pixel gridding, and the bright target's pixel."""
    N = 4096
    rng = np.random.default_rng(4096)
    kx, ky = sasgen.polar_raster(rng, 800, 500, 20.0, theta_jitter_deg=0.02)
    span = max(kx.max() - kx.min(), ky.max() - ky.min())
    lam = sasgen.baseband(kx, ky, 0.9 * 2 * np.pi * N / span)
    M = lam.shape[0]
    tgt = np.array([0.123, -0.231])                 # a point target (fraction of the FOV)
    v = np.exp(-2j * np.pi * lam @ tgt) + 0.1 * (rng.standard_normal(M) +
                                                  1j * rng.standard_normal(M))
    alpha = rng.uniform(0.5, 1.5, M)
    with F.Plan(dev(lam), N, 2.0, 8) as p:
        p.set_weights(dev(alpha))
        img = p.adjoint(dev(v.astype(np.complex64))).cpu().numpy()
    pix = np.concatenate([rng.integers(-N // 2, N // 2, (88, 2)),
                          [[-N // 2, 0], [N // 2 - 1, 0], [0, -N // 2], [0, N // 2 - 1],
                           [-N // 2, -N // 2], [N // 2 - 1, N // 2 - 1],
                           [int(round(tgt[0] * N)), int(round(tgt[1] * N))], [0, 0]]])
    c = alpha.astype(np.float32) * v.astype(np.complex64).astype(np.complex128)
    ref = O.adjoint_pixels(lam, c, N, 2.0, 8, pix)
    got = img[pix[:, 1] + N // 2, pix[:, 0] + N // 2]
    assert O.rel_l2(got, ref) < TOL
    peak = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    assert (peak[1] - N // 2, peak[0] - N // 2) == (int(round(tgt[0] * N)), int(round(tgt[1] * N)))
