"""The gridding window families (Sec. III-A leaves the window open; reading R3): exponential of
semicircle (the default), Kaiser-Bessel and truncated Gaussian, each through both spreading
kernels, the forward operator and a batch, against the FP64 oracle with the same window
(oracle/ftcg_oracle.py `phi`, `kernel_beta`, `phi_hat`) through the C ABI.

Bars: grids and images within the FP32 bound (rel-L2 1e-5, or 5e-8 A where the window division
amplifies FP32 grid rounding by A, computed from the oracle's factors for that window); the
forward operator within 1e-5; the shape parameter reported by the plan equals the oracle's."""
import numpy as np
import pytest

import sasgen
from oracle import ftcg_oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-5
KINDS = [(O.ES, "es"), (O.KB, "kb"), (O.GAUSS, "gauss")]


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    import paper_1706_08575_gb300 as pkg
    return pkg


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def c64(v):
    return np.asarray(v).astype(np.complex64)


def image_tol(N, sigma, w, kind):
    r = O.deapod_factors(N, sigma, w, kind)
    A = float(np.sqrt(np.mean(np.multiply.outer(r, r) ** 2)) / r[N // 2] ** 2)
    return max(TOL, 5e-8 * A)


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["window", "tensor", "block"])
@pytest.mark.parametrize("kind,name", KINDS, ids=[k[1] for k in KINDS])
@pytest.mark.parametrize("N,sigma,w,T", [(64, 2.0, 8, 32), (50, 2.0, 7, 64), (48, 1.5, 8, 32)],
                         ids=["w8", "ragged-w7-T64", "sigma1.5"])
def test_window_family_vs_oracle(F, kernel, kind, name, N, sigma, w, T):
    lam, v = sasgen.random_case(80 + kind, 5000, N, sigma, w, 1.4 * N)
    alpha = np.random.default_rng(81).uniform(0.2, 2.0, lam.shape[0])
    cw = alpha.astype(np.float32) * c64(v).astype(np.complex128)
    try:
        p = F.Plan(dev(lam), N, sigma, w, tile=T, layout=F.LAYOUT_HALO, spread_kernel=kernel,
                   window=kind)
    except F.FtcgError as e:
        # the tensor-core kernel takes a window only where its tap polynomials fit within 1e-6
        assert kernel in (2, 3) and e.status == 4
        return
    with p:
        assert abs(p.info.beta - O.kernel_beta(w, sigma, kind)) < 1e-12 * p.info.beta
        p.set_weights(dev(alpha))
        img = p.adjoint(dev(c64(v))).cpu().numpy()
        grid = p.spread(dev(c64(v))).cpu().numpy()
    assert O.rel_l2(grid, O.spread(lam, cw, N, sigma, w, kind)) < TOL
    assert O.rel_l2(img, O.adjoint(lam, cw, N, sigma, w, kind)) < image_tol(N, sigma, w, kind)


@pytest.mark.parametrize("kind,name", KINDS[1:], ids=[k[1] for k in KINDS[1:]])
def test_window_family_forward_and_batch(F, kind, name):
    lam, c = sasgen.random_case(90 + kind, 3000, 48, spread=70)
    rng = np.random.default_rng(91)
    img = (rng.standard_normal((48, 48)) + 1j * rng.standard_normal((48, 48))).astype(np.complex64)
    with F.Plan(dev(lam), 48, 2.0, 8, window=kind) as p:
        f = p.forward(dev(img)).cpu().numpy()
    assert O.rel_l2(f, O.forward(lam, img.astype(np.complex128), 48, 2.0, 8, kind)) < TOL
    cases = [sasgen.random_case(95 + i, 2000 + 500 * i, N, spread=1.2 * N)
             for i, N in enumerate([32, 64, 256])]
    with F.Batch([dev(q[0]) for q in cases], [32, 64, 256], 2.0, 8, window=kind) as b:
        imgs = [x.cpu().numpy() for x in b.adjoint([dev(c64(q[1])) for q in cases])]
    for (lam_i, v_i), N, got in zip(cases, [32, 64, 256], imgs):
        ref = O.adjoint(lam_i, c64(v_i).astype(np.complex128), N, 2.0, 8, kind)
        assert O.rel_l2(got, ref) < image_tol(N, 2.0, 8, kind)


def test_window_family_refusals(F):
    lam, _ = sasgen.random_case(99, 100, 32)
    with pytest.raises(F.FtcgError) as ei:          # no fourth family
        F.Plan(dev(lam), 32, 2.0, 8, window=3)
    assert ei.value.status == 1
