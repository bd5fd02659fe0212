"""The spreading kernels against the FP64 oracle, element by element, through the C ABI.

The register-window kernel (FTCG_SPREAD_WINDOW), the tensor-core kernel on column bins
(FTCG_SPREAD_TENSOR: chunks of 8 samples of one column bin x a 16-row window per split-TF32
mma.sync.m16n8k8) and the tensor-core kernel on 8 x 8-cell blocks (FTCG_SPREAD_BLOCK: chunks of
8 samples of one block x a 16 x 16 window, two column halves) must give the same grid and image
within the FP32 bar (rel-L2 <= 1e-5 against the oracle on the same inputs). The cases stress what
the chunked plans add: ragged edge tiles, every sample in a handful of cells (many chunks per
column bin or block), first-tap rows spread so that column windows move down by 8 rows and
restart, wrap-around of the periodic grid, w from 6 to 8, both tile sides, BF16 storage, and the
degenerate plans (no sample, one sample).
"""
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


def c64(v):
    return np.asarray(v).astype(np.complex64)


def run(F, lam, v, N, sigma, w, alpha, T, kernel, **kw):
    with F.Plan(dev(lam), N, sigma, w, tile=T, layout=F.LAYOUT_HALO, spread_kernel=kernel,
                **kw) as p:
        if alpha is not None:
            p.set_weights(dev(alpha))
        img = p.adjoint(dev(c64(v)))
        grid = p.spread(dev(c64(v)))
        p.check()
        return img.cpu().numpy(), grid.cpu().numpy()


def clustered(seed, M, N, sigma, w, ncells):
    """M samples inside `ncells` random fine-grid cells (heavy collisions)."""
    rng = np.random.default_rng(seed)
    G = int(round(sigma * N))
    cells = rng.integers(0, G, size=(ncells, 2))
    pick = cells[rng.integers(0, ncells, M)]
    u = pick + rng.random((M, 2))
    lam = u / sigma - G / (2 * sigma)
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    return lam, v


def column_of_rows(seed, M, N, sigma, w):
    """Samples on a few grid columns, rows spread with gaps of 0..20 cells (window shifts by 8
    and window restarts within one column bin)."""
    rng = np.random.default_rng(seed)
    G = int(round(sigma * N))
    cols = rng.integers(0, G, size=4)
    x = cols[rng.integers(0, 4, M)] + rng.random(M)
    y = np.cumsum(rng.choice([0, 0, 0, 1, 2, 5, 9, 13, 20], size=M) + rng.random(M) * 0.3) % G
    lam = np.stack([x, y], 1) / sigma - G / (2 * sigma)
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    return lam, v


CASES = [
    # name, builder, N, sigma, w, T
    ("random-w8-T32", lambda: sasgen.random_case(21, 6000, 64, 2.0, 8, 96), 64, 2.0, 8, 32),
    ("random-w8-T64", lambda: sasgen.random_case(22, 6000, 64, 2.0, 8, 64), 64, 2.0, 8, 64),
    ("ragged-w8", lambda: sasgen.random_case(23, 5000, 50, 2.0, 8, 150), 50, 2.0, 8, 32),
    ("ragged-w7-T64", lambda: sasgen.random_case(24, 4000, 40, 2.0, 7, 80), 40, 2.0, 7, 64),
    ("w6", lambda: sasgen.random_case(25, 4096, 64, 2.0, 6, 150), 64, 2.0, 6, 32),
    ("sigma1.5-w8", lambda: sasgen.random_case(26, 3000, 48, 1.5, 8, 60), 48, 1.5, 8, 32),
    ("sigma1.25-w8", lambda: sasgen.random_case(27, 3000, 64, 1.25, 8, 64), 64, 1.25, 8, 32),
    ("collisions", lambda: clustered(28, 5000, 64, 2.0, 8, 7), 64, 2.0, 8, 32),
    ("collisions-T64", lambda: clustered(29, 4000, 48, 2.0, 8, 3), 48, 2.0, 8, 64),
    ("row-gaps", lambda: column_of_rows(30, 3000, 64, 2.0, 8), 64, 2.0, 8, 32),
    ("single", lambda: sasgen.random_case(31, 1, 32, 2.0, 8, 32), 32, 2.0, 8, 32),
]


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["window", "tensor", "block"])
@pytest.mark.parametrize("name,build,N,sigma,w,T", CASES, ids=[c[0] for c in CASES])
def test_kernel_vs_oracle(F, name, build, N, sigma, w, T, kernel):
    lam, v = build()
    M = lam.shape[0]
    alpha = np.random.default_rng(M + 7).uniform(0.2, 2.0, M)
    img, grid = run(F, lam, v, N, sigma, w, alpha, T, kernel)
    vc = c64(v).astype(np.complex128)
    cw = alpha.astype(np.float32) * vc
    assert O.rel_l2(grid, O.spread(lam, cw, N, sigma, w)) < TOL
    assert O.rel_l2(img, O.adjoint(lam, cw, N, sigma, w)) < TOL


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["window", "tensor", "block"])
def test_kernel_bf16_storage(F, kernel):
    """BF16 values and weights: parity against the oracle on the same bf16-rounded inputs."""
    import torch
    lam, v = sasgen.random_case(40, 5000, 64, 2.0, 8, 64)
    alpha = np.random.default_rng(41).uniform(0.3, 1.7, 5000)
    vb = torch.view_as_real(torch.from_numpy(c64(v))).to(torch.bfloat16)
    with F.Plan(dev(lam), 64, 2.0, 8, tile=32, layout=F.LAYOUT_HALO, spread_kernel=kernel,
                precision=F.PREC_BF16) as p:
        p.set_weights(dev(alpha))
        img = p.adjoint(vb.cuda()).cpu().numpy()
    vr = vb.to(torch.float64).numpy()
    vr = vr[:, 0] + 1j * vr[:, 1]
    ar = torch.from_numpy(alpha.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert O.rel_l2(img, O.adjoint(lam, ar * vr, 64, 2.0, 8)) < TOL


def test_kernels_agree_on_a_polar_ping(F):
    """The two kernels on one jittered polar raster of the batch recipe: each within the bar of
    the oracle, and within 2e-6 of each other."""
    p = sasgen.batch_ping(3)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(p.M) + 1j * rng.standard_normal(p.M)
    alpha = rng.uniform(0.5, 1.5, p.M)
    a, _ = run(F, p.lam, v, p.N, 2.0, 8, alpha, 32, 1)
    b, _ = run(F, p.lam, v, p.N, 2.0, 8, alpha, 32, 2)
    c, _ = run(F, p.lam, v, p.N, 2.0, 8, alpha, 64, 3)
    ref = O.adjoint(p.lam, alpha.astype(np.float32) * c64(v).astype(np.complex128), p.N, 2.0, 8)
    for img in (a, b, c):
        assert O.rel_l2(img, ref) < TOL
    assert O.rel_l2(b, a) < 2e-6
    assert O.rel_l2(c, a) < 2e-6


@pytest.mark.parametrize("kernel", [2, 3], ids=["tensor", "block"])
def test_tensor_kernel_empty_plan(F, kernel):
    lam = np.zeros((0, 2))
    with F.Plan(dev(lam.reshape(0, 2)), 32, 2.0, 8, tile=32, layout=F.LAYOUT_HALO,
                spread_kernel=kernel) as p:
        import torch
        img = p.adjoint(torch.zeros(0, dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert np.all(img == 0)


@pytest.mark.parametrize("kernel", [2, 3], ids=["tensor", "block"])
@pytest.mark.parametrize("kw", [dict(w=10), dict(w=4), dict(w=6, sigma=1.25),
                                dict(layout=1)], ids=["w10", "w4", "w6-sigma1.25", "duplicate"])
def test_tensor_kernel_refuses(F, kw, kernel):
    """Where the tensor-core kernel does not apply, asking for it is NOT_SUPPORTED (status 4)."""
    lam, _ = sasgen.random_case(50, 500, 32, 2.0, 8, 32)
    args = dict(w=8, sigma=2.0, layout=F.LAYOUT_HALO)
    args.update(kw)
    N = 32 if args["sigma"] == 2.0 else 64
    with pytest.raises(F.FtcgError) as ei:
        F.Plan(dev(lam), N, args["sigma"], args["w"], tile=32, layout=args["layout"],
               spread_kernel=kernel)
    assert ei.value.status == 4
