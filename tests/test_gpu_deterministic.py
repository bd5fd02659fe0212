"""opts.deterministic through the C ABI: adjoints bitwise reproducible across calls and across
plans built from the same inputs, still within the FP32 bar of the FP64 oracle; the
configurations it does not cover are refused.

The cases put many samples in the same first-tap cells (the order the plan must fix), wrap
around the periodic grid, and install random weights."""
import ctypes

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


def clustered_case(seed, M, N, cells):
    """M samples in a few first-tap cells' neighbourhoods (heavy collisions) plus a spread part."""
    rng = np.random.default_rng(seed)
    centres = (rng.random((cells, 2)) - 0.5) * 1.5 * N
    lam = centres[rng.integers(0, cells, M // 2)] + rng.uniform(-0.4, 0.4, (M // 2, 2))
    lam = np.concatenate([lam, (rng.random((M - M // 2, 2)) - 0.5) * 1.5 * N])
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    return lam, v.astype(np.complex64), rng.uniform(0.3, 1.7, M)


@pytest.mark.parametrize("N,M,tile", [(64, 20000, 0), (128, 60000, 64), (256, 150000, 32)])
def test_deterministic_bitwise_and_parity(F, N, M, tile):
    lam, v, alpha = clustered_case(N + M, M, N, 40)
    imgs = []
    for _ in range(2):                         # two plans from the same inputs
        with F.Plan(dev(lam), N, 2.0, 8, tile=tile, deterministic=True) as p:
            assert p.info.spread_kernel == F.SPREAD_BLOCK and p.info.layout == F.LAYOUT_HALO
            p.set_weights(dev(alpha))
            for _ in range(2):                 # and two calls of each
                imgs.append(p.adjoint(dev(v)).cpu().numpy())
    for img in imgs[1:]:
        assert np.array_equal(img.view(np.uint64), imgs[0].view(np.uint64))
    ref = O.adjoint(lam, alpha.astype(np.float32) * v.astype(np.complex128), N, 2.0, 8)
    assert O.rel_l2(imgs[0], ref) < TOL


def test_deterministic_large_ping_bitwise(F):
    """The benchmark's geometry (halo layout at T = 32, 1,365 non-empty tiles)."""
    p = sasgen.large_ping()
    lam = dev(p.lam)
    v = dev(sasgen.values_for(p).astype(np.complex64))
    out = []
    for _ in range(2):
        with F.Plan(lam, p.N, p.sigma, p.w, deterministic=True) as pl:
            out.append(pl.adjoint(v).cpu().numpy())
    assert np.array_equal(out[0].view(np.uint64), out[1].view(np.uint64))
    with F.Plan(lam, p.N, p.sigma, p.w) as pl:  # the default plan agrees to rounding
        fast = pl.adjoint(v).cpu().numpy()
    assert O.rel_l2(out[0], fast) < 2e-6


@pytest.mark.parametrize("kw", [dict(w=10), dict(N=50), dict(layout=1), dict(spread_kernel=1)],
                         ids=["w10", "G100", "duplicate", "window-kernel"])
def test_deterministic_refusals(F, kw):
    args = dict(N=64, w=8, layout=0, spread_kernel=0)
    args.update(kw)
    lam, _, _ = clustered_case(1, 500, args["N"], 4)
    with pytest.raises(F.FtcgError) as e:
        F.Plan(dev(lam), args["N"], 2.0, args["w"], layout=args["layout"],
               spread_kernel=args["spread_kernel"], deterministic=True)
    assert e.value.status == 4                 # FTCG_ERR_NOT_SUPPORTED


def test_deterministic_batch_refused(F):
    lam, _, _ = clustered_case(2, 500, 64, 4)
    t = dev(lam)
    lams = (ctypes.c_void_p * 1)(t.data_ptr())
    M = (ctypes.c_int64 * 1)(500)
    N = (ctypes.c_int32 * 1)(64)
    o = F.ftcg.Opts(0, 0, 0, 0, 0, 0, 1)
    h = ctypes.c_void_p()
    st = F.lib().ftcg_plan_batch(ctypes.byref(h), 1, lams, M, N, 2.0, 8, ctypes.byref(o), None)
    assert st == 4 and not h.value
