"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Bars (written here, derived from the arithmetic):
  * images / grids in FP32 storage: rel-L2 <= 1e-5 against the FP64 oracle given the same inputs;
  * weights (FP64 on the device): max relative error <= 1e-9 against the brute-force Fejer sum;
  * plan entries (integer index work): bit-exact.
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


def expected_entries(lam, N, sigma, w, T, halo=False):
    """(tile, cx, cy, sample, dx, dy). Duplicate layout: one entry for every (tile, wrap copy) a
    footprint touches (a new run of taps starts at tap 0, at a tile boundary and where the
    footprint wraps mod G). Halo layout: one entry, in the tile of the first tap."""
    G = O.grid_side(N, sigma)
    c, u = O.tap_origins(lam, N, sigma, w)
    d = (u - c).astype(np.float32)
    ntx = -(-G // T)
    rows = []
    for j in range(lam.shape[0]):
        runs = []
        for ax in (0, 1):
            cw = int(c[j, ax] % G)
            r = []
            for t in range(w):
                col = (cw + t) % G
                if t == 0 or (not halo and col % T == 0):
                    tile = col // T
                    r.append((tile, col - tile * T - t))
            runs.append(r)
        for ty, cyl in runs[1]:
            for tx, cxl in runs[0]:
                rows.append((ty * ntx + tx, cxl, cyl, j, d[j, 0], d[j, 1]))
    return rows


@pytest.mark.parametrize("layout", [1, 2], ids=["duplicate", "halo"])
@pytest.mark.parametrize("N,sigma,w,T,spread", [
    (64, 2.0, 6, 32, 64), (50, 2.0, 8, 32, 150), (40, 1.25, 5, 32, 40), (16, 2.0, 8, 64, 40),
])
def test_plan_entries_bit_exact(F, N, sigma, w, T, spread, layout):
    lam, _ = sasgen.random_case(3, 900, N, sigma, w, spread)
    lam[:5] = np.array([[3.0, -2.5], [0.25, 7.0], [N / 2, -N / 2], [-N / 2, N / 2 - 1e-12],
                        [0.0, 0.0]])          # ties and wrap edges
    with F.Plan(dev(lam), N, sigma, w, tile=T, layout=layout) as p:
        assert p.info.layout == layout
        e = p.entries()
        ncb = T + w - 1
        key = (e["tile"].astype(np.int64) * ncb + e["cx"] + w - 1) * ncb + e["cy"] + w - 1
        assert np.all(np.diff(key) >= 0), "entries not sorted by (tile, column, row)"
        got = sorted(zip(e["tile"].tolist(), e["cx"].tolist(), e["cy"].tolist(),
                         e["sample"].tolist(), e["dx"].tolist(), e["dy"].tolist()))
        exp = sorted((a, b, c, d, float(x), float(y))
                     for a, b, c, d, x, y in expected_entries(lam, N, sigma, w, T, layout == 2))
        assert len(got) == len(exp)
        assert got == exp


def _run_adjoint(F, lam, v, N, sigma, w, alpha=None, T=0, layout=0):
    with F.Plan(dev(lam), N, sigma, w, tile=T, layout=layout) as p:
        if alpha is not None:
            p.set_weights(dev(alpha))
        img = p.adjoint(dev(c64(v)))
        grid = p.spread(dev(c64(v)))
        p.check()
        return img.cpu().numpy(), grid.cpu().numpy()


def image_tol(N, sigma, w):
    """FP32 bound of an image: 1e-5, or 5e-8 A when the window division amplifies FP32 grid
    rounding by A = rms over pixels of r(p_x)^2 r(p_y)^2 / r(0)^4 (r = 1/phi^): A = 2.4 at
    sigma = 2, w = 8, but 413 at sigma = 1.5, w = 16, where the image edge is divided by a window
    transform 83 times smaller than at the centre."""
    r = O.deapod_factors(N, sigma, w)
    A = float(np.sqrt(np.mean(np.multiply.outer(r, r) ** 2)) / r[N // 2] ** 2)
    return max(TOL, 5e-8 * A)


@pytest.mark.parametrize("layout", [1, 2], ids=["duplicate", "halo"])
@pytest.mark.parametrize("M,N,sigma,w,spread,T", [
    (4096, 64, 2.0, 6, 150, 0), (3000, 50, 2.0, 8, 150, 32), (2000, 40, 1.25, 5, 40, 32),
    (5000, 96, 2.0, 7, 96, 64), (3000, 40, 2.0, 10, 120, 32), (1500, 32, 2.0, 13, 32, 32),
    (2500, 48, 1.5, 16, 60, 32), (3000, 64, 2.0, 4, 64, 64), (1, 32, 2.0, 8, 32, 0),
])
def test_adjoint_and_spread_vs_oracle(F, M, N, sigma, w, spread, T, layout):
    lam, v = sasgen.random_case(11 + M, M, N, sigma, w, spread)
    alpha = np.random.default_rng(M).uniform(0.2, 2.0, M)
    vc = c64(v).astype(np.complex128)
    img, grid = _run_adjoint(F, lam, v, N, sigma, w, alpha, T, layout)
    ref = O.adjoint(lam, alpha.astype(np.float32) * vc, N, sigma, w)
    assert O.rel_l2(img, ref) < image_tol(N, sigma, w)
    gref = O.spread(lam, alpha.astype(np.float32) * vc, N, sigma, w)
    assert O.rel_l2(grid, gref) < TOL


@pytest.mark.parametrize("xlo,xhi", [(-3.0, 3.0), (6.0, 14.0), (-32.0, 32.0), (-31.0, -29.5)],
                         ids=["wraps", "one-run", "all-columns", "edge"])
def test_pruned_fft_column_runs(F, xlo, xhi):
    """The inverse FFT transforms only the grid columns that taps reach (one or two periodic runs)
    and only the rows of the crop: samples confined to a band of lambda_x around 0 (the occupied
    columns wrap around G), off centre (one run), everywhere, and at the band edge."""
    rng = np.random.default_rng(int(100 * (xlo + 40)))
    M, N = 2500, 64
    lam = np.stack([rng.uniform(xlo, xhi, M), rng.uniform(-32, 32, M)], axis=1)
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    img, _ = _run_adjoint(F, lam, v, N, 2.0, 8)
    ref = O.adjoint(lam, c64(v).astype(np.complex128), N, 2.0, 8)
    assert O.rel_l2(img, ref) < TOL


@pytest.mark.parametrize("N,sigma,xlo,xhi", [
    (128, 2.0, -3.0, 3.0), (128, 2.0, 6.0, 14.0), (256, 2.0, -128.0, 128.0),
    (512, 2.0, -40.0, 90.0), (160, 1.6, -80.0, 80.0)])
def test_smem_fft_sizes(F, N, sigma, xlo, xhi):
    """Grid sides 256, 512 and 1024 take the shared-memory transforms (column blocks that taps
    reach, then the crop's rows fused with the window division): whole images against the oracle,
    with occupied columns that wrap, form one run, cover everything, or sit off centre."""
    rng = np.random.default_rng(N + int(xlo))
    M = 4000
    lam = np.stack([rng.uniform(xlo, xhi, M), rng.uniform(-N / 2, N / 2, M)], axis=1)
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    img, _ = _run_adjoint(F, lam, v, N, sigma, 8)
    ref = O.adjoint(lam, c64(v).astype(np.complex128), N, sigma, 8)
    assert O.rel_l2(img, ref) < image_tol(N, sigma, 8)


def test_smem_fft_4096_sampled(F):
    """G = 4096 (N = 2048): sampled pixels against the oracle one by one."""
    rng = np.random.default_rng(7)
    M, N = 3000, 2048
    lam = np.stack([rng.uniform(-700, 300, M), rng.uniform(-1024, 1024, M)], axis=1)
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    img, _ = _run_adjoint(F, lam, v, N, 2.0, 8)
    pix = rng.integers(-N // 2, N // 2, size=(40, 2))
    ref = O.adjoint_pixels(lam, c64(v).astype(np.complex128), N, 2.0, 8, pix)
    assert O.rel_l2(img[pix[:, 1] + N // 2, pix[:, 0] + N // 2], ref) < TOL


def test_image_at_8_byte_offset(F):
    """An output image that is only 8-byte aligned takes the element-wise path of the window
    division; N = 64 (the vector path otherwise) so both paths are compared on one raster."""
    import torch
    lam, v = sasgen.random_case(5, 3000, 64, 2.0, 8, 100)
    vc = c64(v)
    with F.Plan(dev(lam), 64, 2.0, 8) as p:
        aligned = p.adjoint(dev(vc)).cpu().numpy()
        buf = torch.zeros(64 * 64 + 1, dtype=torch.complex64, device="cuda")
        view = buf[1:].view(64, 64)
        assert view.data_ptr() % 16 == 8
        p.adjoint(dev(vc), out=view)
        shifted = view.cpu().numpy()
    assert O.rel_l2(shifted, aligned) < 1e-6      # shared-memory atomics: order varies per call
    ref = O.adjoint(lam, vc.astype(np.complex128), 64, 2.0, 8)
    assert O.rel_l2(shifted, ref) < TOL


def test_tiny_config(F):
    """The 4096-sample polar raster: weights, weighted image vs O2 and vs the direct sum."""
    p = sasgen.tiny()
    v = sasgen.values_for(p)
    with F.Plan(dev(p.lam), p.N, p.sigma, p.w) as pl:
        a = pl.weights().cpu().numpy()
        img = pl.adjoint(dev(c64(v))).cpu().numpy()
        pl.check()
    ab, _ = O.weights_brute(p.lam, p.N)
    assert np.max(np.abs(a - ab) / ab) < 1e-9
    vc = c64(v).astype(np.complex128)
    ref = O.adjoint(p.lam, ab * vc, p.N, p.sigma, p.w)
    assert O.rel_l2(img, ref) < TOL
    direct = O.direct_adjoint(p.lam, ab * vc, p.N)
    assert O.rel_l2(img, direct) < 1.2e-5 + TOL    # the w = 6 window's own bound plus FP32


def test_empty_plan(F):
    import torch
    lam = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    with F.Plan(lam, 32, 2.0, 8) as p:
        v = torch.zeros(0, dtype=torch.complex64, device="cuda")
        img = p.adjoint(v)
        assert torch.count_nonzero(img).item() == 0
        p.weights()
        p.check()


@pytest.mark.parametrize("layout", [1, 2], ids=["duplicate", "halo"])
def test_collisions_one_cell(F, layout):
    """Every sample in the same cell: maximal shared-atomic contention."""
    rng = np.random.default_rng(4)
    M, N = 3000, 32
    lam = np.tile([[1.3, -2.7]], (M, 1)) + 1e-3 * rng.random((M, 2))
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    img, _ = _run_adjoint(F, lam, v, N, 2.0, 8, layout=layout)
    ref = O.adjoint(lam, c64(v).astype(np.complex128), N, 2.0, 8)
    assert O.rel_l2(img, ref) < TOL


def test_forward_and_adjointness(F):
    lam, c = sasgen.random_case(21, 3000, 48, spread=100)
    rng = np.random.default_rng(22)
    img = (rng.standard_normal((48, 48)) + 1j * rng.standard_normal((48, 48))).astype(np.complex64)
    with F.Plan(dev(lam), 48, 2.0, 8) as p:
        f = p.forward(dev(img)).cpu().numpy()
        a = p.adjoint(dev(c64(c))).cpu().numpy()
    ref = O.forward(lam, img.astype(np.complex128), 48, 2.0, 8)
    assert O.rel_l2(f, ref) < TOL
    lhs = np.vdot(img.astype(np.complex128), a.astype(np.complex128))
    rhs = np.vdot(f.astype(np.complex128), c64(c).astype(np.complex128))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_weights_random(F):
    lam, _ = sasgen.random_case(31, 3000, 40, spread=30)
    with F.Plan(dev(lam), 40, 2.0, 8) as p:
        a = p.weights().cpu().numpy()
    ab, _ = O.weights_brute(lam, 40)
    assert np.max(np.abs(a - ab) / ab) < 1e-9


@pytest.mark.parametrize("sigma,wa", [(2.0, 12), (1.5, 14), (1.25, 16), (2.0, 16), (2.0, 0)])
def test_weights_widths(F, sigma, wa):
    """The FP64 weight path at several oversampling factors and weight-window widths (0 = the
    default 12), each wide enough that the gridding error of the lag sums is below the 1e-9 bar
    (exp(-beta) <= 1e-12; at sigma = 2, w = 10 the gridding error alone is 2e-9), against the
    brute-force Fejer sum."""
    lam, _ = sasgen.random_case(37, 2500, 40, spread=36)
    with F.Plan(dev(lam), 40, sigma, 8, weight_width=wa) as p:
        a = p.weights().cpu().numpy()
    ab, _ = O.weights_brute(lam, 40)
    assert np.max(np.abs(a - ab) / ab) < 1e-9


def test_weights_uniform_grid(F):
    N = 32
    g = np.arange(-N // 2, N // 2)
    X, Y = np.meshgrid(g, g)
    lam = np.stack([X.ravel(), Y.ravel()], 1).astype(np.float64)
    with F.Plan(dev(lam), N, 2.0, 8) as p:
        a = p.weights().cpu().numpy()
    assert np.max(np.abs(a - 1.0)) < 1e-9


def test_nonfinite_coordinate_reported(F):
    from paper_1706_08575_gb300 import FtcgError
    lam, v = sasgen.random_case(41, 100, 32)
    lam[7, 0] = np.nan
    with pytest.raises(FtcgError) as ei:
        F.Plan(dev(lam), 32, 2.0, 8)
    assert ei.value.status == 5
    p = F.Plan(dev(lam), 32, 2.0, 8, allow_numeric=True)
    img = p.adjoint(dev(c64(v))).cpu().numpy()
    keep = np.ones(100, bool)
    keep[7] = False
    ref = O.adjoint(lam[keep], c64(v[keep]).astype(np.complex128), 32, 2.0, 8)
    assert O.rel_l2(img, ref) < TOL
    p.close()


@pytest.mark.parametrize("N", [64, 128], ids=["cufft-path", "smem-fft-path"])
def test_adjoint_captured_in_cuda_graph(F, N):
    """ftcg_adjoint enqueues only kernels and cuFFT executions on its stream, so it can be captured
    in a CUDA graph and replayed (with new values in the same buffer)."""
    import torch
    lam, v = sasgen.random_case(61, 3000, N, spread=N)
    v2 = np.random.default_rng(62).standard_normal(3000) + 1j
    with F.Plan(dev(lam), N, 2.0, 8) as p:
        vals = dev(c64(v))
        img = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
        p.adjoint(vals, out=img)                       # warm-up outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            p.adjoint(vals, out=img)
        vals.copy_(dev(c64(v2)))
        img.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = img.cpu().numpy()
    ref = O.adjoint(lam, c64(v2).astype(np.complex128), N, 2.0, 8)
    assert O.rel_l2(got, ref) < TOL


@pytest.mark.parametrize("N", [64, 128], ids=["cufft-path", "smem-fft-path"])
@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_adjoint_host_matches_device(F, N, pinned):
    """Host buffers: a pinned image is written in place by the device, a pageable one through a
    staging copy; both equal the device-buffer adjoint."""
    import torch
    lam, v = sasgen.random_case(51, 2000, N, spread=N)
    with F.Plan(dev(lam), N, 2.0, 8) as p:
        a = p.adjoint(dev(c64(v))).cpu()
        hv = torch.from_numpy(c64(v))
        himg = torch.full((N, N), 7.0 + 0j, dtype=torch.complex64)
        if pinned:
            hv, himg = hv.pin_memory(), himg.pin_memory()
        p.adjoint_host(hv, himg)
        p.adjoint_host(hv, himg)                       # twice: the result does not accumulate
    assert O.rel_l2(himg.numpy(), a.numpy()) < 1e-6   # same kernels; atomics order may differ


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_adjoint_host_async_pipeline(F, pinned):
    """ftcg_adjoint_host_async: a stream of calls with different values and two alternating
    images, enqueued back to back (each upload overlapping the previous adjoint); after one
    synchronisation every image equals the device adjoint of its own values."""
    import torch
    N = 64
    lam, _ = sasgen.random_case(52, 3000, N, spread=N)
    rng = np.random.default_rng(53)
    vs = [c64(rng.standard_normal(3000) + 1j * rng.standard_normal(3000)) for _ in range(5)]
    with F.Plan(dev(lam), N, 2.0, 8) as p:
        refs = [p.adjoint(dev(v)).cpu().numpy() for v in vs]
        hvs = [torch.from_numpy(v) for v in vs]
        imgs = [[torch.full((N, N), 7.0 + 0j, dtype=torch.complex64) for _ in range(2)]
                for _ in vs]
        if pinned:
            hvs = [h.pin_memory() for h in hvs]
            imgs = [[i.pin_memory() for i in pair] for pair in imgs]
        s = torch.cuda.Stream()
        outs = []
        for k, hv in enumerate(hvs):
            outs.append(p.adjoint_host_async(hv, imgs[k][k % 2], stream=s))
        s.synchronize()
    for got, ref in zip(outs, refs):
        assert O.rel_l2(got.numpy(), ref) < 1e-6
