"""Batched pings through the C ABI: one persistent spreading launch, batched FFTs per grid side,
one window-division launch; with and without CUDA-graph capture. Every image is compared with
the FP64 oracle (and with the single-ping path) element by element."""
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


def small_batch(seed=0):
    rng = np.random.default_rng(seed)
    cases = []
    for i, N in enumerate([32, 64, 48, 64, 32, 96, 40]):
        M = int(rng.integers(200, 6000)) if i != 4 else 0
        lam, v = sasgen.random_case(seed * 100 + i, M, N, 2.0, 8, spread=1.5 * N)
        alpha = rng.uniform(0.3, 1.7, M)
        cases.append((lam, v.astype(np.complex64), alpha, N))
    return cases


@pytest.mark.parametrize("layout", [0, 1, 2], ids=["auto", "duplicate", "halo"])
def test_batch_vs_oracle_and_single(F, layout):
    cases = small_batch(1)
    lams = [dev(c[0]) for c in cases]
    vals = [dev(c[1]) for c in cases]
    alphas = [dev(c[2]) for c in cases]
    with F.Batch(lams, [c[3] for c in cases], 2.0, 8, layout=layout) as b:
        tiles, entries, _ = b.info()
        assert set(tiles) <= {32, 64}
        b.set_weights(alphas)
        imgs = [x.cpu().numpy() for x in b.adjoint(vals)]
    for (lam, v, a, N), img in zip(cases, imgs):
        ref = O.adjoint(lam, a.astype(np.float32) * v.astype(np.complex128), N, 2.0, 8)
        if lam.shape[0] == 0:
            assert np.count_nonzero(img) == 0
            continue
        assert O.rel_l2(img, ref) < TOL
        with F.Plan(dev(lam), N, 2.0, 8) as p:
            p.set_weights(dev(a))
            single = p.adjoint(dev(v)).cpu().numpy()
        assert O.rel_l2(img, single) < 1e-6


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["window", "tensor", "block"])
def test_batch_each_spread_kernel(F, kernel):
    """The persistent batched launch with each spreading kernel forced (halo layout), over pings
    of both FFT paths (cuFFT below G = 256, shared-memory passes from 256) and an empty ping,
    against the oracle."""
    rng = np.random.default_rng(20 + kernel)
    cases = []
    for i, N in enumerate([32, 128, 64, 256, 48]):
        M = 0 if i == 2 else int(rng.integers(800, 6000))
        lam, v = sasgen.random_case(300 + 10 * kernel + i, M, N, 2.0, 8, spread=1.2 * N)
        cases.append((lam, v.astype(np.complex64), rng.uniform(0.3, 1.7, M), N))
    with F.Batch([dev(c[0]) for c in cases], [c[3] for c in cases], 2.0, 8,
                 layout=F.LAYOUT_HALO, spread_kernel=kernel) as b:
        b.set_weights([dev(c[2]) for c in cases])
        imgs = [x.cpu().numpy() for x in b.adjoint([dev(c[1]) for c in cases])]
    for (lam, v, a, N), img in zip(cases, imgs):
        if lam.shape[0] == 0:
            assert np.count_nonzero(img) == 0
            continue
        ref = O.adjoint(lam, a.astype(np.float32) * v.astype(np.complex128), N, 2.0, 8)
        assert O.rel_l2(img, ref) < TOL


def test_batch_graph_replay(F):
    import torch
    cases = [c for c in small_batch(2) if c[0].shape[0] > 0]
    lams = [dev(c[0]) for c in cases]
    vals = [dev(c[1]) for c in cases]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s), F.Batch(lams, [c[3] for c in cases], 2.0, 8, tile=32) as b:
        imgs = b.capture(vals)
        for x in imgs:
            x.zero_()
        b.launch()
        b.launch()
        s.synchronize()
        got = [x.cpu().numpy() for x in imgs]
    for (lam, v, a, N), img in zip(cases, got):
        ref = O.adjoint(lam, v.astype(np.complex128), N, 2.0, 8)
        assert O.rel_l2(img, ref) < TOL


def test_batch_bf16_values_and_weights(F):
    import torch
    cases = [c for c in small_batch(3) if c[0].shape[0] > 0][:4]
    lams = [dev(c[0]) for c in cases]
    vb = [torch.view_as_real(torch.from_numpy(c[1])).to(torch.bfloat16).cuda() for c in cases]
    with F.Batch(lams, [c[3] for c in cases], 2.0, 8, precision=F.PREC_BF16) as b:
        alphas = b.weights()
        imgs = [x.cpu().numpy() for x in b.adjoint(vb)]
        alphas = [a.cpu().numpy() for a in alphas]
    for (lam, v, _, N), img, a, vbt in zip(cases, imgs, alphas, vb):
        ab, _ = O.weights_brute(lam, N)
        assert np.max(np.abs(a - ab) / ab) < 1e-9
        vr = vbt.cpu().to(torch.float64).numpy()
        vr = vr[:, 0] + 1j * vr[:, 1]
        a_r = torch.from_numpy(ab.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
        ref = O.adjoint(lam, a_r * vr, N, 2.0, 8)
        assert O.rel_l2(img, ref) < TOL


def test_batch_of_sas_pings_sampled(F):
    """Eight pings of the uneven SAS batch recipe (20k-400k samples, N in {256, 512, 1024}):
    sampled pixels against the oracle one by one."""
    pings = [sasgen.batch_ping(b) for b in range(8)]
    vals = [sasgen.values_for(p, device="cuda").astype(np.complex64) for p in pings]
    with F.Batch([dev(p.lam) for p in pings], [p.N for p in pings], 2.0, 8) as b:
        imgs = [x.cpu().numpy() for x in b.adjoint([dev(v) for v in vals])]
    rng = np.random.default_rng(4)
    for p, v, img in zip(pings, vals, imgs):
        pix = np.concatenate([rng.integers(-p.N // 2, p.N // 2, size=(6, 2)), p.bright_pixels])
        ref = O.adjoint_pixels(p.lam, v.astype(np.complex128), p.N, 2.0, 8, pix)
        got = img[pix[:, 1] + p.N // 2, pix[:, 0] + p.N // 2]
        assert O.rel_l2(got, ref) < TOL


def test_batch_mixed_fft_classes_and_graph(F):
    """Pings whose grid side is a power of two from 256 take the shared-memory FFT passes (column
    blocks that taps reach, then the rows fused with the window division); the others cuFFT and a
    separate window division. A batch mixing both, with an empty ping, against the oracle, directly
    and replayed from a CUDA graph."""
    import torch
    rng = np.random.default_rng(9)
    cases = []
    for i, N in enumerate([128, 96, 256, 128, 128]):
        M = 0 if i == 3 else int(rng.integers(1500, 5000))
        lo = -N / 2 if i != 4 else -3.0
        hi = N / 2 if i != 4 else 3.0
        lam = np.stack([rng.uniform(lo, hi, M), rng.uniform(-N / 2, N / 2, M)], axis=1)
        v = (rng.standard_normal(M) + 1j * rng.standard_normal(M)).astype(np.complex64)
        cases.append((lam, v, N))
    lams = [dev(c[0]) for c in cases]
    vals = [dev(c[1]) for c in cases]
    refs = [O.adjoint(lam, v.astype(np.complex128), N, 2.0, 8) if lam.shape[0] else None
            for lam, v, N in cases]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s), F.Batch(lams, [c[2] for c in cases], 2.0, 8) as b:
        direct = [x.cpu().numpy() for x in b.adjoint(vals)]
        imgs = b.capture(vals)
        for x in imgs:
            x.fill_(1.0)
        b.launch()
        s.synchronize()
        replay = [x.cpu().numpy() for x in imgs]
    for ref, d, r in zip(refs, direct, replay):
        if ref is None:
            assert np.count_nonzero(d) == 0 and np.count_nonzero(r) == 0
            continue
        assert O.rel_l2(d, ref) < TOL
        assert O.rel_l2(r, ref) < TOL


def test_batch_bf16_smem_classes(F):
    """BF16 values and weights through the shared-memory FFT classes (G = 256 and 512) and a
    cuFFT class, against the oracle on the same bf16-rounded inputs."""
    import torch
    rng = np.random.default_rng(21)
    cases = []
    for N in [128, 256, 96]:
        M = int(rng.integers(2000, 5000))
        lam = np.stack([rng.uniform(-N / 2, N / 2, M), rng.uniform(-N / 2, N / 2, M)], axis=1)
        v = (rng.standard_normal(M) + 1j * rng.standard_normal(M)).astype(np.complex64)
        cases.append((lam, v, N))
    vb = [torch.view_as_real(torch.from_numpy(c[1])).to(torch.bfloat16).cuda() for c in cases]
    with F.Batch([dev(c[0]) for c in cases], [c[2] for c in cases], 2.0, 8,
                 precision=F.PREC_BF16) as b:
        alphas = [a.cpu().numpy() for a in b.weights()]
        imgs = [x.cpu().numpy() for x in b.adjoint(vb)]
    for (lam, _, N), img, a, vbt in zip(cases, imgs, alphas, vb):
        vr = vbt.cpu().to(torch.float64).numpy()
        vr = vr[:, 0] + 1j * vr[:, 1]
        a_r = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
        ref = O.adjoint(lam, a_r * vr, N, 2.0, 8)
        assert O.rel_l2(img, ref) < TOL


def test_batch_of_one_ping(F):
    """A batch of one ping (its plan is built on the caller's thread) against the oracle."""
    lam, v, a, N = small_batch(5)[0]
    with F.Batch([dev(lam)], [N], 2.0, 8) as b:
        b.set_weights([dev(a)])
        img = b.adjoint([dev(v)])[0].cpu().numpy()
    ref = O.adjoint(lam, a.astype(np.float32) * v.astype(np.complex128), N, 2.0, 8)
    assert O.rel_l2(img, ref) < TOL


def test_batch_ping_with_nonfinite_coordinate(F):
    """A ping with a NaN coordinate among pings planned concurrently: the batch is built, that
    sample is dropped (the image equals the oracle without it), the other pings are unaffected."""
    cases = [c for c in small_batch(6) if c[0].shape[0] > 0]
    lam_bad = cases[2][0].copy()
    lam_bad[5, 0] = np.nan
    lams = [dev(c[0]) if k != 2 else dev(lam_bad) for k, c in enumerate(cases)]
    vals = [dev(c[1]) for c in cases]
    with F.Batch(lams, [c[3] for c in cases], 2.0, 8) as b:
        imgs = [x.cpu().numpy() for x in b.adjoint(vals)]
    for k, ((lam, v, a, N), img) in enumerate(zip(cases, imgs)):
        keep = np.ones(lam.shape[0], bool)
        if k == 2:
            keep[5] = False
        ref = O.adjoint(lam[keep], v[keep].astype(np.complex128), N, 2.0, 8)
        assert O.rel_l2(img, ref) < TOL, k


def test_batch_tuner_one_choice_for_the_mix(F, tmp_path):
    """The batch tuner times its candidates on the batch's mix of pings and records one choice
    for every key it decides (w = 7 here, a width no other test of this process tunes); the
    batch built with that choice still matches the oracle."""
    import json
    rng = np.random.default_rng(77)
    cases = []
    for i, (N, M) in enumerate([(32, 300), (64, 9000), (48, 2500), (96, 30000), (40, 80),
                                (64, 600), (128, 50000)]):
        lam, v = sasgen.random_case(7700 + i, M, N, 2.0, 7, spread=1.5 * N)
        cases.append((lam, v.astype(np.complex64), rng.uniform(0.3, 1.7, M), N))
    with F.Batch([dev(c[0]) for c in cases], [c[3] for c in cases], 2.0, 7) as b:
        b.set_weights([dev(c[2]) for c in cases])
        imgs = [x.cpu().numpy() for x in b.adjoint([dev(c[1]) for c in cases])]
    path = tmp_path / "tuner.json"
    F.ftcg.tuner_save(path)
    ent = [e for e in json.loads(path.read_text())["entries"] if e["batch"] == 1 and e["w"] == 7]
    assert len({e["bucket"] for e in ent}) >= 3          # several keys, decided together
    assert len({(e["tile"], e["layout"], e["spread"]) for e in ent}) == 1
    for (lam, v, a, N), img in zip(cases, imgs):
        ref = O.adjoint(lam, a.astype(np.float32) * v.astype(np.complex128), N, 2.0, 7)
        assert O.rel_l2(img, ref) < TOL
