"""The exact judge and fallback of predicted weights (ftcg_weights_judge,
ftcg_batch_weights_judge): exact Fejer sums at K samples (Eq. difopt at r = 1) calibrate the
predictions by their median ratio and estimate the remaining relative error; within the bound the
calibrated predictions are installed, otherwise the exact weights.

Bars: a prediction that is the exact weights times a constant is accepted with that constant as
its median ratio (to the judge's own accuracy, 1e-6) and gridded within the FP32 bar (1e-5) of
the exact-weight image; a prediction with 5% random errors is rejected and the exact weights are
installed instead (image within 1e-5)."""
import numpy as np
import pytest

import sasgen
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


def test_judge_accepts_a_scaled_exact_prediction_and_rejects_a_noisy_one(F):
    q = sasgen.batch_ping(1)
    rng = np.random.default_rng(2)
    v = dev((rng.standard_normal(q.M) + 1j * rng.standard_normal(q.M)).astype(np.complex64))
    with F.Plan(dev(q.lam), q.N, 2.0, 8) as p:
        a = p.weights()
        ref = p.adjoint(v).cpu().numpy()
        ok, st = p.judge_weights(a * 1.3, K=128, max_rel_err=5e-4)
        assert ok and abs(st["median_ratio"] - 1.3) < 1e-6 * 1.3 and st["rms"] < 1e-6
        img = p.adjoint(v).cpu().numpy()
        assert O.rel_l2(img, ref) < 1e-5
        noisy = a * dev(rng.uniform(0.95, 1.05, q.M))
        ok, st = p.judge_weights(noisy, K=128, max_rel_err=5e-4)
        assert not ok and st["rms"] > 1e-2
        img = p.adjoint(v).cpu().numpy()
        assert O.rel_l2(img, ref) < 1e-5


def test_judge_sums_are_the_exact_weight_sums(F):
    """The judge's median ratio for unit predictions is the median of S_k over its samples:
    checked against the brute-force oracle sums at the same samples."""
    lam, _ = sasgen.random_case(3, 5000, 64, 2.0, 8, 40)
    K = 64
    ks = (np.arange(K) * 2 + 1) * 5000 // (2 * K)
    _, S = O.weights_brute(lam, 64, ks)
    import torch
    with F.Plan(dev(lam), 64, 2.0, 8) as p:
        ok, st = p.judge_weights(torch.ones(5000, dtype=torch.float64, device="cuda"), K=K,
                                 max_rel_err=1.0)
    assert abs(st["median_ratio"] - np.median(S)) < 1e-6 * np.median(S)
    r = S / np.median(S) - 1
    assert abs(st["rms"] - np.sqrt(np.mean(r ** 2))) < 1e-6


def test_batch_judge_per_ping(F):
    pings = [sasgen.batch_ping(b) for b in (1, 2, 3)]
    with F.Batch([dev(q.lam) for q in pings], [q.N for q in pings], 2.0, 8) as b:
        exact = b.weights()
        rng = np.random.default_rng(4)
        pred = [exact[0] * 0.8, exact[1] * dev(rng.uniform(0.9, 1.1, pings[1].M)), exact[2]]
        res = b.judge_weights(pred, K=64, max_rel_err=5e-4)
        vals = [dev((rng.standard_normal(q.M) + 0j).astype(np.complex64)) for q in pings]
        imgs = [i.cpu().numpy() for i in b.adjoint(vals)]
    assert [r[0] for r in res] == [True, False, True]
    assert abs(res[0][1][0] - 0.8) < 1e-6
    for q, x, a, img in zip(pings, vals, exact, imgs):
        ref = O.adjoint(q.lam, a.cpu().numpy().astype(np.float32) *
                        x.cpu().numpy().astype(np.complex128), q.N, 2.0, 8)
        assert O.rel_l2(img, ref) < 1e-5



def test_judge_leaves_out_nonfinite_samples(F):
    """A raster holding non-finite coordinates (the gridding drops them, their exact weight is 0):
    the judge leaves them out of the sums and of the ratios, so a scaled exact prediction is still
    accepted with its factor, and its sums still match the brute-force sums over the finite
    samples."""
    lam, _ = sasgen.random_case(8, 3000, 48, 2.0, 8, 40)
    lam = lam.copy()
    bad = [5, 1500, 2999]
    lam[bad] = [[np.nan, 0.0], [0.0, np.inf], [np.nan, np.nan]]
    with F.Plan(dev(lam), 48, 2.0, 8, allow_numeric=True) as p:
        a = p.weights()
        assert np.all(a.cpu().numpy()[bad] == 0)
        ok, st = p.judge_weights(a * 0.7, K=3000, max_rel_err=5e-4)
    assert ok and abs(st["median_ratio"] - 0.7) < 1e-6 * 0.7 and st["rms"] < 1e-6
