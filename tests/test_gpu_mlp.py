"""The learned-weight path on the GPU against the FP64 oracle: exact kNN features, BF16
tensor-core forward and gradients, on-device training, checkpoint continuation, and the gain the
trained network brings over gridding without weights.

Bars: neighbour indices bit-exact; feature values within bfloat16 rounding (2^-8 relative).
Forward y, the loss and every gradient tensor are held to a bar derived per tensor from the
device's arithmetic: the device rounds to bfloat16 (unit roundoff 2^-9) exactly at six points,
the activations h1, h2, h3 and the back-propagated dz3, dz2, dz1, and computes everything else
in FP32 on bf16-rounded parameters and features. `bf16_model` repeats the network in FP64 with
those six roundings; its distance E from the FP64 oracle (no rounding) is the error the
roundings alone cause for that tensor, and the device must lie within 4 E + 1e-5 of the oracle
(the factor covers roundings that fall differently on FP32 inputs; 1e-5 the FP32 accumulation),
and within 1e-3 of the model itself."""
import numpy as np
import pytest

import sasgen
from oracle import ftcg_oracle as O
from oracle import mlp_oracle as L

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


def bf16(x):
    import torch
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def nrel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def bf16_model(P, X, t):
    """The network's forward pass, loss and gradients in FP64 with bfloat16 rounding where the
    device rounds (h1, h2, h3 and dz3, dz2, dz1); P holds the bf16-rounded weights."""
    r = bf16
    z1 = X @ P["W1"] + P["b1"]
    h1 = r(L.gelu(z1))
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = r(L.gelu(z2))
    z3 = h2 @ P["W3"] + P["b3"]
    h3 = r(L.gelu(z3))
    y = h3 @ P["w4"] + P["b4"][0]
    dy = 2.0 * (y - t) / y.shape[0]
    g = {"w4": h3.T @ dy, "b4": np.array([dy.sum()])}
    dz3 = r(np.outer(dy, P["w4"]) * L.gelu_grad(z3))
    g["W3"], g["b3"] = h2.T @ dz3, dz3.sum(0)
    dz2 = r((dz3 @ P["W3"].T) * L.gelu_grad(z2))
    g["W2"], g["b2"] = h1.T @ dz2, dz2.sum(0)
    dz1 = r((dz2 @ P["W2"].T) * L.gelu_grad(z1))
    g["W1"], g["b1"] = X.T @ dz1, dz1.sum(0)
    return y, g, L.loss(y, t)


def test_features_exact_neighbours(F):
    rng = np.random.default_rng(0)
    lam = rng.random((3000, 2)) * 40 - 20
    g = np.arange(8.0)
    X, Y = np.meshgrid(g, g)
    lat = np.stack([X.ravel(), Y.ravel()], 1) * 0.5 + 30.0       # a lattice: many exact ties
    lam = np.concatenate([lam, lat])
    aux = rng.uniform(-0.1, 0.1, lam.shape[0])
    feats, nb = F.features(dev(lam), dev(aux), neighbors=True)
    ref, idx = L.knn_features(lam, aux)
    assert np.array_equal(nb.cpu().numpy(), idx)
    got = feats.cpu().float().numpy().astype(np.float64)
    assert np.all(got[:, L.D_IN:] == 0)
    err = np.abs(got[:, :L.D_IN] - ref)
    assert np.all(err <= 2.0 ** -8 * np.abs(ref) + 1e-30)


def test_features_unaligned_outputs(F):
    """Outputs that are only 4-byte aligned take the element-wise store path: same features and
    neighbours as the 16-byte vector path."""
    import ctypes
    import torch
    from paper_1706_08575_gb300 import ftcg as A
    rng = np.random.default_rng(1)
    lam = dev(rng.random((2000, 2)) * 30 - 15)
    aux = dev(rng.uniform(-0.1, 0.1, 2000))
    feats, nb = F.features(lam, aux, neighbors=True)
    M = 2000
    fbuf = torch.zeros(M * 48 + 2, dtype=torch.bfloat16, device="cuda")
    nbuf = torch.zeros(M * 16 + 1, dtype=torch.int32, device="cuda")
    fptr, nptr = fbuf.data_ptr() + 4, nbuf.data_ptr() + 4          # 4-byte offsets
    assert fptr % 16 != 0 and nptr % 16 != 0
    st = A.lib().ftcg_features(ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(aux.data_ptr()),
                               ctypes.c_int64(M), ctypes.c_void_p(fptr), ctypes.c_void_p(nptr),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert torch.equal(fbuf[2:].view(M, 48), feats)
    assert torch.equal(nbuf[1:].view(M, 16), nb)


def test_features_batch_matches_single_calls(F):
    """Several rasters in one request (an empty one, one with fewer than 16 other samples, uneven
    sizes, aux given for some): features and neighbours bit-identical to one call per raster,
    and neighbours of the small raster checked against the oracle."""
    import torch
    from paper_1706_08575_gb300 import FtcgError
    rng = np.random.default_rng(4)
    sizes = [1500, 0, 5, 7000, 300, 2500]
    lams = [dev(rng.random((m, 2)) * 30 - 15) for m in sizes]
    auxs = [dev(rng.uniform(-0.1, 0.1, m)) if k % 2 == 0 else None for k, m in enumerate(sizes)]
    parts, nbs = F.features_batch(lams, auxs, neighbors=True)
    for lam, aux, fp, nbp, m in zip(lams, auxs, parts, nbs, sizes):
        assert fp.shape == (m, 48) and nbp.shape == (m, 16)
        if m == 0:
            continue
        f1, n1 = F.features(lam, aux, neighbors=True)
        assert torch.equal(fp, f1) and torch.equal(nbp, n1)
    _, idx = L.knn_features(lams[4].cpu().numpy(), np.zeros(sizes[4]))
    assert np.array_equal(nbs[4].cpu().numpy(), idx)
    cat = F.features_batch(lams, None, concat=True)
    assert cat.shape == (sum(sizes), 48)
    assert torch.equal(cat[:1500, :32], parts[0][:, :32])
    assert F.features_batch([]) == []
    for v in (float("nan"), float("inf")):
        bad = lams[3].clone()
        bad[17, 1] = v
        with pytest.raises(FtcgError) as ei:
            F.features_batch([lams[0], bad])
        assert ei.value.status == 5 and "raster 1" in str(ei.value)
        with pytest.raises(FtcgError) as ei:
            F.features(bad)
        assert ei.value.status == 5


def test_forward_and_grads_vs_oracle(F):
    import torch
    rng = np.random.default_rng(1)
    P = L.init_params(rng)
    P["w4"] = rng.standard_normal(L.HID) * 0.2
    P["b1"] = rng.standard_normal(L.HID) * 0.1
    flat = L.pack(P).astype(np.float32)
    B = 777
    X = bf16(rng.standard_normal((B, L.D_IN)) * 0.7)
    t = rng.standard_normal(B) * 0.5
    Xg = np.zeros((B, 48), np.float32)
    Xg[:, :L.D_IN] = X
    Xt = torch.from_numpy(Xg).to(torch.bfloat16).cuda()
    mlp = F.Mlp(flat)
    alpha = mlp.predict(Xt).cpu().numpy()
    Pr = L.unpack(flat)
    for k in ("W1", "W2", "W3", "w4"):
        Pr[k] = bf16(Pr[k])
    y_ref, cache = L.forward(Pr, X)
    g_ref = L.backward(Pr, cache, y_ref, t)
    l_ref = L.loss(y_ref, t)
    y_m, g_m, l_m = bf16_model(Pr, X, t)
    y_dev = np.log(alpha)
    assert nrel(y_dev, y_ref) <= 4 * nrel(y_m, y_ref) + 1e-5
    assert nrel(y_dev, y_m) < 1e-3
    g, loss = mlp.grads(Xt, dev(t))
    assert abs(loss - l_ref) / l_ref <= 4 * abs(l_m - l_ref) / l_ref + 1e-5
    G = L.unpack(g)
    for k, _ in L.ORDER:
        bar = 4 * nrel(g_m[k], g_ref[k]) + 1e-5
        assert nrel(G[k], g_ref[k]) <= bar, (k, nrel(G[k], g_ref[k]), bar)
        assert nrel(G[k], g_m[k]) < 1e-3, k
    mlp.close()


def test_checkpoint_continuation_is_bitwise(F):
    import torch
    rng = np.random.default_rng(2)
    flat = L.pack(L.init_params(rng)).astype(np.float32)
    X = torch.from_numpy(rng.standard_normal((512, 48)).astype(np.float32)).to(torch.bfloat16).cuda()
    t = dev(rng.standard_normal(512))
    idx = torch.arange(512, dtype=torch.int32, device="cuda")
    a = F.Mlp(flat)
    for _ in range(3):
        a.train_step(X, t, idx, 1e-3)
    st = a.state()
    b = F.Mlp(st["params"])
    b.load_state(st)
    for m in (a, b):
        for _ in range(2):
            m.train_step(X, t, idx, 1e-3)
    sa, sb = a.state(), b.state()
    assert np.array_equal(sa["params"], sb["params"]) and sa["step"] == sb["step"] == 5


def test_adam_steps_vs_oracle(F):
    """Two device Adam steps (ftcg_mlp_train_step, bias corrections at t = 1 and t = 2) against
    mlp_oracle.adam_step given the same gradients (ftcg_mlp_grads at the same parameters and
    batch: the device reductions have a fixed order, so train_step sees these very gradients)
    and the device's own moments before the step.

    Bound, with u = 2^-24 (FP32 unit roundoff): the new moments m = b1 m + (1 - b1) g and
    v = b2 v + (1 - b2) g^2 take at most three rounded operations on constants held within
    u/2 of their FP64 values, so |m - m_ref| <= 4u (|b1 m| + |(1-b1) g|), and one more for g^2
    in v (5u). The update d = lr (m / c1) / (sqrt(v / c2) + eps) adds the divisions by the bias
    corrections, the square root, the addition of eps, the division and the scaling by lr
    (<= 8u, the square root halving the error of v): |d - d_ref| <= 16u |d_ref|. The new
    parameter is rounded once more: |P - P_ref| <= u |P_ref| + 16u |d_ref|. The test allows
    twice these."""
    import torch
    rng = np.random.default_rng(9)
    flat = L.pack(L.init_params(rng)).astype(np.float32)
    B = 700
    X = rng.standard_normal((B, 48)).astype(np.float32)
    X[:, L.D_IN:] = 0
    Xt = torch.from_numpy(X).to(torch.bfloat16).cuda()
    t = dev(rng.standard_normal(B) * 0.5)
    idx = torch.from_numpy(rng.permutation(B).astype(np.int32)).cuda()
    lr, u = 3e-3, 2.0 ** -24
    mlp = F.Mlp(flat)
    st = mlp.state()
    for step in (1, 2):
        g, _ = mlp.grads(Xt, t, idx)
        mlp.train_step(Xt, t, idx, lr)
        new = mlp.state()
        assert new["step"] == step
        P = L.unpack(st["params"])
        G = L.unpack(g)
        state = {"t": step - 1}
        m_old, v_old = L.unpack(st["m"]), L.unpack(st["v"])
        for k, _ in L.ORDER:
            state["m_" + k] = m_old[k].copy()
            state["v_" + k] = v_old[k].copy()
        ref = L.adam_step({k: P[k].copy() for k, _ in L.ORDER}, G, state, lr=lr)
        Pn, mn, vn = L.unpack(new["params"]), L.unpack(new["m"]), L.unpack(new["v"])
        for k, _ in L.ORDER:
            bm = 4 * u * (0.9 * np.abs(m_old[k]) + 0.1 * np.abs(G[k]))
            bv = 5 * u * (0.999 * np.abs(v_old[k]) + 0.001 * G[k] ** 2)
            assert np.all(np.abs(mn[k] - state["m_" + k]) <= 2 * bm + 1e-38), k
            assert np.all(np.abs(vn[k] - state["v_" + k]) <= 2 * bv + 1e-38), k
            d = P[k] - ref[k]
            bp = u * np.abs(ref[k]) + 16 * u * np.abs(d)
            assert np.all(np.abs(Pn[k] - ref[k]) <= 2 * bp + 1e-38), k
        st = new
    mlp.close()


def test_trained_network_gain(F, tmp_path):
    """Train on exact weights of random jittered polar geometries, then grid a held-out ping with
    the predicted weights: its image is closer to the exact-weight oracle image than the
    unweighted one. The weights depend on the local density in cycles, so the training
    geometries span the densities of the held-out one (log-uniform sample counts). The FP64
    oracle network reaches 0.7-2.5% median weight error on such held-out geometries and the
    device-trained one 2.5% (image error 0.39 of the unweighted one); the bars are 5% and one
    half."""
    import torch
    from paper_1706_08575_gb300 import learn
    rng = np.random.default_rng(3)
    geos, Ns = [], []
    for lam, N, kr in sasgen.training_geometries(rng, 24, N_choices=(128, 256),
                                                 M_range=(3000, 12000)):
        geos.append((lam, kr))
        Ns.append(N)
    feats, targ = learn.build_dataset(geos, Ns)
    mlp = F.Mlp(learn.init_params(0))
    hist = learn.train(mlp, feats, targ, steps=8000, batch=8192, lr=3e-3, log_every=2000)
    assert hist[-1][1] < 0.2 * hist[0][1]
    learn.save_checkpoint(tmp_path / "m.npz", mlp)
    m2 = learn.load_checkpoint(tmp_path / "m.npz")
    # held-out ping
    lam, N, kr = sasgen.random_geometry(np.random.default_rng(99), N_choices=(128,),
                                        M_range=(6000, 6000))   # inside the training range
    a_ref, _ = O.weights_brute(lam, N)
    lt = dev(lam)
    fe = F.features(lt, dev(learn.kr_feature(kr)))
    a_nn = m2.predict(fe).cpu().numpy()
    w_err = float(np.median(np.abs(a_nn - a_ref) / a_ref))
    v = rng.standard_normal(lam.shape[0]) + 1j * rng.standard_normal(lam.shape[0])
    ref = O.adjoint(lam, a_ref * v, N, 2.0, 8)
    with F.Plan(lt, N, 2.0, 8) as p:
        p.set_weights(dev(a_nn))
        img_nn = p.adjoint(dev(v.astype(np.complex64))).cpu().numpy()
        p.set_weights(None)
        img_1 = p.adjoint(dev(v.astype(np.complex64))).cpu().numpy()
    e_nn, e_1 = O.rel_l2(img_nn, ref), O.rel_l2(img_1, ref)
    print(f"learned: median weight error {w_err:.2e}, image rel-L2 {e_nn:.2e}; "
          f"unweighted image rel-L2 {e_1:.2e}")
    assert w_err < 0.05
    assert e_nn < 0.5 * e_1
    mlp.close()
    m2.close()
