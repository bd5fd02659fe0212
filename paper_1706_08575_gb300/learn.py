"""Training and use of the weight-predicting network (argument marshalling around libftcg).

Labels are the exact FTCG weights of each training geometry (ftcg_weights, FP64 on the device);
features come from ftcg_features; every forward, backward and Adam step runs in the library's
BF16 tensor-core kernels. PyTorch only holds device buffers and draws batch indices.
"""
from __future__ import annotations

import numpy as np

from . import ftcg as F

KR_MID = 4 * np.pi * 115e3 / 1500.0     # range wavenumber at the band centre, rad/m


def kr_feature(kr):
    """The auxiliary input: the range wavenumber relative to the band centre."""
    return np.asarray(kr, np.float64) / KR_MID - 1.0


def init_params(seed=0):
    """He-normal weights, zero biases, packed in the library's order."""
    rng = np.random.default_rng(seed)

    def lin(i, o):
        return rng.standard_normal((i, o)) * np.sqrt(2.0 / i)

    parts = [lin(33, 64), np.zeros(64), lin(64, 64), np.zeros(64), lin(64, 64), np.zeros(64),
             lin(64, 1)[:, 0] * 0.1, np.zeros(1)]
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def build_dataset(geometries, N_of, sigma=2.0, w=8, device="cuda"):
    """Features and log exact weights of a list of (lam (M, 2) numpy, kr (M,) numpy) geometries,
    concatenated on the device. N_of[i] is the image side of geometry i."""
    import torch
    feats, targets = [], []
    for (lam, kr), N in zip(geometries, N_of):
        lt = torch.from_numpy(np.ascontiguousarray(lam)).to(device)
        with F.Plan(lt, N, sigma, w) as p:
            alpha = p.weights()
        aux = torch.from_numpy(kr_feature(kr)).to(device)
        feats.append(F.features(lt, aux))
        targets.append(torch.log(alpha))
    return torch.cat(feats), torch.cat(targets)


def train(mlp, feats, targets, steps, batch=8192, lr=2e-3, lr_end=1e-4, seed=0, log_every=0):
    """Adam on random batches with a cosine learning-rate decay; returns the loss history."""
    import torch
    g = torch.Generator(device=feats.device)
    g.manual_seed(seed)
    n = int(feats.shape[0])
    hist = []
    for s in range(steps):
        lr_s = lr_end + 0.5 * (lr - lr_end) * (1 + np.cos(np.pi * s / max(1, steps - 1)))
        idx = torch.randint(0, n, (batch,), device=feats.device, generator=g, dtype=torch.int32)
        want = bool(log_every) and (s % log_every == 0 or s == steps - 1)
        l = mlp.train_step(feats, targets, idx, lr_s, want_loss=want)
        if want:
            hist.append((s, l))
    return hist


def save_checkpoint(path, mlp):
    st = mlp.state()
    np.savez(path, params=st["params"], m=st["m"], v=st["v"], step=st["step"])


def load_checkpoint(path):
    d = np.load(path)
    mlp = F.Mlp(d["params"])
    mlp.load_state({"params": d["params"], "m": d["m"], "v": d["v"], "step": int(d["step"])})
    return mlp
