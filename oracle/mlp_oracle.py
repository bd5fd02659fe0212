"""FP64 CPU oracle of the learned-weight model (test infrastructure only; no product code imports
this module).

The learned part predicts the FTCG diagonal weight of each sample (Eq. difopt at r = 1) from its
local k-space neighbourhood:
  features  x_k = (lambda_{n_1} - lambda_k, ..., lambda_{n_16} - lambda_k, a_k)   (33 values)
            n_1..n_16 the 16 nearest other samples by Euclidean distance in lambda (cycles per
            FOV), ties broken by the smaller index; a_k a per-sample auxiliary scalar (the range
            wavenumber, normalised by the caller);
  network   h1 = gelu(x W1 + b1), h2 = gelu(h1 W2 + b2), h3 = gelu(h2 W3 + b3), y = h3 w4 + b4,
            33 -> 64 -> 64 -> 64 -> 1, predicted alpha = exp(y);
  gelu      the tanh form 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)));
  training  mean squared error of y against log alpha_exact, Adam.
Everything here is plain numpy in float64; the device kernels compute the same functions in BF16
with FP32 accumulation.
"""
from __future__ import annotations

import numpy as np

K_NN = 16
D_IN = 2 * K_NN + 1
HID = 64
_C = np.sqrt(2.0 / np.pi)


def knn_features(lam, aux, k=K_NN):
    """Brute force: for every sample, all squared distances, ordered by (distance, index)."""
    lam = np.asarray(lam, np.float64)
    M = lam.shape[0]
    X = np.empty((M, 2 * k + 1), np.float64)
    idx = np.empty((M, k), np.int64)
    for i in range(M):
        d = lam - lam[i]
        d2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
        d2[i] = np.inf
        order = np.lexsort((np.arange(M), d2))[:k]
        idx[i] = order
        X[i, :2 * k] = d[order].reshape(-1)
        X[i, 2 * k] = aux[i]
    return X, idx


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    u = _C * (z + 0.044715 * z ** 3)
    t = np.tanh(u)
    du = _C * (1.0 + 3 * 0.044715 * z * z)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * du


def init_params(rng):
    def lin(fan_in, fan_out):
        return rng.standard_normal((fan_in, fan_out)) * np.sqrt(2.0 / fan_in)
    return {"W1": lin(D_IN, HID), "b1": np.zeros(HID), "W2": lin(HID, HID), "b2": np.zeros(HID),
            "W3": lin(HID, HID), "b3": np.zeros(HID), "w4": lin(HID, 1)[:, 0] * 0.1,
            "b4": np.zeros(1)}


def forward(P, X):
    z1 = X @ P["W1"] + P["b1"]
    h1 = gelu(z1)
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = gelu(z2)
    z3 = h2 @ P["W3"] + P["b3"]
    h3 = gelu(z3)
    y = h3 @ P["w4"] + P["b4"][0]
    return y, (X, z1, h1, z2, h2, z3, h3)


def loss(y, t):
    return float(np.mean((y - t) ** 2))


def backward(P, cache, y, t):
    """Gradients of the mean squared error with respect to every parameter."""
    X, z1, h1, z2, h2, z3, h3 = cache
    B = y.shape[0]
    dy = 2.0 * (y - t) / B
    g = {"w4": h3.T @ dy, "b4": np.array([dy.sum()])}
    dh3 = np.outer(dy, P["w4"])
    dz3 = dh3 * gelu_grad(z3)
    g["W3"] = h2.T @ dz3
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ P["W3"].T) * gelu_grad(z2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"].T) * gelu_grad(z1)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return g


def adam_step(P, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) with bias correction; state holds m, v and t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P


ORDER = [("W1", (D_IN, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
         ("W3", (HID, HID)), ("b3", (HID,)), ("w4", (HID,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in ORDER)


def unpack(flat):
    """Flat parameter vector (order W1, b1, W2, b2, W3, b3, w4, b4; W as [input][output]) to a
    dict of float64 arrays."""
    flat = np.asarray(flat, np.float64)
    out, o = {}, 0
    for k, shp in ORDER:
        n = int(np.prod(shp))
        out[k] = flat[o:o + n].reshape(shp).copy()
        o += n
    return out


def pack(P):
    return np.concatenate([np.asarray(P[k], np.float64).reshape(-1) for k, _ in ORDER])
