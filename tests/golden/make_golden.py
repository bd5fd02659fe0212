"""Writes ftcg_polar_n32.txt, the stored small case of the weighted adjoint: a jittered polar
raster, two point scatterers, the exact FTCG weights (Eq. difopt at r = 1, by the brute-force
Fejer sums) and the image at 64 pixels by the gridding algorithm (Eq. twodcg, sigma = 2, w = 8)
and by the direct sum. It calls only the FP64 oracle and the input generators.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import sasgen  # noqa: E402
from oracle import ftcg_oracle as O  # noqa: E402

N, SIGMA, W = 32, 2.0, 8
SCATTERERS = [((5, -7), 1.0), ((-9, 4), 0.6)]    # (pixel offset (x, y), amplitude)
OUT = os.path.join(HERE, "ftcg_polar_n32.txt")


def make():
    rng = np.random.default_rng(20170626)
    kx, ky = sasgen.polar_raster(rng, 12, 8, 12.0, theta_jitter_deg=0.02)
    lam0 = sasgen.baseband(kx, ky, 1.0)
    # the field of view chosen so that the sample span fills 80% of the N x N frequency square
    span = max(np.ptp(lam0[:, 0]), np.ptp(lam0[:, 1]))
    lam = lam0 * (0.8 * N / span)
    v = np.zeros(lam.shape[0], np.complex128)
    for (px, py), a in SCATTERERS:
        v += a * np.exp(-2j * np.pi * (lam[:, 0] * px + lam[:, 1] * py) / N)
    alpha, _ = O.weights_brute(lam, N)
    c = alpha * v
    img2 = O.adjoint(lam, c, N, SIGMA, W)
    img1 = O.direct_adjoint(lam, c, N)
    # pixels: each scatterer and its 8 neighbours, then seeded random pixels (64 in all)
    pix = []
    for (px, py), _ in SCATTERERS:
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                pix.append((px + dx, py + dy))
    seen = set(pix)
    while len(pix) < 64:
        p = tuple(int(t) for t in rng.integers(-N // 2, N // 2, 2))
        if p not in seen:
            seen.add(p)
            pix.append(p)
    pix = np.array(pix, np.int64)
    iy, ix = pix[:, 1] + N // 2, pix[:, 0] + N // 2
    return lam, v, alpha, pix, img2[iy, ix], img1[iy, ix]


def write(path=OUT):
    lam, v, alpha, pix, o2, o1 = make()
    f = lambda x: repr(float(x))
    with open(path, "w") as fh:
        fh.write("# Weighted adjoint of a jittered polar raster: exact FTCG weights and image pixels.\n")
        fh.write("# Weights: alpha_k = 1 / sum_j F_N(lambda_j - lambda_k) (Eq. difopt, diagonal D, r = 1).\n")
        fh.write("# Image: I_p = sum_j alpha_j v_j exp(+2 pi i lambda_j . p / N) at pixel p (Eq. twodcg):\n")
        fh.write("#   'o2' by the gridding algorithm (sigma = 2, w = 8, ES window), 'o1' by the direct sum.\n")
        fh.write("# Raster: 12 range wavenumbers x 8 angles over 12 deg, angle jitter 0.02 deg, baseband,\n")
        fh.write("#   scaled to span 80% of N; values: point scatterers at pixel offsets (5, -7), amplitude 1,\n")
        fh.write("#   and (-9, 4), amplitude 0.6. Written by tests/golden/make_golden.py (FP64 oracle).\n")
        fh.write(f"N {N} sigma {SIGMA} w {W} M {lam.shape[0]} pixels {pix.shape[0]}\n")
        fh.write("# samples: lambda_x lambda_y re(v) im(v) alpha\n")
        for j in range(lam.shape[0]):
            fh.write(" ".join(f(t) for t in (lam[j, 0], lam[j, 1], v[j].real, v[j].imag,
                                              alpha[j])) + "\n")
        fh.write("# pixels: p_x p_y re(o2) im(o2) re(o1) im(o1)\n")
        for k in range(pix.shape[0]):
            fh.write(f"{pix[k, 0]} {pix[k, 1]} " + " ".join(
                f(t) for t in (o2[k].real, o2[k].imag, o1[k].real, o1[k].imag)) + "\n")


def read(path=OUT):
    """(meta, lam, v, alpha, pix, o2, o1) of a stored case."""
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    head = rows[0]
    meta = {head[i]: float(head[i + 1]) for i in range(0, len(head), 2)}
    M, P = int(meta["M"]), int(meta["pixels"])
    s = np.array(rows[1:1 + M], np.float64)
    p = np.array(rows[1 + M:1 + M + P], np.float64)
    return (meta, s[:, :2].copy(), s[:, 2] + 1j * s[:, 3], s[:, 4].copy(),
            p[:, :2].astype(np.int64), p[:, 2] + 1j * p[:, 3], p[:, 4] + 1j * p[:, 5])


if __name__ == "__main__":
    write()
    print("wrote", OUT)
