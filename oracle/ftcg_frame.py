"""FP64 CPU oracle for the frame approximation computed iteratively, with the FTCG weights as
the row weighting (Sec. III-B, Sec. V).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this module: only the tests do.
It shares no code with the CUDA library; plain numpy in float64 / complex128.

The frame approximation reconstructs with the dual frame, which for N x N pixel coefficients
means the minimum-norm least-squares image x = E^+ v of the data frame E_jp =
exp(-2 pi i lambda_j.p / N) (reading R1). Forming E^+ costs O(M N^2) memory and more, so it is
computed here by CGLS (conjugate gradients on the normal equations, Hestenes-Stiefel form as in
Bjorck, Numerical Methods for Least Squares Problems, 1996), which needs only E and E^H: the
direct sums, or the gridded operators that the library also has. Row weights w_j (for example
the FTCG weights alpha_j) turn the problem into min || W^(1/2) (E x - v) ||; started from zero,
the first iterate is a multiple of E^H W v, the FTCG image, and for data that E can fit exactly
the weighted and unweighted iterations reach the same minimum-norm image.
"""
from __future__ import annotations

import numpy as np

from . import ftcg_oracle as O


def operators(lam, N, sigma=2.0, w=8, gridded=False):
    """(E, E^H) as functions: the direct sums, or the gridding algorithm's forward and adjoint
    (O2) at oversampling sigma and width w."""
    if gridded:
        return (lambda x: O.forward(lam, x, N, sigma, w),
                lambda c: O.adjoint(lam, c, N, sigma, w))
    return (lambda x: O.direct_forward(lam, x, N),
            lambda c: O.direct_adjoint(lam, c, N))


def cgls(lam, v, N, weights=None, iters=100, sigma=2.0, w=8, gridded=False, tol=0.0):
    """CGLS for min || W^(1/2) (E x - v) ||_2 from x = 0. Returns (x, history), x an N x N
    image indexed [p_y + N/2, p_x + N/2] and history the list of iterates' normal-equation
    residual norms || E^H W (v - E x) ||."""
    E, EH = operators(lam, N, sigma, w, gridded)
    v = np.asarray(v, np.complex128)
    sw = np.ones(v.shape[0]) if weights is None else np.sqrt(np.asarray(weights, np.float64))
    A = lambda x: sw * E(x)
    AH = lambda r: EH(sw * r)
    x = np.zeros((N, N), np.complex128)
    r = sw * v
    s = AH(r)
    p = s.copy()
    gamma = float(np.vdot(s, s).real)
    hist = [np.sqrt(gamma)]
    for _ in range(iters):
        if gamma <= tol * tol:
            break
        q = A(p)
        qq = float(np.vdot(q, q).real)
        if qq == 0.0:
            break
        a = gamma / qq
        x = x + a * p
        r = r - a * q
        s = AH(r)
        g_new = float(np.vdot(s, s).real)
        p = s + (g_new / gamma) * p
        gamma = g_new
        hist.append(np.sqrt(gamma))
    return x, hist
