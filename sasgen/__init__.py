"""Seeded synthetic SAS inputs: polar k-space rasters, point-scatterer scenes, sample values.

This module is shared by the FP64 oracle and the CUDA path. It holds none of the gridding
method's arithmetic: it only draws geometries and scenes and evaluates the forward model
(the data frame of Eq. (twoddataframe), a sum of point scatterers) to synthesise samples.

Conventions (Sec. IV, Eq. (twoddataframe); sign and units are a reading, the paper fixes none):
  * k-space samples come from the Fourier slice projection theorem on a polar raster (Sec. II):
    kx = kr cos(theta), ky = kr sin(theta) in rad/m.
  * they are base-banded and scaled to cycles per field of view (FOV):
    lambda = (k - k_c) * L / (2 pi), k_c = ((min kx + max kx) / 2, 0), L the FOV side in metres.
  * a scatterer of complex amplitude a at position r (metres, FOV centred on 0) contributes
    a * exp(-2 pi i lambda . r / L) to each sample, so the adjoint peaks at pixel N r / L.
  * acquisition order is range-fastest within angle: j = i_theta * n_kr + i_kr.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 170608575
SOUND_SPEED = 1500.0          # m/s
F_LO, F_HI = 100e3, 130e3     # Hz: the band of every raster below


@dataclasses.dataclass
class Scene:
    pos: np.ndarray    # S x 2 float64, metres, (x, y)
    amp: np.ndarray    # S complex128
    L: float           # FOV side, metres


@dataclasses.dataclass
class Ping:
    lam: np.ndarray            # M x 2 float64, cycles per FOV, (x, y), acquisition order
    N: int
    sigma: float
    w: int
    scene: Scene
    noise_snr_db: float | None
    seed: int
    name: str
    bright_pixels: np.ndarray | None = None   # B x 2 int (px, py) pixel offsets of bright targets
    kr: np.ndarray | None = None              # M range wavenumbers |k| (rad/m)

    @property
    def M(self) -> int:
        return int(self.lam.shape[0])


def polar_raster(rng, n_kr, n_theta, span_deg, kr_scale=1.0, theta_jitter_deg=0.0,
                 f_lo=F_LO, f_hi=F_HI, c=SOUND_SPEED):
    """Polar k-space raster (Sec. II, Sec. V-C 'side-scan-SAS-like' arrangement).

    Range wavenumbers kr = 4 pi f / c uniform over [f_lo, f_hi] (endpoints included), scaled by
    kr_scale (a sound-speed mismatch); aspect angles uniform over [-span/2, span/2] (endpoints
    included) plus independent Gaussian jitter per sample. Returns kx, ky in rad/m (M,)."""
    kr = np.linspace(4 * np.pi * f_lo / c, 4 * np.pi * f_hi / c, n_kr) * kr_scale
    th = np.deg2rad(np.linspace(-span_deg / 2, span_deg / 2, n_theta))
    TH, KR = np.meshgrid(th, kr, indexing="ij")           # angle-major, range-fastest
    TH = TH.reshape(-1).copy()
    KR = KR.reshape(-1)
    if theta_jitter_deg > 0:
        TH += np.deg2rad(theta_jitter_deg) * rng.standard_normal(TH.shape[0])
    return KR * np.cos(TH), KR * np.sin(TH)


def baseband(kx, ky, L):
    """lambda = (k - k_c) L / (2 pi), k_c = ((min kx + max kx)/2, 0)."""
    kc = 0.5 * (kx.min() + kx.max())
    return np.stack([(kx - kc) * L / (2 * np.pi), ky * L / (2 * np.pi)], axis=1)


def speckle_scene(rng, n_speckle, n_bright, L, N, bright_amp=10.0, extent=0.8):
    """Rayleigh-amplitude, uniform-phase speckle over the central `extent` of the FOV plus bright
    targets (|a| = bright_amp, random phase) centred on pixels. Returns (Scene, bright pixels)."""
    pos = (rng.random((n_speckle, 2)) - 0.5) * extent * L
    # Rayleigh amplitude with E|a|^2 = 1: |a| = sqrt(-log U)
    mag = np.sqrt(-np.log(1.0 - rng.random(n_speckle)))
    amp = mag * np.exp(2j * np.pi * rng.random(n_speckle))
    half = int(0.4 * N)
    bp = rng.integers(-half, half, size=(n_bright, 2))
    bpos = bp.astype(np.float64) * (L / N)
    bamp = bright_amp * np.exp(2j * np.pi * rng.random(n_bright))
    return Scene(np.concatenate([pos, bpos]), np.concatenate([amp, bamp]), L), bp


def point_scene(rng, n_points, L, half_extent=1.0):
    pos = (rng.random((n_points, 2)) * 2 - 1) * half_extent
    amp = np.exp(2j * np.pi * rng.random(n_points))
    return Scene(pos, amp, L)


def sample_values(lam, scene, chunk=1 << 16, device=None):
    """Exact Fourier sum of the scene's point scatterers at every sample (FP64, complex128).

    v_j = sum_s a_s exp(-2 pi i lambda_j . r_s / L). With device=None it runs in numpy on the
    host; with a torch device (e.g. 'cuda') it runs in plain FP64 PyTorch there and returns a
    numpy array on the host."""
    r = scene.pos / scene.L
    if device is None:
        out = np.empty(lam.shape[0], np.complex128)
        for s in range(0, lam.shape[0], chunk):
            ph = -2 * np.pi * (lam[s:s + chunk] @ r.T)
            out[s:s + chunk] = np.exp(1j * ph) @ scene.amp
        return out
    import torch
    lt = torch.as_tensor(lam, dtype=torch.float64, device=device)
    rt = torch.as_tensor(r, dtype=torch.float64, device=device)
    at = torch.as_tensor(scene.amp, dtype=torch.complex128, device=device)
    out = torch.empty(lam.shape[0], dtype=torch.complex128, device=device)
    step = max(1, (1 << 26) // max(1, r.shape[0]))
    for s in range(0, lam.shape[0], step):
        ph = (-2 * math.pi) * (lt[s:s + step] @ rt.T)
        out[s:s + step] = torch.polar(torch.ones_like(ph), ph) @ at
    return out.cpu().numpy()


def add_noise(rng, v, snr_db):
    """Circular complex Gaussian noise: SNR = mean|v|^2 / noise variance (split over re/im)."""
    var = np.mean(np.abs(v) ** 2) / (10 ** (snr_db / 10))
    return v + np.sqrt(var / 2) * (rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape))


# --------------------------------------------------------------------------------------------
# The workloads. Each is a full recipe: raster, scene, N, sigma, w.
# --------------------------------------------------------------------------------------------

def tiny(seed=BASE_SEED + 0):
    """64 kr x 64 angles over [-10, 10] deg; 5 unit points in a 2 m x 2 m patch; 30 dB SNR;
    N = 64, sigma = 2, w = 6; FOV L = 2 m (the data span 84 x 120 cycles wraps, period N)."""
    rng = np.random.default_rng(seed)
    kx, ky = polar_raster(rng, 64, 64, 20.0)
    L = 2.0
    lam = baseband(kx, ky, L)
    scene = point_scene(rng, 5, L, half_extent=1.0)
    return Ping(lam, 64, 2.0, 6, scene, 30.0, seed, "tiny-4096", kr=np.hypot(kx, ky))


def large_ping(seed=BASE_SEED + 1, n_kr=2048, n_theta=1024, N=1024, L=10.0, w=8):
    """2048 kr x 1024 angles over [-15, 15] deg; kr x 1.01 (1% sound-speed mismatch); angle
    jitter N(0, 0.02 deg); 2000 speckle + 20 bright (+20 dB) targets; N = 1024, sigma = 2, w = 8."""
    rng = np.random.default_rng(seed)
    kx, ky = polar_raster(rng, n_kr, n_theta, 30.0, kr_scale=1.01, theta_jitter_deg=0.02)
    lam = baseband(kx, ky, L)
    scene, bp = speckle_scene(rng, 2000, 20, L, N)
    return Ping(lam, N, 2.0, w, scene, None, seed, f"large-ping-{n_kr * n_theta}", bp,
                np.hypot(kx, ky))


def precision_sweep(seed=BASE_SEED + 2):
    """The large-ping geometry with 2048 x 2048 samples at N = 2048 (FOV 20 m)."""
    p = large_ping(seed, n_kr=2048, n_theta=2048, N=2048, L=20.0)
    p.name = "precision-4194304"
    return p


def _batch_ping_draws(rng):
    """The first draws of a batch ping: (n_kr, n_theta, span, kr error, N)."""
    M = int(rng.integers(20_000, 400_001))
    span = float(rng.uniform(5.0, 20.0))
    e = float(rng.uniform(-0.02, 0.02))
    N = int(rng.choice([256, 512, 1024]))
    n_th = max(2, int(round(math.sqrt(M / 2))))
    n_kr = max(2, int(round(M / n_th)))
    return n_kr, n_th, span, e, N


def batch_ping_size(b, seed_base=BASE_SEED + 3):
    """(M, N) of batch ping b without drawing its raster (the same draws as batch_ping)."""
    n_kr, n_th, _, _, N = _batch_ping_draws(np.random.default_rng(seed_base + 1000 * b))
    return n_kr * n_th, N


def batch_ping(b, seed_base=BASE_SEED + 3):
    """Ping b of the uneven batch: M ~ U{20k..400k}, span ~ U[5, 20] deg, kr x (1+e) with
    e ~ U[-2%, 2%], angle jitter N(0, 0.02 deg), N ~ {256, 512, 1024}; 500 speckle + 5 bright;
    sigma = 2, w = 8; the FOV is sized so that the lambda span fills 90% of N."""
    seed = seed_base + 1000 * b
    rng = np.random.default_rng(seed)
    n_kr, n_th, span, e, N = _batch_ping_draws(rng)
    kx, ky = polar_raster(rng, n_kr, n_th, span, kr_scale=1 + e, theta_jitter_deg=0.02)
    kspan = max(kx.max() - kx.min(), ky.max() - ky.min())
    L = 0.9 * 2 * np.pi * N / kspan
    lam = baseband(kx, ky, L)
    scene, bp = speckle_scene(rng, 500, 5, L, N)
    return Ping(lam, N, 2.0, 8, scene, None, seed, f"batch-ping-{b}", bp, np.hypot(kx, ky))


def random_geometry(rng, N_choices=(256, 512), M_range=(2_000, 20_000), log_uniform=False):
    """A random jittered polar geometry for weight learning: angle jitter sd ~ U[0, 0.05] deg,
    sound-speed error ~ U[-3%, 3%], span ~ U[5, 20] deg, N from N_choices, M uniform (or
    log-uniform) over M_range; the FOV is sized so that the raster fills 90% of N."""
    if log_uniform:
        M = int(round(np.exp(rng.uniform(np.log(M_range[0]), np.log(M_range[1])))))
    else:
        M = int(rng.integers(M_range[0], M_range[1] + 1))
    span = float(rng.uniform(5.0, 20.0))
    e = float(rng.uniform(-0.03, 0.03))
    jit = float(rng.uniform(0.0, 0.05))
    N = int(rng.choice(list(N_choices)))
    n_th = max(2, int(round(math.sqrt(M / 2))))
    n_kr = max(2, int(round(M / n_th)))
    kx, ky = polar_raster(rng, n_kr, n_th, span, kr_scale=1 + e, theta_jitter_deg=jit)
    kspan = max(kx.max() - kx.min(), ky.max() - ky.min())
    L = 0.9 * 2 * np.pi * N / kspan
    lam = baseband(kx, ky, L)
    kr = np.hypot(kx, ky)
    return lam, N, kr


def training_geometries(rng, n, N_choices=(128, 256, 512), M_range=(5_000, 60_000)):
    """Geometries for learning the weights. The weights depend on the local sample density in
    cycles per FOV, not on N, so small images with log-uniform sample counts span the densities
    of the uneven batch (about 0.02 to 9 samples per square cycle). Returns [(lam, N, kr)]."""
    return [random_geometry(rng, N_choices, M_range, log_uniform=True) for _ in range(n)]


def values_for(ping: Ping, device=None):
    """Sample values of a ping (complex128), noise included when the recipe has some."""
    v = sample_values(ping.lam, ping.scene, device=device)
    if ping.noise_snr_db is not None:
        rng = np.random.default_rng(ping.seed + 7)
        v = add_noise(rng, v, ping.noise_snr_db)
    return v


def random_case(seed, M, N, sigma=2.0, w=8, spread=None):
    """Generic random samples for edge-case tests: lambda uniform over a square of side `spread`
    cycles (default N, i.e. one period) and unit-variance complex values."""
    rng = np.random.default_rng(seed)
    s = N if spread is None else spread
    lam = (rng.random((M, 2)) - 0.5) * s
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    return lam, v


# ---------------------------------------------------------------------------------------------
# The paper's small rasters (Sec. V) and its test function
# ---------------------------------------------------------------------------------------------

def noisy_grid(seed=BASE_SEED + 21, n=30):
    """lambda_n in [n1 - 1/4, n1 + 1/4] x [n2 - 1/4, n2 + 1/4] for n in {-n/2 .. n/2 - 1}^2
    (uniform jitter, Sec. V-A): n^2 samples (900 for n = 30), acquisition order n1 fastest."""
    rng = np.random.default_rng(seed)
    g = np.arange(-(n // 2), n - n // 2, dtype=np.float64)
    X, Y = np.meshgrid(g, g)
    lam = np.stack([X.ravel(), Y.ravel()], 1)
    return lam + rng.uniform(-0.25, 0.25, lam.shape)


def asterisk(seed=BASE_SEED + 22, lines=8, per_line=28, extent=14.0, jitter=0.05):
    """Diameters through the origin at angles k pi / lines (Sec. V-B), per_line samples on each
    (radii uniform in [-extent, extent] without 0) plus the origin once, with a small radial
    jitter: lines * per_line + 1 samples (225 by default), acquisition order line by line."""
    rng = np.random.default_rng(seed)
    r = np.linspace(-extent, extent, per_line + 1)     # odd count: the middle one is 0
    r = np.delete(r, per_line // 2)
    pts = [np.zeros((1, 2))]
    for k in range(lines):
        th = np.pi * k / lines
        rr = r + rng.uniform(-jitter, jitter, r.shape)
        pts.append(np.stack([rr * np.cos(th), rr * np.sin(th)], 1))
    return np.concatenate(pts)


def sas_like(seed=BASE_SEED + 23, n_kr=40, n_theta=25, span_deg=30.0, extent=14.0):
    """A side-scan-SAS-like polar wedge (Sec. V-C): n_kr range wavenumbers x n_theta jittered
    angles of the 100-130 kHz band, base-banded and scaled so that the wedge spans about
    [-extent, extent] cycles: n_kr * n_theta samples (1000 by default), range fastest."""
    rng = np.random.default_rng(seed)
    kx, ky = polar_raster(rng, n_kr, n_theta, span_deg, theta_jitter_deg=0.05)
    kspan = max(kx.max() - kx.min(), ky.max() - ky.min())
    return baseband(kx, ky, 2 * np.pi * 2 * extent / kspan)


def jittered_1d(seed, n):
    """The 1-D raster lambda_k in [k - 1/4, k + 1/4], k = -n..n (2n + 1 samples, Sec. III-C and
    Sec. V-A), embedded in 2-D with lambda_y = 0."""
    rng = np.random.default_rng(seed)
    k = np.arange(-n, n + 1, dtype=np.float64)
    return np.stack([k + rng.uniform(-0.25, 0.25, k.shape), np.zeros_like(k)], 1)


def _sine_ft(a, lam):
    """int_0^1 sin(2 pi a x) exp(-2 pi i lam x) dx for an integer a, then shifted to the centred
    field of view [-1/2, 1/2) (a factor exp(i pi lam))."""
    lam = np.asarray(lam, np.float64)

    def E(u):       # int_0^1 exp(2 pi i u x) dx
        small = np.abs(u) < 1e-12
        us = np.where(small, 1.0, u)
        return np.where(small, 1.0, (np.exp(2j * np.pi * us) - 1.0) / (2j * np.pi * us))

    # sin(2 pi a x) = (exp(2 pi i a x) - exp(-2 pi i a x)) / 2i
    return (E(a - lam) - E(-a - lam)) / 2j * np.exp(1j * np.pi * lam)


def test_function_values(lam):
    """Fourier data of the paper's test function f(x) = sin(4 pi x1) sin(2 pi x2) on [0, 1]^2
    (Eq. eq2), on the centred field of view: v(lambda) = F_2(lambda_x) F_1(lambda_y)."""
    lam = np.asarray(lam, np.float64)
    return _sine_ft(2, lam[:, 0]) * _sine_ft(1, lam[:, 1])


def test_function_image(N):
    """f on the N x N pixel grid of the centred field of view, x = p / N + 1/2, indexed
    [p_y + N/2, p_x + N/2]."""
    x = (np.arange(-(N // 2), N - N // 2) / N) + 0.5
    return np.multiply.outer(np.sin(2 * np.pi * x), np.sin(4 * np.pi * x)).astype(np.complex128)


def test_function_1d_values(lam):
    """Fourier data of f(x) = sin(4 pi x) on [0, 1] at lam[:, 0] (the 1-D experiment)."""
    return _sine_ft(2, np.asarray(lam, np.float64)[:, 0])
