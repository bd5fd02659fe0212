#!/usr/bin/env python
"""Benchmark of the FTCG weighted adjoint on one GB300 (prints ONE JSON line on rank 0).

Workload: one large polar ping per GPU (2048 range wavenumbers x 1024 jittered angles =
2,097,152 samples, 1% sound-speed mismatch, 2000 speckle + 20 bright scatterers), N = 1024,
sigma = 2, w = 8, exact FTCG weights installed. A step is one weighted adjoint of the ping (spread
with the weights, inverse FFT, window division + crop) with the plan and weights built once per
geometry; `per_ping` times the plan and the weights too. Inputs are resident in HBM; L2 is
flushed (a 256 MB write) before every timed step, outside its events.

--impl reference times the FP64 CPU oracle on the host cores (a spawned process pool over sample
slices) for the same workload and metric.
Under torchrun (N > 1) the pings are the independent units: rank r grids its own ping (seed
170608576 + 100000 r), with no collective on the data path; only the timing is reduced (max
over ranks) and `value` counts the samples of all ranks (weak scaling). The 512-ping batch extra
is split across ranks by work (shard_pings).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "non-uniform samples gridded/sec on 1 GB300 (+% HBM roofline) at rel-L2 err vs FP64"
E2E_PINGS = 4     # distinct pings fed round robin in the pipelined end-to-end measurement
UNIT = "samples/s"
WORKLOAD = ("large ping per GPU (rank r: seed 170608576 + 100000 r): 2048 kr x 1024 theta polar "
            "(M=2097152), kr x1.01, theta jitter 0.02 deg, 2000 speckle + 20 bright, N=1024, "
            "sigma=2, w=8, exact FTCG weights")
L2_NOTE = ("GPU arm: L2 flushed (a write of >= 2 x L2, at least 256 MiB) before every timed step; "
           "warm_l2 repeats the step without the flush. CPU oracle arm: host memory, no flush")


def headline_config(world):
    """The workload's config, identical on both arms."""
    return {"workload": WORKLOAD, "M": 2097152, "N": 1024, "sigma": 2.0, "w": 8, "G": 2048,
            "l2": L2_NOTE,
            "parallelism": ("1 GPU" if world == 1 else
                            f"{world} GPUs, one independent ping per rank, no collective")}


def rank_ping(rank):
    import sasgen
    return sasgen.large_ping(seed=sasgen.BASE_SEED + 1 + 100_000 * rank)


# ---------------------------------------------------------------------------------------------
# rank plumbing (tested with gloo on CPU)
# ---------------------------------------------------------------------------------------------
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(value, device=None):
    """Max of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, device=None):
    """Sum of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def shard_pings(costs, world):
    """Split independent pings across ranks by work: greedy largest-first, each ping to the rank
    with the least work so far (ties to the lower rank). costs[i] = M_i + G_i^2, the samples
    spread plus the grid cells stored and transformed. Every rank computes the same split from
    the same costs; returns one ascending index list per rank. As any such list schedule, the
    largest rank load is at most the mean load plus one ping's cost."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += costs[i]
        parts[r].append(i)
    return [sorted(p) for p in parts]


def batch_costs(n_pings):
    """costs of the uneven batch recipe's pings (sizes only, no raster is drawn)."""
    import sasgen
    out = []
    for b in range(n_pings):
        M, N = sasgen.batch_ping_size(b)
        out.append(M + (2 * N) ** 2)
    return out


# ---------------------------------------------------------------------------------------------
# clocks: NVML read-only queries (SM clock, max SM clock, clock event reasons) sampled in a thread
# ---------------------------------------------------------------------------------------------
_REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
            0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
            0x100: "display_clock_setting"}


class ClockSampler:
    def __init__(self, index=0, period_s=0.002):
        self.ok = False
        self.samples = []
        self.period = period_s
        try:
            self.nv = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nv.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            bus = None
            try:
                import torch
                bus = getattr(torch.cuda.get_device_properties(index), "pci_bus_id", None)
            except Exception:
                bus = None
            found = False
            if isinstance(bus, str) and bus:
                found = self.nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(),
                                                                 ctypes.byref(self.h)) == 0
            if not found and self.nv.nvmlDeviceGetHandleByIndex_v2(index,
                                                                   ctypes.byref(self.h)) != 0:
                return
            mx = ctypes.c_uint()
            self.max_mhz = None
            if self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = int(mx.value)
            self.ok = True
        except OSError:
            pass

    def _one(self):
        mhz = ctypes.c_uint()
        reasons = ctypes.c_ulonglong()
        self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(mhz))
        f = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
        f(self.h, ctypes.byref(reasons))
        self.samples.append((int(mhz.value), int(reasons.value)))

    def _loop(self):
        while not self._stop.is_set():
            self._one()
            time.sleep(self.period)

    def start(self):
        if not self.ok:
            return
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._loop, daemon=True)
        self._t.start()

    def stop(self):
        if not self.ok:
            return None
        self._stop.set()
        self._t.join()
        if not self.samples:
            self._one()
        mhz = [m for m, _ in self.samples]
        bits = 0
        for _, r in self.samples:
            bits |= r
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": self.max_mhz,
                "reasons": [n for b, n in _REASONS.items() if bits & b and n != "gpu_idle"],
                "samples": len(mhz)}


# ---------------------------------------------------------------------------------------------
# the CPU oracle leg: oracle/ftcg_oracle.py as it stands, on the host cores
# ---------------------------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_spread_part(args):
    """One worker's share of the oracle's spreading sum: the samples of one slice."""
    lam, c, N, sigma, w = args
    from oracle import ftcg_oracle as O
    return O.spread(lam, c, N, sigma, w)


def _oracle_adjoint_whole(args):
    """One worker's whole oracle adjoint of one raster (pings are independent units)."""
    lam, c, N, sigma, w = args
    from oracle import ftcg_oracle as O
    return O.adjoint(lam, c, N, sigma, w)


def _pool_ready(_):
    import numpy  # noqa: F401
    from oracle import ftcg_oracle  # noqa: F401
    return 0


class OracleRunner:
    """The FP64 oracle's adjoint (O.adjoint) with its spreading sum split over contiguous sample
    slices in a spawned process pool (one process per core), the per-slice grids summed, then the
    oracle's inverse FFT, crop and window division in this process. procs = 1 runs the oracle
    unchanged in this process."""

    def __init__(self, procs):
        self.procs = max(1, int(procs))
        self.pool = None
        if self.procs > 1:
            import multiprocessing as mp
            self.pool = mp.get_context("spawn").Pool(self.procs)
            self.pool.map(_pool_ready, range(self.procs))     # start-up outside any timing

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None

    def spread(self, lam, c, N, sigma, w):
        from oracle import ftcg_oracle as O
        if self.pool is None:
            return O.spread(lam, c, N, sigma, w)
        M = lam.shape[0]
        cuts = [M * k // self.procs for k in range(self.procs + 1)]
        parts = [(lam[a:b], c[a:b], N, sigma, w) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        grids = self.pool.map(_oracle_spread_part, parts)
        g = grids[0]
        for x in grids[1:]:
            g += x
        return g

    def adjoint_many(self, items):
        """Whole oracle adjoints of independent rasters [(lam, c, N, sigma, w)], one per worker
        at a time; returns (images, seconds)."""
        from oracle import ftcg_oracle as O
        t0 = time.perf_counter()
        if self.pool is None:
            imgs = [O.adjoint(*it) for it in items]
        else:
            imgs = self.pool.map(_oracle_adjoint_whole, items, chunksize=1)
        return imgs, time.perf_counter() - t0

    def adjoint(self, lam, c, N, sigma, w):
        """(image, spread seconds, FFT + crop + window division seconds)."""
        import numpy as np

        from oracle import ftcg_oracle as O
        t0 = time.perf_counter()
        g = self.spread(lam, c, N, sigma, w)
        t1 = time.perf_counter()
        G = g.shape[0]
        h = np.fft.ifft2(g) * (G * G)
        q = np.mod(O.pixel_range(N), G)
        r = O.deapod_factors(N, sigma, w)
        img = h[np.ix_(q, q)] * r[:, None] * r[None, :]
        t2 = time.perf_counter()
        return img, t1 - t0, t2 - t1


def oracle_rate(runner, lam, c, N, sigma, w, budget_s, min_m=4096):
    """Samples/s of the oracle's adjoint on one raster. The whole raster when it fits the budget,
    else a contiguous slice of m samples (acquisition order) charged m/M of one full-size inverse
    FFT, crop and window division. Returns (value, description)."""
    M = lam.shape[0]
    _, ts, tr = runner.adjoint(lam[:min(M, min_m)], c[:min(M, min_m)], N, sigma, w)  # warm-up
    m0 = min(M, max(min_m, M // 16))
    _, ts0, tr = runner.adjoint(lam[:m0], c[:m0], N, sigma, w)
    per_sample = ts0 / m0
    if per_sample * M + tr <= budget_s:
        _, ts, tr = runner.adjoint(lam, c, N, sigma, w)
        return M / (ts + tr), f"the whole raster ({M} samples; spread {ts:.2f} s, FFT etc. {tr:.2f} s)"
    m = int(min(M, max(m0, (budget_s - tr) / per_sample)))
    _, ts, tr = runner.adjoint(lam[:m], c[:m], N, sigma, w)
    sec = ts + tr * m / M
    return m / sec, (f"the spread of the first {m} of {M} samples ({ts:.2f} s) + {m}/{M} of one "
                     f"full-size inverse FFT, crop and window division ({tr:.2f} s per pass)")


def cpu_baselines(p, v, alpha, budget_s=12.0, extra=True):
    """The oracle as it stands on the host cores: one process, and one process per core, on the
    large ping and (extra) on the tiny raster, the precision raster and 8 pings of the batch."""
    import numpy as np

    import sasgen
    cores = host_cores()
    one, allc = OracleRunner(1), OracleRunner(cores)
    out = {}
    try:
        c = alpha * v.astype(np.complex128)
        v1, d1 = oracle_rate(one, p.lam, c, p.N, p.sigma, p.w, budget_s)
        va, da = oracle_rate(allc, p.lam, c, p.N, p.sigma, p.w, 4 * budget_s)
        out["large"] = {"one_core": {"value": v1, "sample": d1},
                        "all_cores": {"value": va, "sample": da}}
        if extra:
            rng = np.random.default_rng(9)
            tiny = sasgen.tiny()
            ct = sasgen.values_for(tiny)
            out["tiny"] = {k: {"value": r(tiny.lam, ct, tiny.N, tiny.sigma, tiny.w)[0]}
                           for k, r in (("one_core", lambda *a: oracle_rate(one, *a, 2.0)),
                                        ("all_cores", lambda *a: oracle_rate(allc, *a, 2.0)))}
            ps = sasgen.precision_sweep()
            cp = rng.standard_normal(ps.M) + 1j * rng.standard_normal(ps.M)
            v1, d1 = oracle_rate(one, ps.lam, cp, ps.N, ps.sigma, ps.w, budget_s)
            va, da = oracle_rate(allc, ps.lam, cp, ps.N, ps.sigma, ps.w, 4 * budget_s)
            out["precision"] = {"one_core": {"value": v1, "sample": d1},
                                "all_cores": {"value": va, "sample": da}}
            nb = max(8, host_cores())
            pings = [sasgen.batch_ping(b) for b in range(nb)]
            tot = sum(q.M for q in pings)
            items = [(q.lam, rng.standard_normal(q.M) + 1j * rng.standard_normal(q.M), q.N, 2.0,
                      8) for q in pings]
            for key, runner in (("one_core", one), ("all_cores", allc)):
                _, t = runner.adjoint_many(items)
                out.setdefault("batch_pings", {})[key] = {
                    "value": tot / t,
                    "sample": f"pings 0-{nb - 1} of the batch recipe ({tot} samples), whole, "
                              + ("one process" if key == "one_core" else "one ping per process")}
    finally:
        one.close()
        allc.close()
    large = out["large"]
    return {"value": large["all_cores"]["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "numpy FP64 oracle, one spawned process per core over sample slices: " +
                      large["all_cores"]["sample"],
            "one_core": dict(large["one_core"], cores=1), "configs": out}


def run_reference(args):
    import numpy as np

    import sasgen
    rank, world, _ = dist_env()
    if rank != 0:
        return
    p = rank_ping(0)
    # the oracle's cost does not depend on the values: a seeded stand-in of the same shape (the
    # values by the direct sum on the host would take hours at this size)
    rng = np.random.default_rng(p.seed)
    c = rng.standard_normal(p.M) + 1j * rng.standard_normal(p.M)
    cores = host_cores()
    runner = OracleRunner(cores)
    try:
        # the whole ping per step when the run fits a few minutes, else a slice per step
        _, ts0, tr = runner.adjoint(p.lam[:p.M // 16], c[:p.M // 16], p.N, p.sigma, p.w)
        per_sample = ts0 / (p.M // 16)
        per_step = max(0.2, 150.0 / max(1, args.steps + args.warmup))
        m = int(min(p.M, max(p.M // 16, (per_step - tr) / per_sample)))
        times = []
        for i in range(args.warmup + args.steps):
            off = (i * m) % max(1, p.M - m + 1)
            _, ts, tr = runner.adjoint(p.lam[off:off + m], c[off:off + m], p.N, p.sigma, p.w)
            if i >= args.warmup:
                times.append(ts + tr * m / p.M)
    finally:
        runner.close()
    tot = sum(times)
    value = m * len(times) / tot
    sample = (f"numpy FP64 oracle, {cores} spawned processes over sample slices; each step spreads "
              f"{m} of the ping's {p.M} samples and is charged {m}/{p.M} of one full 2048^2 "
              f"inverse FFT + crop + window division ({tr:.2f} s per pass)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": headline_config(args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# the GPU leg
# ---------------------------------------------------------------------------------------------
def learned_vs_plain(device, large=None, n_pings=64, train_geos=60, train_steps=8000, seed=5):
    """Pings of the uneven batch recipe, per-ping end to end (geometry changes every ping):
    plain  = per ping: plan, exact FP64 FTCG weights, FP32 adjoint;
    learned + batched = one batched plan, kNN features of all pings in one request, one MLP pass
    over all their samples, one batched adjoint.
    The network is trained here on exact weights of random jittered polar geometries (about 1M
    samples). `large` = (ping, lam, values) also evaluates the large ping."""
    import numpy as np
    import torch

    import paper_1706_08575_gb300 as F
    import sasgen
    from paper_1706_08575_gb300 import learn

    rng = np.random.default_rng(seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    geos, Ns = [], []
    for lam, N, kr in sasgen.training_geometries(rng, train_geos):
        geos.append((lam, kr))
        Ns.append(N)
    feats, targ = learn.build_dataset(geos, Ns)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    mlp = F.Mlp(learn.init_params(0))
    t0 = time.perf_counter()
    hist = learn.train(mlp, feats, targ, steps=train_steps, batch=8192, lr=3e-3, log_every=2000)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del feats, targ

    pings = [sasgen.batch_ping(b) for b in range(n_pings)]
    lams = [torch.from_numpy(p.lam).to(device) for p in pings]
    auxs = [torch.from_numpy(learn.kr_feature(p.kr)).to(device) for p in pings]
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    vals = [torch.randn(p.M, dtype=torch.complex64, device=device, generator=g) for p in pings]
    M_tot = sum(p.M for p in pings)
    # warm the kernels, the autotuner's choices for every ping class (single-ping and batched) and
    # the lag transforms' cuFFT plans of every ping's weights in both arms, so that neither arm
    # times first-use work
    for lam, p, v in zip(lams, pings, vals):
        with F.Plan(lam, p.N, 2.0, 8) as pl:
            pl.weights()
            pl.adjoint(v)
    with F.Batch(lams, [p.N for p in pings], 2.0, 8) as b:
        b.weights()
        b.weights()
    # plain: one ping after another
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_imgs = []
    for lam, v, p in zip(lams, vals, pings):
        with F.Plan(lam, p.N, 2.0, 8) as pl:
            pl.weights()
            plain_imgs.append(pl.adjoint(v))
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    # learned + batched
    t0 = time.perf_counter()
    with F.Batch(lams, [p.N for p in pings], 2.0, 8) as b:
        # features of all pings in one request, one network pass over all their rows
        alpha = mlp.predict(F.features_batch(lams, auxs, concat=True))
        b.set_weights(list(torch.split(alpha, [p.M for p in pings])))
        imgs = b.adjoint(vals)
        torch.cuda.synchronize()
        t_learned = time.perf_counter() - t0
        # the same batch, adjoint only, replayed from a CUDA graph
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            gi = b.capture(vals)
            s.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(5):
                b.launch()
            e1.record(s)
            s.synchronize()
            t_graph = e0.elapsed_time(e1) / 5e3
        errs = [float(torch.linalg.vector_norm(a - r) / torch.linalg.vector_norm(r))
                for a, r in zip(imgs, plain_imgs)]
        tiles, entries, _ = b.info()
    # learned + batched with the exact judge (K = 256 exact sums per ping; calibrated predictions
    # kept where the estimated error is within 5e-4, the exact weights computed otherwise)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with F.Batch(lams, [p.N for p in pings], 2.0, 8) as b:
        alpha = mlp.predict(F.features_batch(lams, auxs, concat=True))
        verdict = b.judge_weights(list(torch.split(alpha, [p.M for p in pings])), K=256,
                                  max_rel_err=5e-4)
        jimgs = b.adjoint(vals)
        torch.cuda.synchronize()
        t_judged = time.perf_counter() - t0
        jerrs = [float(torch.linalg.vector_norm(a - r) / torch.linalg.vector_norm(r))
                 for a, r in zip(jimgs, plain_imgs)]
    accepted = sum(1 for ok, _ in verdict if ok)
    est = [st[1] for _, st in verdict]
    large_eval = None
    if large is not None:
        p, lam, v = large
        with F.Plan(lam, p.N, p.sigma, p.w) as pl:
            a_ex = pl.weights()
            img_ex = pl.adjoint(v).clone()
            aux = torch.from_numpy(learn.kr_feature(p.kr)).to(device)   # an input, like lambda
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            a_nn = mlp.predict(F.features(lam, aux))
            pl.set_weights(a_nn)
            img_nn = pl.adjoint(v)
            torch.cuda.synchronize()
            t_nn = time.perf_counter() - t0
            pl.set_weights(None)
            img_1 = pl.adjoint(v)
            rel = lambda a, r: float(torch.linalg.vector_norm(a - r) / torch.linalg.vector_norm(r))
            large_eval = {"weights_median_rel_err": float(torch.median(torch.abs(a_nn / a_ex - 1))),
                          "image_rel_l2_learned_vs_exact": rel(img_nn, img_ex),
                          "image_rel_l2_unweighted_vs_exact": rel(img_1, img_ex),
                          "features_predict_adjoint_ms": 1e3 * t_nn}
    mlp.close()
    return {"pings": n_pings, "samples": M_tot,
            "plain_single_ping_fp32": {"value": M_tot / t_plain, "unit": UNIT, "s": t_plain},
            "learned_batched_judged": {
                "value": M_tot / t_judged, "unit": UNIT, "s": t_judged,
                "speedup_vs_plain": t_plain / t_judged,
                "accepted_pings": accepted, "fallback_pings": n_pings - accepted,
                "judge_estimated_weight_error": {"median": float(np.median(est)),
                                                 "max": float(np.max(est))},
                "image_rel_l2_vs_exact": {"median": float(np.median(jerrs)),
                                          "max": float(np.max(jerrs))}},
            "learned_batched": {"value": M_tot / t_learned, "unit": UNIT, "s": t_learned,
                                "note": "predicted weights installed without the judge"},
            "speedup": t_plain / t_learned,
            "batched_adjoint_graph": {"value": M_tot / t_graph, "unit": UNIT, "ms": 1e3 * t_graph},
            "image_rel_l2_learned_vs_exact": {"median": float(np.median(errs)),
                                              "max": float(np.max(errs))},
            "train": {"geometries": train_geos, "samples": int(sum(len(gg[0]) for gg in geos)),
                      "steps": train_steps, "batch": 8192, "s": t_train, "data_s": t_data,
                      "loss_first_last": [hist[0][1], hist[-1][1]]},
            "tiles_chosen": sorted(set(tiles)),
            "large_ping": large_eval}


SPREAD_SOURCES = ["paper_1706_08575_gb300/csrc/spread_tile.cuh",
                  "paper_1706_08575_gb300/csrc/spread.cu", "paper_1706_08575_gb300/csrc/plan.cu",
                  "paper_1706_08575_gb300/csrc/spread_mma.cuh",
                  "paper_1706_08575_gb300/csrc/spread_mma.cu",
                  "paper_1706_08575_gb300/csrc/spread_blk.cuh"]

# the spreading kernel of each FTCG_SPREAD_* value, and how the headline line describes it
SPREAD_KERNELS = {1: ("k_spread", "register-window (k_spread)"),
                  2: ("k_spread_mma", "tensor-core, column-bin chunks (k_spread_mma)"),
                  3: ("k_spread_blk", "tensor-core, 8x8-block chunks (k_spread_blk)")}


def spread_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in SPREAD_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_capture(tile, kernel):
    """The committed ncu summary of the spreading kernel on this workload, or None if it is of
    another tile side or kernel, or the spreading sources changed since that capture."""
    with open(os.path.join(ROOT, "profiles", "k_spread_traffic.json")) as f:
        d = json.load(f)
    if (d.get("source_sha") != spread_source_hash() or int(d.get("tile", -1)) != int(tile) or
            not str(d.get("kernel", "")).startswith(kernel + "<")):
        return None
    return d


def recorded_issue(tile, kernel):
    """Instruction issue of the recorded spreading capture (warp instructions per SM per cycle,
    at most 4 on this GPU), or None if it does not apply."""
    try:
        d = recorded_capture(tile, kernel)
        if d is None:
            return None
        ipc = float(d["warp_inst_per_sm_cycle"])
        return {"bound": "issue", "achieved": ipc, "peak": 4.0,
                "unit": "warp instructions / SM / cycle", "frac": ipc / 4.0,
                "warp_instructions_per_launch": d.get("warp_inst_per_launch"),
                "source": d.get("source", "profiles")}
    except Exception:
        return None


def recorded_traffic(tile, kernel):
    """DRAM bytes (read + write) of one spreading launch on this workload from the committed ncu
    summary, or None if it does not apply."""
    try:
        d = recorded_capture(tile, kernel)
        if d is None:
            return None
        return float(d["dram_bytes_per_launch"])
    except Exception:
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def l2_flush_bytes(device):
    """A write of at least twice the L2 (queried; 129 MB if the property is missing), >= 256 MB."""
    import torch
    l2 = getattr(torch.cuda.get_device_properties(device), "L2_cache_size", 0) or 129 * 2 ** 20
    return max(256 * 2 ** 20, 2 * int(l2) + 2 ** 20) // 4 * 4


def precision_sweep_extra(device, reps=20):
    """The 4.2M-sample precision raster (N = 2048, G = 4096) with exact weights: adjoint samples/s
    in FP32 and in BF16 storage (L2 flushed before each call), and each image's sampled rel-L2
    against the FP64 oracle on the FP64 inputs (the BF16 figure is its precision error)."""
    import numpy as np
    import torch
    import sasgen
    import paper_1706_08575_gb300 as F
    from oracle import ftcg_oracle as O
    p = sasgen.precision_sweep()
    lam = torch.from_numpy(p.lam).to(device)
    g = torch.Generator(device=device)
    g.manual_seed(11)
    v = torch.randn(p.M, dtype=torch.complex64, device=device, generator=g)
    vb = torch.view_as_real(v).to(torch.bfloat16)
    flush = torch.empty(l2_flush_bytes(device) // 4, dtype=torch.float32, device=device)
    out = {"workload": "precision raster: 2048 kr x 2048 theta (M=4194304), N=2048, sigma=2, w=8"}
    alpha = None
    for name, prec, vals in [("fp32", F.PREC_FP32, v), ("bf16", F.PREC_BF16, vb)]:
        with F.Plan(lam, p.N, p.sigma, p.w, precision=prec) as pl:
            a = pl.weights()
            if alpha is None:
                alpha = a.cpu().numpy()
            img = pl.adjoint(vals)
            for _ in range(3):
                flush.zero_()
                pl.adjoint(vals, out=img)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(reps)]
            pl.profile(True)
            for e0, e1 in ev:
                flush.zero_()
                e0.record()
                pl.adjoint(vals, out=img)
                e1.record()
            torch.cuda.synchronize()
            (sp_ms, fft_ms, dp_ms), _ = pl.stage_times()
            pl.profile(False)
            ms = statistics.median(a.elapsed_time(b) for a, b in ev)
            inf = pl.info
        G = inf.G
        alg = (20 if name == "fp32" else 14) * p.M + 8 * G * G
        peak, kind = load_peaks()
        ach = alg / (sp_ms * 1e-3) / 1e9
        out[name] = {"value": p.M / (ms * 1e-3), "unit": UNIT, "ms_median": ms, "tile": inf.tile,
                     "layout": inf.layout, "stages_ms": {"spread": sp_ms, "fft": fft_ms,
                                                         "deapod_crop": dp_ms},
                     "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                  "frac": ach / peak, "peak_kind": kind,
                                  "alg_bytes_per_launch": alg, "traffic": None,
                                  "kernel": "spreading stage (spread + halo fix-up)"}}
    # both whole images against the same FP64 reference (inputs in FP64): the rounding of the
    # stored values and weights is part of the BF16 error
    ref = O.adjoint(p.lam, alpha * v.cpu().numpy().astype(np.complex128), p.N, p.sigma, p.w)
    for name, prec, vals in [("fp32", F.PREC_FP32, v), ("bf16", F.PREC_BF16, vb)]:
        with F.Plan(lam, p.N, p.sigma, p.w, precision=prec) as pl:
            pl.set_weights(torch.from_numpy(alpha).to(device))
            got = pl.adjoint(vals).cpu().numpy()
        out[name]["rel_l2_vs_fp64_oracle"] = O.rel_l2(got, ref)
    return out


def psnr(img, ref):
    """10 log10(max |ref|^2 / mean |img - ref|^2) over the pixels (the paper does not state its
    normalisation; this is the usual peak form)."""
    import numpy as np
    mse = float(np.mean(np.abs(np.asarray(img) - ref) ** 2))
    return 10 * math.log10(float(np.max(np.abs(ref)) ** 2) / mse)


def paper_experiments(device, iters=300):
    """The paper's raster experiments (Sec. V) with its test function sin(4 pi x1) sin(2 pi x2)
    (Eq. eq2) on the device: the noisy grid (900 samples, band 15), the asterisk (225 samples,
    band 23) and the side-scan-SAS-like wedge (1000 samples, band 15), N = 30. For each, the
    PSNR against the function of: gridding with the exact diagonal FTCG weights (r = 1), FTCG
    with the banded C (ftcg_band), and the frame approximation (ftcg_cgls to convergence), plus
    the CGLS iterations to a 1e-4 residual without and with the FTCG row weights (the
    preconditioning remark of Sec. V-C). Then the 1-D study of Sec. III-C (Fig. errorComp):
    relative l2 error against sin(4 pi x) for jittered rasters of 2n + 1 samples, the same three
    methods with r = ceil(log(2n + 1))."""
    import numpy as np
    import torch
    import paper_1706_08575_gb300 as F
    import sasgen

    def run(lam, v, N, r):
        out = {}
        lt = torch.from_numpy(lam).to(device)
        vt = torch.from_numpy(v.astype(np.complex64)).to(device)
        with F.Plan(lt, N, 2.0, 8) as p:
            a = p.weights()
            out["cg_diag"] = p.adjoint(vt).cpu().numpy()
            p.band(r)
            out["ftcg_band"] = p.adjoint(vt).cpu().numpy()
            p.set_weights(None)
            x, h, k = p.cgls(vt, iters=iters, tol=1e-7)
            out["frame"] = x.cpu().numpy() * N * N
            _, h0, k0 = p.cgls(vt, iters=iters, tol=1e-4)
            _, h1, k1 = p.cgls(vt, weights=a, iters=iters, tol=1e-4)
        return out, {"plain": int(k0), "ftcg_weights": int(k1)}, int(k)

    res = {}
    for name, lam, r, paper in (
            ("noisy_grid", sasgen.noisy_grid(), 8, {"frame": 39.79, "ftcg_band": 25.91}),
            ("asterisk", sasgen.asterisk(), 12, {"frame": 40.06, "ftcg_band": 37.48}),
            ("sas_like", sasgen.sas_like(), 8, {"frame": 21.04, "ftcg_band": 23.27})):
        N = 30
        imgs, cg_iters, k = run(lam, sasgen.test_function_values(lam), N, r)
        ref = sasgen.test_function_image(N)
        res[name] = {"samples": int(lam.shape[0]), "N": N, "band": 2 * r - 1,
                     "psnr_db": {m: psnr(i, ref) for m, i in imgs.items()},
                     "paper_psnr_db": paper, "frame_cgls_iters": k,
                     "cgls_iters_to_1e-4": cg_iters}
    one_d = []
    for n in (8, 16, 32, 64, 128):
        lam = sasgen.jittered_1d(sasgen.BASE_SEED + 30 + n, n)
        N = 2 * n + 2
        r = int(math.ceil(math.log(2 * n + 1)))
        imgs, _, _ = run(lam, sasgen.test_function_1d_values(lam), N, r)
        x = np.arange(-(N // 2), N - N // 2) / N + 0.5
        ref = np.sin(4 * np.pi * x)
        row = {m: float(np.linalg.norm(i[N // 2] - ref) / np.linalg.norm(ref))
               for m, i in imgs.items()}
        one_d.append({"samples": 2 * n + 1, "N": N, "r": r, "rel_l2": row})
    res["one_d_error_vs_raster"] = one_d
    return res


def tiny_extra(device, reps=50):
    """The 4,096-sample raster (N = 64, w = 6): launch-latency bound, reported in microseconds
    (median of CUDA-event times, warm L2), with its sampled error against the direct sum."""
    import numpy as np
    import torch
    import sasgen
    import paper_1706_08575_gb300 as F
    from oracle import ftcg_oracle as O
    p = sasgen.tiny()
    v = sasgen.values_for(p).astype(np.complex64)
    with F.Plan(torch.from_numpy(p.lam).to(device), p.N, p.sigma, p.w) as pl:
        alpha = pl.weights().cpu().numpy()
        vals = torch.from_numpy(v).to(device)
        img = pl.adjoint(vals)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for e0, e1 in ev:
            e0.record()
            pl.adjoint(vals, out=img)
            e1.record()
        torch.cuda.synchronize()
        us = 1e3 * statistics.median(a.elapsed_time(b) for a, b in ev)
        got = img.cpu().numpy()
        info = pl.info
        # the banded FTCG matrix at r = ceil(log(2N + 1)) (the paper's suggestion): its FP64
        # construction once, then the banded adjoint (tau = C v, spread with unit weights)
        r = int(math.ceil(math.log(2 * p.N + 1)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pl.band(r)
        torch.cuda.synchronize()
        t_band = time.perf_counter() - t0
        bimg = pl.adjoint(vals, out=torch.empty_like(img))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for e0, e1 in ev:
            e0.record()
            pl.adjoint(vals, out=bimg)
            e1.record()
        torch.cuda.synchronize()
        us_band = 1e3 * statistics.median(a.elapsed_time(b) for a, b in ev)
    ref = O.direct_adjoint(p.lam, alpha * v.astype(np.complex128), p.N)
    return {"workload": "tiny: 64 kr x 64 theta (M=4096), N=64, sigma=2, w=6", "us_median": us,
            "value": p.M / (us * 1e-6), "unit": UNIT, "tile": info.tile,
            "rel_l2_vs_direct_sum": O.rel_l2(got, ref),
            "band": {"r": r, "construction_ms": 1e3 * t_band, "adjoint_us_median": us_band,
                     "value": p.M / (us_band * 1e-6), "unit": UNIT}}


def batch_full_extra(device, n_pings=512, reps=5, rank=0, world=1):
    """The uneven batch recipe at full size (512 pings, 20k-400k samples, N in {256, 512, 1024}):
    one batched plan per rank over its share of the pings (shard_pings: split by M + G^2), unit
    weights, random values; the adjoint replayed from a CUDA graph (the inputs, about 9.7 GB
    per batch, are far larger than L2); the spreading stage's roofline from the batch's own stage
    events on non-graph calls. With several ranks the time is the maximum over ranks and the
    samples are those of all ranks."""
    import torch
    import sasgen
    import paper_1706_08575_gb300 as F
    mine = shard_pings(batch_costs(n_pings), world)[rank]
    t0 = time.perf_counter()
    pings = [sasgen.batch_ping(b) for b in mine]
    lams = [torch.from_numpy(p.lam).to(device) for p in pings]
    g = torch.Generator(device=device)
    g.manual_seed(13 + rank)
    vals = [torch.randn(p.M, dtype=torch.complex64, device=device, generator=g) for p in pings]
    M_mine = sum(p.M for p in pings)
    alg = sum(20 * p.M + 8 * (2 * p.N) ** 2 for p in pings)
    t_gen = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with F.Batch(lams, [p.N for p in pings], 2.0, 8) as b:
        torch.cuda.synchronize()
        t_plan = time.perf_counter() - t0
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            b.adjoint(vals, stream=s)              # first call (kernel loading) not timed
            s.synchronize()
            b.profile(True)
            for _ in range(reps):
                b.adjoint(vals, stream=s)
            (sp_ms, rest_ms), ncalls = b.stage_times()
            b.profile(False)
            b.capture(vals)
            b.launch()
            s.synchronize()
            barrier(device)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                b.launch()
            e1.record(s)
            s.synchronize()
            ms = e0.elapsed_time(e1) / reps
    ms_max = reduce_max(ms, device)
    M_tot = int(round(reduce_sum(M_mine, device)))
    peak, kind = load_peaks()
    ach = alg / (sp_ms * 1e-3) / 1e9
    return {"pings": n_pings, "ranks": world, "samples": M_tot, "plan_s": t_plan,
            "generate_s": t_gen,
            "adjoint_graph": {"value": M_tot / (ms_max * 1e-3), "unit": UNIT, "ms": ms_max},
            "stages_ms_rank0": {"spread": sp_ms, "fft_deapod_crop": rest_ms, "calls": ncalls},
            "roofline_rank0": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                               "frac": ach / peak, "peak_kind": kind, "alg_bytes_per_launch": alg,
                               "traffic": None,
                               "kernel": "spreading stage (persistent spread + halo fix-up)"}}


def run_weights_only(args):
    """The exact FP64 weights of the large ping, --steps calls after --warmup (CUDA-event times
    per call); for profiling the weight kernels alone."""
    import statistics
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_1706_08575_gb300 as F
    import sasgen
    device = torch.device("cuda", 0)
    p = sasgen.large_ping()
    with F.Plan(torch.from_numpy(p.lam).to(device), p.N, p.sigma, p.w) as pl:
        out = torch.empty(p.M, dtype=torch.float64, device=device)
        for _ in range(args.warmup):
            pl.weights(out=out)
        ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pl.weights(out=out)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    print(json.dumps({"weights_only": {"workload": "large ping", "M": p.M, "N": p.N,
                                       "ms_median": statistics.median(ms), "calls": len(ms)}}),
          flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    barrier(device)
    import paper_1706_08575_gb300 as F
    import sasgen
    if args.tuner_load and os.path.exists(args.tuner_load):
        F.ftcg.tuner_load(args.tuner_load)      # the autotuner's choices of an earlier process

    p = rank_ping(rank)
    v_np = sasgen.values_for(p, device=device).astype(np.complex64)
    lam = torch.from_numpy(p.lam).to(device)
    vals = torch.from_numpy(v_np).to(device)
    img = torch.empty((p.N, p.N), dtype=torch.complex64, device=device)
    flush_bytes = l2_flush_bytes(device)
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device=device)   # >= 2 x L2
    stream = torch.cuda.current_stream()

    # per-ping: plan + exact weights + one adjoint (host wall clock, synchronised)
    per_ping = []
    plan = None
    for _ in range(2):
        if plan is not None:
            plan.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = F.Plan(lam, p.N, p.sigma, p.w)
        t1 = time.perf_counter()
        plan.weights()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        plan.adjoint(vals, out=img)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        per_ping.append((t1 - t0, t2 - t1, t3 - t2))
    pp = per_ping[-1]

    for _ in range(args.warmup):
        flush.zero_()
        plan.adjoint(vals, out=img)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    plan.profile(True)
    clocks = ClockSampler(local)
    barrier(device)
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("ftcg_timed")        # profilers can select the timed launches
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        plan.adjoint(vals, out=img)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    barrier(device)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    (sp_ms, fft_ms, dp_ms), ncalls = plan.stage_times()
    plan.profile(False)
    total_s = sum(step_ms) / 1e3
    total_max = reduce_max(total_s, device)

    # the same step with a warm L2 (no flush between steps): median of the event times
    wev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(min(args.steps, 50))]
    for e0, e1 in wev:
        e0.record(stream)
        plan.adjoint(vals, out=img)
        e1.record(stream)
    torch.cuda.synchronize()
    warm_ms = statistics.median(a.elapsed_time(b) for a, b in wev)
    warm = {"ms_per_step": warm_ms, "value": world * p.M / (warm_ms * 1e-3), "unit": UNIT}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    hv = torch.from_numpy(v_np).pin_memory()
    himg = torch.empty((p.N, p.N), dtype=torch.complex64).pin_memory()
    for _ in range(2):
        plan.adjoint_host(hv, himg)
    e2e_t = []
    for _ in range(max(3, min(args.steps, 20))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.adjoint_host(hv, himg)
        e2e_t.append(time.perf_counter() - t0)
    e2e_sync_max = reduce_max(statistics.median(e2e_t), device)
    # the same through ftcg_adjoint_host_async, the way a stream of pings is fed: a round robin
    # over E2E_PINGS distinct pings of the workload (the rank's and E2E_PINGS - 1 more seeds),
    # each with its own plan, exact weights and stream. Every step uploads its ping's values from
    # pinned host memory and writes its image back to pinned host memory. The pings' plan data, values, grids and strips (about 100 MB
    # each) together exceed L2, so the steps need no flush: a ping's data has been evicted by
    # the others' before its next turn.
    e2e_plans, e2e_vals, e2e_imgs = [plan], [hv], [himg]
    for i in range(1, E2E_PINGS):
        q = sasgen.large_ping(seed=sasgen.BASE_SEED + 1 + 100_000 * rank + 1_000 * i)
        pl = F.Plan(torch.from_numpy(q.lam).to(device), q.N, q.sigma, q.w)
        pl.weights()
        e2e_plans.append(pl)
        e2e_vals.append(torch.from_numpy(
            sasgen.values_for(q, device=device).astype(np.complex64)).pin_memory())
        e2e_imgs.append(torch.empty((q.N, q.N), dtype=torch.complex64).pin_memory())
    e2e_footprint = sum(pl.info.device_bytes for pl in e2e_plans)
    n_e2e = E2E_PINGS * max(3, min(args.steps, 50) // E2E_PINGS)
    # each plan on its own stream (plans share no buffers), so that one ping's transfers overlap
    # another's compute
    e2e_streams = [torch.cuda.Stream(device) for _ in range(E2E_PINGS)]

    def e2e_round(n):
        for k in range(n):
            i = k % E2E_PINGS
            e2e_plans[i].adjoint_host_async(e2e_vals[i], e2e_imgs[i], stream=e2e_streams[i])

    e2e_round(2 * E2E_PINGS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_round(n_e2e)
    torch.cuda.synchronize()
    e2e_max = reduce_max((time.perf_counter() - t0) / n_e2e, device)
    for pl in e2e_plans[1:]:
        pl.close()

    # parity of this very image against the FP64 oracle, every pixel (O.adjoint on the same
    # FP32-rounded weights and values)
    rel = None
    if rank == 0:
        from oracle import ftcg_oracle as O
        alpha = plan.weights().cpu().numpy()     # the plan's own weights, for the same product
        plan.adjoint(vals, out=img)
        got_img = img.cpu().numpy()
        ref = O.adjoint(p.lam, alpha.astype(np.float32) * v_np.astype(np.complex128), p.N,
                        p.sigma, p.w)
        rel = {"value": O.rel_l2(got_img, ref), "pixels": p.N * p.N,
               "oracle": "O.adjoint (FP64 gridding, every pixel)"}

    info = plan.info
    G = info.G
    kname, kdesc = SPREAD_KERNELS[info.spread_kernel]
    smem_fft = 256 <= G <= 4096 and (G & (G - 1)) == 0
    alg_bytes = 20 * p.M + 8 * G * G              # spreading: 20 B per sample + the grid write
    peak, peak_kind = load_peaks()
    achieved = alg_bytes / (sp_ms * 1e-3) / 1e9
    value = world * p.M * args.steps / total_max

    more = {}
    if not args.no_extras:
        # every rank grids its share of the batch (the time is the maximum over ranks)
        try:
            more["batch_512_pings"] = batch_full_extra(device, rank=rank, world=world)
        except Exception as e:
            more["batch_512_pings"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        extras = None
        if not args.no_extras:
            try:
                extras = learned_vs_plain(device, large=(p, lam, vals),
                                          n_pings=args.extras_pings)
            except Exception as e:       # the headline line must still print
                extras = {"error": f"{type(e).__name__}: {e}"}
            for key, fn in [("precision_sweep", precision_sweep_extra), ("tiny", tiny_extra),
                            ("paper_experiments", paper_experiments)]:
                try:
                    more[key] = fn(device)
                except Exception as e:
                    more[key] = {"error": f"{type(e).__name__}: {e}"}
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            alpha = plan.weights().cpu().numpy()
            cpu = cpu_baselines(p, v_np, alpha, budget_s=args.cpu_budget,
                                extra=not args.no_extras)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": headline_config(world),
            "plan": {"tile": info.tile, "layout": info.layout, "entries": info.entries,
                     "spread_kernel": kdesc,
                     "l2_flush_mib": flush_bytes / 2**20},
            "stages_ms": {"spread": sp_ms, "fft": fft_ms, "deapod_crop": dp_ms, "calls": ncalls,
                          "note": ("fft = column pass; deapod_crop = row pass fused with the "
                                   "window division and crop") if smem_fft else "cuFFT + k_deapod_crop"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": recorded_traffic(info.tile, kname),
                         "kernel": kname +
                                   " + k_halo_add (the spreading stage)",
                         "peak_kind": peak_kind,
                         "issue": recorded_issue(info.tile, kname),
                         "alg_bytes_per_launch": alg_bytes},
            "rel_l2_vs_fp64_oracle": rel,
            "per_ping": {"value": p.M / sum(pp), "unit": UNIT,
                         "plan_ms": 1e3 * pp[0], "weights_ms": 1e3 * pp[1],
                         "adjoint_ms": 1e3 * pp[2]},
            "e2e": {"value": world * p.M / e2e_max, "unit": UNIT,
                    "h2d_bytes_per_step": int(p.M * 8), "d2h_bytes_per_step": int(p.N * p.N * 8),
                    "api": f"ftcg_adjoint_host_async, round robin over {E2E_PINGS} distinct "
                           f"large pings, each with its own plan, exact weights, pinned values "
                           f"and image and its own CUDA stream (uploads, adjoints and write-backs "
                           f"of different pings overlap); {e2e_footprint / 2**20:.0f} MiB of "
                           f"plan data alone, above L2, so no flush between steps",
                    "synchronous_call": {"value": world * p.M / e2e_sync_max, "unit": UNIT,
                                         "api": "ftcg_adjoint_host (one call, synchronised)"}},
            # per step: k_spread, k_halo_add (halo layout only), then for power-of-two G in
            # 256..4096 the two shared-memory FFT passes (the second fused with the window
            # division), otherwise k_deapod_crop after cuFFT (whose kernels are not counted)
            "gpu_launches": ((2 if info.layout == 2 else 1) + (2 if smem_fft else 1)) * args.steps,
            "wall_s_timed_region": wall,
            "clocks": clk,
            "cpu_baseline": cpu,
            "learned_vs_plain_per_ping": extras,
            "warm_l2": warm,
            **more,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def run_learned_kernels(args):
    """Only the learned-weight kernels on the large ping, for profiling: the kNN features and one
    network forward pass (random network parameters; the cost does not depend on them), repeated
    `steps` times after `warmup`; prints their mean times as one JSON line (not the headline)."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    import paper_1706_08575_gb300 as F
    import sasgen
    from paper_1706_08575_gb300 import learn
    p = rank_ping(0)
    lam = torch.from_numpy(p.lam).cuda()
    aux = torch.from_numpy(learn.kr_feature(p.kr)).cuda()
    mlp = F.Mlp(learn.init_params(0))
    for _ in range(args.warmup):
        mlp.predict(F.features(lam, aux))
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tf = tp = 0.0
    for _ in range(args.steps):
        e[0].record()
        feats = F.features(lam, aux)
        e[1].record()
        mlp.predict(feats)
        e[2].record()
        torch.cuda.synchronize()
        tf += e[0].elapsed_time(e[1])
        tp += e[1].elapsed_time(e[2])
    mlp.close()
    print(json.dumps({"learned_kernels": "large ping", "M": p.M, "features_ms": tf / args.steps,
                      "predict_ms": tp / args.steps, "steps": args.steps}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--extras-pings", type=int, default=64)
    ap.add_argument("--only", choices=["learned-kernels", "batch", "weights", "learned"],
                    default=None,
                    help="run one part alone for profiling (prints its own line, not the headline)")
    ap.add_argument("--batch-pings", type=int, default=512)
    ap.add_argument("--tuner-load", default=None,
                    help="load the autotuner's choices from this file first (ftcg_tuner_load), "
                         "e.g. to profile the launches an unprofiled run chose")
    ap.add_argument("--tuner-save", default=None,
                    help="write the autotuner's choices to this file at the end (ftcg_tuner_save)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.only == "learned-kernels":
        run_learned_kernels(args)
    elif args.only == "batch":
        import torch
        import __graft_entry__ as ge
        ge.build()
        if args.tuner_load and os.path.exists(args.tuner_load):
            import paper_1706_08575_gb300 as F
            F.ftcg.tuner_load(args.tuner_load)
        print(json.dumps({"batch": batch_full_extra(torch.device("cuda", 0),
                                                    n_pings=args.batch_pings,
                                                    reps=args.steps)}), flush=True)
    elif args.only == "weights":
        run_weights_only(args)
    elif args.only == "learned":
        import torch
        import __graft_entry__ as ge
        ge.build()
        print(json.dumps({"learned_vs_plain_per_ping": learned_vs_plain(
            torch.device("cuda", 0), n_pings=args.extras_pings)}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    if args.tuner_save and args.impl == "ours" and dist_env()[0] == 0:
        import paper_1706_08575_gb300 as F
        F.ftcg.tuner_save(args.tuner_save)


if __name__ == "__main__":
    main()
