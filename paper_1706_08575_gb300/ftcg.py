"""Python binding of libftcg (argument marshalling only; every step runs in the CUDA library).

PyTorch provides device memory and streams: inputs and outputs are torch tensors on a CUDA
device, the calls are queued on torch's current stream. If the library is not built this module
raises at import of the library, never falls back to a CPU path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

C64, BF16X2 = 0, 1           # value storage
F64, F32 = 0, 1              # weight storage
PREC_FP32, PREC_BF16 = 0, 1  # plan precision

_STATUS = {
    0: "FTCG_SUCCESS", 1: "FTCG_ERR_INVALID_VALUE", 2: "FTCG_ERR_OUT_OF_MEMORY", 3: "FTCG_ERR_CUDA",
    4: "FTCG_ERR_NOT_SUPPORTED", 5: "FTCG_ERR_NUMERIC", 6: "FTCG_ERR_TIMEOUT",
}


class FtcgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


LAYOUT_AUTO, LAYOUT_DUPLICATE, LAYOUT_HALO = 0, 1, 2
SPREAD_AUTO, SPREAD_WINDOW, SPREAD_TENSOR, SPREAD_BLOCK = 0, 1, 2, 3
WINDOW_ES, WINDOW_KB, WINDOW_GAUSS = 0, 1, 2  # gridding window families


class Opts(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("weight_width", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("spread_kernel", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int32), ("G", ctypes.c_int32),
                ("w", ctypes.c_int32), ("tile", ctypes.c_int32), ("tiles_x", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("entries", ctypes.c_int64), ("beta", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("spread_kernel", ctypes.c_int32),
                ("pad0", ctypes.c_int32), ("chunks", ctypes.c_int64)]


_lib = None

# (name, restype, argtypes) of every exported entry point, mirroring include/ftcg.h.
_VP, _I32, _I64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = [
    ("ftcg_plan", _I32, [ctypes.POINTER(_VP), _VP, _I64, _I32, _D, _I32, ctypes.POINTER(Opts), _VP]),
    ("ftcg_plan_info", _I32, [_VP, ctypes.POINTER(PlanInfo)]),
    ("ftcg_weights", _I32, [_VP, _VP, _VP]),
    ("ftcg_set_weights", _I32, [_VP, _VP, _I32, _VP]),
    ("ftcg_spread", _I32, [_VP, _VP, _I32, _VP, _VP]),
    ("ftcg_adjoint", _I32, [_VP, _VP, _I32, _VP, _VP]),
    ("ftcg_adjoint_host", _I32, [_VP, _VP, _I32, _VP, _VP]),
    ("ftcg_adjoint_host_async", _I32, [_VP, _VP, _I32, _VP, _VP]),
    ("ftcg_forward", _I32, [_VP, _VP, _VP, _VP]),
    ("ftcg_check", _I32, [_VP]),
    ("ftcg_plan_entries", _I32, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("ftcg_profile", _I32, [_VP, _I32]),
    ("ftcg_stage_times", _I32, [_VP, _VP, _VP]),
    ("ftcg_plan_batch", _I32, [ctypes.POINTER(_VP), _I32, _VP, _VP, _VP, _D, _I32,
                                ctypes.POINTER(Opts), _VP]),
    ("ftcg_batch_set_weights", _I32, [_VP, _VP, _I32, _VP]),
    ("ftcg_batch_weights", _I32, [_VP, _VP, _VP]),
    ("ftcg_adjoint_batch", _I32, [_VP, _VP, _I32, _VP, _VP]),
    ("ftcg_batch_capture", _I32, [_VP, _VP, _I32, _VP, _VP]),
    ("ftcg_batch_launch", _I32, [_VP, _VP]),
    ("ftcg_batch_info", _I32, [_VP, _VP, _VP, _VP]),
    ("ftcg_batch_destroy", _I32, [_VP]),
    ("ftcg_batch_profile", _I32, [_VP, _I32]),
    ("ftcg_batch_stage_times", _I32, [_VP, _VP, _VP]),
    ("ftcg_features", _I32, [_VP, _VP, _I64, _VP, _VP, _VP]),
    ("ftcg_features_batch", _I32, [_I32, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("ftcg_tuner_save", _I32, [ctypes.c_char_p]),
    ("ftcg_tuner_load", _I32, [ctypes.c_char_p]),
    ("ftcg_mlp_create", _I32, [ctypes.POINTER(_VP), _VP]),
    ("ftcg_mlp_state", _I32, [_VP, _VP, _VP, _VP, _VP, _I32]),
    ("ftcg_mlp_predict", _I32, [_VP, _VP, _I64, _VP, _VP]),
    ("ftcg_mlp_grads", _I32, [_VP, _VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    ("ftcg_mlp_train_step", _I32, [_VP, _VP, _VP, _VP, _I64, ctypes.c_float, _VP, _VP]),
    ("ftcg_mlp_destroy", _I32, [_VP]),
    ("ftcg_adjoint_small_noalloc", _I32, [_VP, _VP, _VP, _I64, _I32, _D, _I32, _VP, _VP]),
    ("ftcg_cgls", _I32, [_VP, _VP, _VP, _I32, _D, _VP, _VP, _VP, _VP]),
    ("ftcg_band", _I32, [_VP, _I32, _VP, _VP]),
    ("ftcg_weights_judge", _I32, [_VP, _VP, _I32, _D, _VP, _VP, _VP]),
    ("ftcg_batch_weights_judge", _I32, [_VP, _VP, _I32, _D, _VP, _VP, _VP]),
    ("ftcg_destroy", _I32, [_VP]),
    ("ftcg_status_string", ctypes.c_char_p, [_I32]),
    ("ftcg_last_error", ctypes.c_char_p, []),
    ("ftcg_version", ctypes.c_char_p, []),
]


def lib_path():
    return _build.LIB_PATH


def lib():
    """Load libftcg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libftcg.so is not built ({path}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise FtcgError(status, lib().ftcg_last_error().decode())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _values_dtype(v):
    import torch
    if v.dtype == torch.complex64:
        return C64
    if v.dtype == torch.bfloat16 and v.dim() == 2 and v.shape[1] == 2:
        return BF16X2
    raise TypeError("values must be complex64 (M,) or bfloat16 (M, 2)")


class Plan:
    """A binned geometry: ftcg_plan on lam (torch float64, M x 2, CUDA)."""

    def __init__(self, lam, N, sigma=2.0, w=8, tile=0, precision=PREC_FP32, weight_width=0,
                 stream=None, allow_numeric=False, layout=LAYOUT_AUTO, spread_kernel=SPREAD_AUTO,
                 window=WINDOW_ES, deterministic=False):
        import torch
        if lam.dtype != torch.float64 or lam.dim() != 2 or lam.shape[1] != 2 or not lam.is_cuda:
            raise TypeError("lam must be a CUDA float64 tensor of shape (M, 2)")
        lam = lam.contiguous()
        self.M, self.N, self.sigma, self.w = int(lam.shape[0]), int(N), float(sigma), int(w)
        self.device = lam.device
        opts = Opts(window, precision, tile, weight_width, layout, spread_kernel,
                    1 if deterministic else 0)
        h = ctypes.c_void_p()
        st = lib().ftcg_plan(ctypes.byref(h), _ptr(lam), self.M, self.N, self.sigma, self.w,
                             ctypes.byref(opts), _stream(stream))
        self._h = h if h.value else None
        if st == 5 and allow_numeric:
            self.numeric_warning = lib().ftcg_last_error().decode()
        else:
            _check(st)
        self.info = self.plan_info()
        self.G = self.info.G

    # --- plumbing -------------------------------------------------------------------------
    def plan_info(self):
        info = PlanInfo()
        _check(lib().ftcg_plan_info(self._h, ctypes.byref(info)))
        return info

    def tensor_core(self):
        """True when the plan spreads with one of the tensor-core kernels (column or block)."""
        return self.info.spread_kernel in (SPREAD_TENSOR, SPREAD_BLOCK)

    def close(self):
        if getattr(self, "_h", None):
            lib().ftcg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- the operations --------------------------------------------------------------------
    def weights(self, out=None, stream=None):
        """Exact FTCG weights (FP64, acquisition order); also installed in the plan."""
        import torch
        if out is None:
            out = torch.empty(self.M, dtype=torch.float64, device=self.device)
        _check(lib().ftcg_weights(self._h, _ptr(out), _stream(stream)))
        return out

    def set_weights(self, alpha, stream=None):
        import torch
        if alpha is None:
            _check(lib().ftcg_set_weights(self._h, None, F64, _stream(stream)))
            return
        dt = F64 if alpha.dtype == torch.float64 else F32
        if alpha.dtype not in (torch.float64, torch.float32):
            raise TypeError("alpha must be float64 or float32")
        _check(lib().ftcg_set_weights(self._h, _ptr(alpha.contiguous()), dt, _stream(stream)))

    def spread(self, values, out=None, stream=None):
        import torch
        vd = _values_dtype(values)
        if out is None:
            out = torch.empty((self.G, self.G), dtype=torch.complex64, device=self.device)
        _check(lib().ftcg_spread(self._h, _ptr(values.contiguous()), vd, _ptr(out), _stream(stream)))
        return out

    def adjoint(self, values, out=None, stream=None):
        import torch
        vd = _values_dtype(values)
        if out is None:
            out = torch.empty((self.N, self.N), dtype=torch.complex64, device=self.device)
        _check(lib().ftcg_adjoint(self._h, _ptr(values.contiguous()), vd, _ptr(out),
                                  _stream(stream)))
        return out

    def adjoint_host(self, values_host, image_host, stream=None):
        """values_host / image_host: torch CPU tensors (pinned for speed)."""
        vd = _values_dtype(values_host)
        _check(lib().ftcg_adjoint_host(self._h, _ptr(values_host), vd, _ptr(image_host),
                                       _stream(stream)))
        return image_host

    def adjoint_host_async(self, values_host, image_host, stream=None):
        """Enqueue ftcg_adjoint_host_async (no synchronisation): the upload overlaps the previous
        call's adjoint. Keep both tensors alive and unchanged until the stream has run it."""
        vd = _values_dtype(values_host)
        _check(lib().ftcg_adjoint_host_async(self._h, _ptr(values_host), vd, _ptr(image_host),
                                             _stream(stream)))
        return image_host

    def forward(self, image, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.M, dtype=torch.complex64, device=self.device)
        _check(lib().ftcg_forward(self._h, _ptr(image.contiguous()), _ptr(out), _stream(stream)))
        return out

    def judge_weights(self, alpha, K=256, max_rel_err=5e-4, stream=None):
        """Judge predicted weights against exact sums at K samples: install the calibrated
        predictions if their estimated error is within max_rel_err, else the exact weights.
        Returns (accepted, {"median_ratio", "rms", "max"})."""
        import torch
        a = alpha.to(torch.float64).contiguous()
        acc = ctypes.c_int32()
        st = (ctypes.c_double * 3)()
        _check(lib().ftcg_weights_judge(self._h, _ptr(a), int(K), float(max_rel_err),
                                        ctypes.byref(acc), ctypes.cast(st, ctypes.c_void_p),
                                        _stream(stream)))
        return bool(acc.value), {"median_ratio": st[0], "rms": st[1], "max": st[2]}

    def band(self, r, stream=None):
        """Banded FTCG coefficients for band r (installed in the plan); returns them as an
        M x (2r - 1) complex128 tensor (row k: column k of C at rows k - r + 1 .. k + r - 1)."""
        import torch
        if int(r) < 1:
            _check(lib().ftcg_band(self._h, int(r), None, _stream(stream)))
        out = torch.zeros((self.M, 2 * int(r) - 1), dtype=torch.complex128, device=self.device)
        _check(lib().ftcg_band(self._h, int(r), _ptr(out), _stream(stream)))
        return out

    def cgls(self, values, weights=None, iters=50, tol=0.0, out=None, stream=None):
        """The frame approximation (minimum-norm least squares, row weights optional) by CGLS
        with this plan's operators. Returns (image, residual norms, iterations that moved x)."""
        import torch
        if values.dtype != torch.complex64:
            raise TypeError("values must be complex64")
        if out is None:
            out = torch.empty((self.N, self.N), dtype=torch.complex64, device=self.device)
        w = None
        if weights is not None:
            w = weights.to(torch.float64).contiguous()
        hist = np.empty(int(iters) + 1, np.float64)
        done = ctypes.c_int32()
        _check(lib().ftcg_cgls(self._h, _ptr(values.contiguous()), _ptr(w), int(iters),
                               float(tol), _ptr(out), hist.ctypes.data_as(ctypes.c_void_p),
                               ctypes.byref(done), _stream(stream)))
        return out, hist, done.value

    def check(self):
        _check(lib().ftcg_check(self._h))

    def profile(self, enable=True):
        _check(lib().ftcg_profile(self._h, 1 if enable else 0))

    def stage_times(self):
        """Mean (spread, fft, deapod) milliseconds over the adjoint calls since the last read."""
        ms = (ctypes.c_float * 3)()
        n = ctypes.c_int32()
        _check(lib().ftcg_stage_times(self._h, ctypes.cast(ms, ctypes.c_void_p),
                                      ctypes.byref(n)))
        return tuple(ms), n.value

    def entries(self):
        n = int(self.info.entries)
        arrs = {k: np.empty(n, np.int32) for k in ("tile", "cx", "cy", "sample")}
        arrs["dx"] = np.empty(n, np.float32)
        arrs["dy"] = np.empty(n, np.float32)
        p = {k: arrs[k].ctypes.data_as(ctypes.c_void_p) for k in arrs}
        _check(lib().ftcg_plan_entries(self._h, p["tile"], p["cx"], p["cy"], p["sample"],
                                       p["dx"], p["dy"]))
        return arrs


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = t.data_ptr() if t is not None else None
    return arr


class Batch:
    """Many pings gridded together: ftcg_plan_batch on a list of (M_i, 2) float64 CUDA tensors."""

    def __init__(self, lams, Ns, sigma=2.0, w=8, tile=0, precision=PREC_FP32, stream=None,
                 layout=LAYOUT_AUTO, spread_kernel=SPREAD_AUTO, window=WINDOW_ES):
        import torch
        self.n = len(lams)
        self.lams = [l.contiguous() for l in lams]
        for l in self.lams:
            if l.dtype != torch.float64 or l.dim() != 2 or l.shape[1] != 2 or not l.is_cuda:
                raise TypeError("every lam must be a CUDA float64 tensor of shape (M, 2)")
        self.Ms = [int(l.shape[0]) for l in self.lams]
        self.Ns = [int(n) for n in Ns]
        self.device = self.lams[0].device
        M_arr = (ctypes.c_int64 * self.n)(*self.Ms)
        N_arr = (ctypes.c_int32 * self.n)(*self.Ns)
        opts = Opts(window, precision, tile, 0, layout, spread_kernel)
        h = ctypes.c_void_p()
        st = lib().ftcg_plan_batch(ctypes.byref(h), self.n, _ptr_array(self.lams), M_arr, N_arr,
                                   float(sigma), int(w), ctypes.byref(opts), _stream(stream))
        self._h = h if h.value else None
        _check(st)

    def close(self):
        if getattr(self, "_h", None):
            lib().ftcg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self):
        tiles = (ctypes.c_int32 * self.n)()
        ent = ctypes.c_int64()
        by = ctypes.c_int64()
        _check(lib().ftcg_batch_info(self._h, ctypes.cast(tiles, ctypes.c_void_p),
                                     ctypes.byref(ent), ctypes.byref(by)))
        return list(tiles), ent.value, by.value

    def set_weights(self, alphas, stream=None):
        import torch
        if alphas is None:
            _check(lib().ftcg_batch_set_weights(self._h, None, F64, _stream(stream)))
            return
        dt = F64 if alphas[0].dtype == torch.float64 else F32
        self._alphas = [a.contiguous() for a in alphas]
        _check(lib().ftcg_batch_set_weights(self._h, _ptr_array(self._alphas), dt,
                                            _stream(stream)))

    def judge_weights(self, alphas, K=256, max_rel_err=5e-4, stream=None):
        """ftcg_batch_weights_judge: per ping (accepted, (median ratio, rms, max))."""
        import torch
        self._alphas = [a.to(torch.float64).contiguous() for a in alphas]
        acc = (ctypes.c_int32 * self.n)()
        st = (ctypes.c_double * (3 * self.n))()
        _check(lib().ftcg_batch_weights_judge(self._h, _ptr_array(self._alphas), int(K),
                                              float(max_rel_err), ctypes.cast(acc, ctypes.c_void_p),
                                              ctypes.cast(st, ctypes.c_void_p), _stream(stream)))
        return [(bool(acc[i]), tuple(st[3 * i:3 * i + 3])) for i in range(self.n)]

    def weights(self, stream=None):
        import torch
        outs = [torch.empty(m, dtype=torch.float64, device=self.device) for m in self.Ms]
        _check(lib().ftcg_batch_weights(self._h, _ptr_array(outs), _stream(stream)))
        return outs

    def _io(self, values, images):
        import torch
        vd = _values_dtype(values[0])
        if images is None:
            images = [torch.empty((n, n), dtype=torch.complex64, device=self.device)
                      for n in self.Ns]
        self._keep = ([v.contiguous() for v in values], images)
        return vd, self._keep[0], images

    def adjoint(self, values, images=None, stream=None):
        vd, vals, images = self._io(values, images)
        _check(lib().ftcg_adjoint_batch(self._h, _ptr_array(vals), vd, _ptr_array(images),
                                        _stream(stream)))
        return images

    def capture(self, values, images=None, stream=None):
        """Capture the batched adjoint into a CUDA graph bound to these buffers."""
        vd, vals, images = self._io(values, images)
        _check(lib().ftcg_batch_capture(self._h, _ptr_array(vals), vd, _ptr_array(images),
                                        _stream(stream)))
        return images

    def launch(self, stream=None):
        _check(lib().ftcg_batch_launch(self._h, _stream(stream)))

    def profile(self, enable=True):
        _check(lib().ftcg_batch_profile(self._h, 1 if enable else 0))

    def stage_times(self):
        """Mean (spread, fft + window division + crop) milliseconds of the ftcg_adjoint_batch
        calls since the last read, and their count."""
        ms = (ctypes.c_float * 2)()
        n = ctypes.c_int32()
        _check(lib().ftcg_batch_stage_times(self._h, ctypes.cast(ms, ctypes.c_void_p),
                                            ctypes.byref(n)))
        return tuple(ms), n.value


def tuner_save(path):
    """Write the tile autotuner's choices of this process to a JSON file (ftcg_tuner_save)."""
    _check(lib().ftcg_tuner_save(os.fsencode(str(path))))


def tuner_load(path):
    """Add the tile autotuner's choices from a JSON file (ftcg_tuner_load)."""
    _check(lib().ftcg_tuner_load(os.fsencode(str(path))))


MLP_PARAMS = 10561
FEAT_WIDTH = 48


def features(lam, aux=None, neighbors=False, stream=None):
    """kNN features (M x 48 bfloat16) of a CUDA float64 (M, 2) raster; optionally the neighbour
    indices (M x 16 int32)."""
    import torch
    M = int(lam.shape[0])
    lam = lam.contiguous()
    out = torch.empty((M, FEAT_WIDTH), dtype=torch.bfloat16, device=lam.device)
    nb = torch.empty((M, 16), dtype=torch.int32, device=lam.device) if neighbors else None
    a = aux.contiguous().to(torch.float64) if aux is not None else None
    _check(lib().ftcg_features(_ptr(lam), _ptr(a), M, _ptr(out), _ptr(nb), _stream(stream)))
    return (out, nb) if neighbors else out


def features_batch(lams, auxs=None, neighbors=False, stream=None, concat=False):
    """kNN features of several independent rasters in one request (ftcg_features_batch).
    Returns the list of per-raster (M_i x 48) bfloat16 tensors, views of one (sum M_i, 48) tensor
    (returned itself with concat=True, rows in raster order); with neighbors=True a pair
    (features, neighbour indices) of such results."""
    import torch
    n = len(lams)
    lams = [l.contiguous() for l in lams]
    for l in lams:
        if l.dtype != torch.float64 or l.dim() != 2 or l.shape[1] != 2 or not l.is_cuda:
            raise TypeError("every lam must be a CUDA float64 tensor of shape (M, 2)")
    if auxs is not None:
        if len(auxs) != n:
            raise ValueError("one aux tensor per raster")
        auxs = [a.contiguous().to(torch.float64) if a is not None else None for a in auxs]
    Ms = [int(l.shape[0]) for l in lams]
    dev = lams[0].device if n else torch.device("cuda")
    cat = torch.empty((sum(Ms), FEAT_WIDTH), dtype=torch.bfloat16, device=dev)
    parts = list(torch.split(cat, Ms)) if n else []
    nb_cat = torch.empty((sum(Ms), 16), dtype=torch.int32, device=dev) if neighbors else None
    nb_parts = list(torch.split(nb_cat, Ms)) if neighbors and n else None
    M_arr = (ctypes.c_int64 * max(n, 1))(*Ms)
    _check(lib().ftcg_features_batch(n, _ptr_array(lams),
                                     _ptr_array(auxs) if auxs is not None else None, M_arr,
                                     _ptr_array(parts), _ptr_array(nb_parts) if neighbors else None,
                                     _stream(stream)))
    if concat:
        return (cat, nb_cat) if neighbors else cat
    return (parts, nb_parts) if neighbors else parts


class Mlp:
    """The weight-predicting network; params: packed FP32 numpy array of MLP_PARAMS values."""

    def __init__(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_PARAMS:
            raise ValueError(f"expected {MLP_PARAMS} parameters")
        h = ctypes.c_void_p()
        _check(lib().ftcg_mlp_create(ctypes.byref(h), p.ctypes.data_as(ctypes.c_void_p)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().ftcg_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def state(self):
        P = np.empty(MLP_PARAMS, np.float32)
        m = np.empty(MLP_PARAMS, np.float32)
        v = np.empty(MLP_PARAMS, np.float32)
        step = ctypes.c_int64()
        _check(lib().ftcg_mlp_state(self._h, P.ctypes.data_as(ctypes.c_void_p),
                                    m.ctypes.data_as(ctypes.c_void_p),
                                    v.ctypes.data_as(ctypes.c_void_p), ctypes.byref(step), 0))
        return {"params": P, "m": m, "v": v, "step": step.value}

    def load_state(self, st):
        P = np.ascontiguousarray(st["params"], np.float32)
        m = np.ascontiguousarray(st["m"], np.float32)
        v = np.ascontiguousarray(st["v"], np.float32)
        step = ctypes.c_int64(int(st["step"]))
        _check(lib().ftcg_mlp_state(self._h, P.ctypes.data_as(ctypes.c_void_p),
                                    m.ctypes.data_as(ctypes.c_void_p),
                                    v.ctypes.data_as(ctypes.c_void_p), ctypes.byref(step), 1))

    def predict(self, feats, out=None, stream=None):
        import torch
        M = int(feats.shape[0])
        if out is None:
            out = torch.empty(M, dtype=torch.float64, device=feats.device)
        _check(lib().ftcg_mlp_predict(self._h, _ptr(feats), M, _ptr(out), _stream(stream)))
        return out

    def grads(self, feats, target, index=None, stream=None):
        B = int(index.shape[0]) if index is not None else int(feats.shape[0])
        g = np.empty(MLP_PARAMS, np.float32)
        loss = ctypes.c_float()
        _check(lib().ftcg_mlp_grads(self._h, _ptr(feats), _ptr(target), _ptr(index), B,
                                    g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss),
                                    _stream(stream)))
        return g, loss.value

    def train_step(self, feats, target, index, lr, want_loss=False, stream=None):
        loss = ctypes.c_float()
        _check(lib().ftcg_mlp_train_step(self._h, _ptr(feats), _ptr(target), _ptr(index),
                                         int(index.shape[0]), float(lr),
                                         ctypes.byref(loss) if want_loss else None,
                                         _stream(stream)))
        return loss.value if want_loss else None
