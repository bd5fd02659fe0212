"""The C-ABI library loads, exports every symbol include/ftcg.h declares, and rejects bad
arguments before touching the device (runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1706_08575_gb300 import build as b
    b.build()
    from paper_1706_08575_gb300 import ftcg
    return ftcg.lib()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "ftcg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ftcg_[a-z0-9_]+)\s*\(", txt)))


def test_header_symbols_exported(L):
    syms = header_symbols()
    assert "ftcg_adjoint" in syms and "ftcg_plan" in syms
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1706_08575_gb300 import ftcg
    bound = {n for n, _, _ in ftcg.SIGNATURES}
    assert set(header_symbols()) <= bound


def test_version_and_strings(L):
    assert L.ftcg_version().startswith(b"ftcg")
    assert L.ftcg_status_string(0) == b"FTCG_SUCCESS"
    assert L.ftcg_status_string(5) == b"FTCG_ERR_NUMERIC"
    assert L.ftcg_destroy(None) == 0


def _plan(L, M=16, N=16, sigma=2.0, w=8, opts=None, lam=1, out=True):
    from paper_1706_08575_gb300 import ftcg
    h = ctypes.c_void_p()
    o = ctypes.byref(opts) if opts is not None else None
    return L.ftcg_plan(ctypes.byref(h) if out else None, ctypes.c_void_p(lam) if lam else None,
                       M, N, sigma, w, o, None)


@pytest.mark.parametrize("kw,status", [
    (dict(N=15), 1), (dict(N=0), 1), (dict(w=1), 1), (dict(w=17), 1), (dict(sigma=0.5), 1),
    (dict(sigma=1.3, N=16), 1),          # sigma N not an integer
    (dict(sigma=1.0, N=6, w=4), 1),      # G < 2 w
    (dict(M=-1), 1), (dict(lam=0), 1), (dict(out=False), 1),
    (dict(M=1 << 25), 4),                # beyond the packed entry format
    (dict(N=1 << 16, sigma=2.0), 4),     # G too large
])
def test_plan_rejects(L, kw, status):
    assert _plan(L, **kw) == status
    assert L.ftcg_last_error() != b""


def test_plan_rejects_opts(L):
    from paper_1706_08575_gb300 import ftcg
    assert _plan(L, opts=ftcg.Opts(3, 0, 0, 0)) == 1                 # window family
    assert _plan(L, opts=ftcg.Opts(0, 2, 0, 0)) == 1                 # precision
    assert _plan(L, opts=ftcg.Opts(0, 0, 48, 0)) == 1                # tile
    assert _plan(L, opts=ftcg.Opts(0, 0, 0, 3)) == 1                 # weight width
    assert _plan(L, opts=ftcg.Opts(0, 0, 0, 0, 3)) == 1              # layout
    assert _plan(L, opts=ftcg.Opts(0, 0, 0, 0, 0, 4)) == 1           # spreading kernel
    o = ftcg.Opts(0, 0, 0, 0)
    o.reserved = 1
    assert _plan(L, opts=o) == 1
    assert _plan(L, opts=ftcg.Opts(0, 0, 0, 0, 0, 0, 2)) == 1        # deterministic is 0 or 1


def test_null_plan_calls(L):
    assert L.ftcg_adjoint(None, None, 0, None, None) == 1
    assert L.ftcg_weights(None, None, None) == 1
    assert L.ftcg_check(None) == 1
    assert L.ftcg_plan_info(None, None) == 1


def test_features_batch_rejects(L):
    """Argument errors of the multi-raster feature request are found before any device call."""
    M = (ctypes.c_int64 * 2)(5, 0)
    null2 = (ctypes.c_void_p * 2)(None, None)
    assert L.ftcg_features_batch(-1, None, None, None, None, None, None) == 1
    assert L.ftcg_features_batch(2, None, None, M, null2, None, None) == 1
    assert L.ftcg_features_batch(2, null2, None, M, null2, None, None) == 1
    assert b"raster 0" in L.ftcg_last_error()
    bad = (ctypes.c_int64 * 2)(0, -3)
    assert L.ftcg_features_batch(2, null2, None, bad, null2, None, None) == 1
    assert b"raster 1" in L.ftcg_last_error()


def test_features_batch_binding_checks_inputs():
    """The binding refuses host tensors and mismatched aux lists before any library call."""
    import torch
    from paper_1706_08575_gb300 import ftcg
    with pytest.raises(TypeError):
        ftcg.features_batch([torch.zeros((3, 2), dtype=torch.float64)])
    with pytest.raises(TypeError):
        ftcg.features_batch([torch.zeros((3, 3), dtype=torch.float64)])


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the shared library absent, every call path raises."""
    from paper_1706_08575_gb300 import ftcg
    monkeypatch.setattr(ftcg, "_lib", None)
    monkeypatch.setattr(ftcg, "lib_path", lambda: str(tmp_path / "libftcg.so"))
    with pytest.raises(RuntimeError, match="not built"):
        ftcg.lib()
    with pytest.raises(RuntimeError, match="not built"):
        ftcg.Mlp(__import__("numpy").zeros(ftcg.MLP_PARAMS, "float32"))


def test_tuner_file_round_trip(L, tmp_path):
    """The autotuner's choices go to a JSON file and come back (host only, no device work); an
    invalid entry or a foreign file is refused and adds nothing."""
    import json
    from paper_1706_08575_gb300 import ftcg
    entries = [{"G": 2048, "w": 8, "precision": 0, "bucket": -3, "tile_req": 0, "layout_req": 0,
                "tile": 32, "layout": 2},
               {"G": 512, "w": 6, "precision": 1, "bucket": 1, "tile_req": 64, "layout_req": 0,
                "tile": 64, "layout": 1},
               {"G": 1024, "w": 8, "precision": 0, "bucket": -1, "tile_req": 0, "layout_req": 0,
                "spread_req": 2, "tile": 64, "layout": 2, "spread": 2},
               {"G": 8192, "w": 8, "precision": 0, "bucket": -8, "tile_req": 0, "layout_req": 0,
                "spread_req": 0, "tile": 32, "layout": 2, "spread": 1},
               {"G": 8192, "w": 8, "precision": 0, "bucket": -8, "tile_req": 0, "layout_req": 0,
                "spread_req": 0, "batch": 1, "tile": 64, "layout": 2, "spread": 2}]
    src = tmp_path / "tuner.json"
    src.write_text('{"ftcg_tuner": 1, "entries": [\n' +
                   ",\n".join(json.dumps(e) for e in entries) + "\n]}\n")
    ftcg.tuner_load(src)
    out = tmp_path / "saved.json"
    ftcg.tuner_save(out)
    saved = json.loads(out.read_text())
    assert saved["ftcg_tuner"] == 1
    for e in entries:               # files written before the spreading-kernel choice load as 0
        assert dict(e, spread_req=e.get("spread_req", 0), batch=e.get("batch", 0),
                    window=e.get("window", 0),
                    spread=e.get("spread", e.get("spread_req", 0))) in saved["entries"]
    bad = tmp_path / "bad.json"
    bad.write_text('{"ftcg_tuner": 1, "entries": [\n' + json.dumps(dict(entries[0], G=1000, tile=48))
                   + "\n]}\n")
    assert L.ftcg_tuner_load(str(bad).encode()) == 1
    assert b"line 2" in L.ftcg_last_error()
    bad.write_text('{"ftcg_tuner": 1, "entries": [\n' + json.dumps(dict(entries[2], layout=1))
                   + "\n]}\n")          # the tensor-core kernel needs the halo layout
    assert L.ftcg_tuner_load(str(bad).encode()) == 1
    bad.write_text('{"ftcg_tuner": 1, "entries": [\n' + json.dumps(dict(entries[4], batch=2))
                   + "\n]}\n")
    assert L.ftcg_tuner_load(str(bad).encode()) == 1
    bad.write_text('{"ftcg_tuner": 1, "entries": [\n' + json.dumps(dict(entries[4], window=3))
                   + "\n]}\n")
    assert L.ftcg_tuner_load(str(bad).encode()) == 1
    other = tmp_path / "other.json"
    other.write_text(json.dumps({"entries": [dict(entries[0], G=4096)]}) + "\n")
    assert L.ftcg_tuner_load(str(other).encode()) == 1
    assert L.ftcg_tuner_load(str(tmp_path / "absent.json").encode()) == 1
    ftcg.tuner_save(out)
    # neither the refused entry nor the foreign file's entry was added (other entries of this
    # process, from plans built earlier, may be present)
    after = json.loads(out.read_text())["entries"]
    assert all(e["G"] != 1000 for e in after)
    assert not any(e["G"] == 4096 and e["bucket"] == entries[0]["bucket"] and e["w"] == 8 and
                   e["tile_req"] == 0 and e["layout_req"] == 0 and e["tile"] == 32 for e in after)


def test_library_carries_its_source_hash():
    """The built library names the sources it was built from; build() rebuilds when they differ
    (a library left over from other sources is never reused)."""
    from paper_1706_08575_gb300 import build as B
    from paper_1706_08575_gb300 import ftcg
    h = B.source_hash()
    assert len(h) == 16
    assert B.built_hash() == h
    assert ftcg.lib().ftcg_version().decode().endswith("ftcg-src-hash:" + h)
    assert B.up_to_date()
