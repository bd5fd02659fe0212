"""Build libftcg.so (the C-ABI library) in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked with cuFFT. No cmake, no torch
extension machinery: the library has no torch types in its interface.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libftcg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# Per-file extra flags: the FP32 spreading/interpolation kernels evaluate the window with the
# fast single-precision exp/sqrt; FP64 code (weights, window transform, planning) is unaffected.
EXTRA = {
    "spread.cu": ["--use_fast_math"],
    "spread_any.cu": ["--use_fast_math"],
    "batch.cu": ["--use_fast_math"],
    "batch_window.cu": ["--use_fast_math"],
    "batch_window_any.cu": ["--use_fast_math"],
}


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(src, verbose=False, src_hash="unknown"):
    obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(CSRC, src), "-o", obj,
           f'-DFTCG_SOURCE_HASH="{src_hash}"', *EXTRA.get(src, [])]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def source_hash():
    """SHA-256 (first 16 hex digits) of every source the library is built from: the csrc files,
    the public header and this script (names and contents, in a fixed order)."""
    h = hashlib.sha256()
    deps = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cuh", ".h"))]
    deps.append(os.path.join(HERE, "..", "include", "ftcg.h"))
    deps.append(os.path.abspath(__file__))
    for d in deps:
        h.update(os.path.basename(d).encode())
        with open(d, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def built_hash(path=None):
    """The source hash embedded in a built library (its version string), or None."""
    path = path or LIB_PATH
    try:
        with open(path, "rb") as f:
            data = f.read()
    except OSError:
        return None
    m = re.search(rb"ftcg-src-hash:([0-9a-f]{16})", data)
    return m.group(1).decode() if m else None


def up_to_date():
    """The library exists and was built from exactly the current sources."""
    return built_hash() == source_hash()


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = sources()
    src_hash = source_hash()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, src_hash), srcs))
    if verbose:
        for (_, log), s in zip(results, srcs):
            sys.stderr.write(f"== {s}\n{log}")
    objs = [o for o, _ in results]
    tmp = LIB_PATH + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcufft", "-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
