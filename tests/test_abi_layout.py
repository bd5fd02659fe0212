"""The ctypes structures of the binding against the C header: a small C program compiled against
include/ftcg.h prints the size and every field offset of ftcg_opts_t and ftcg_plan_info_t, and
they must equal the binding's (a field added to one side only would shift the others)."""
import os
import shutil
import subprocess

import pytest

from paper_1706_08575_gb300 import ftcg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def c_layout(tmp_path, struct, fields):
    src = tmp_path / "layout.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ftcg.h"', "int main(void) {",
             f'    printf("size %zu\\n", sizeof({struct}));']
    lines += [f'    printf("{f} %zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["    return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("struct,cls", [("ftcg_opts_t", ftcg.Opts), ("ftcg_plan_info_t", ftcg.PlanInfo)])
def test_struct_layout_matches_header(tmp_path, struct, cls):
    names = [f[0] for f in cls._fields_]
    got = c_layout(tmp_path, struct, names)
    import ctypes
    assert got["size"] == ctypes.sizeof(cls)
    for n in names:
        assert got[n] == getattr(cls, n).offset, n
