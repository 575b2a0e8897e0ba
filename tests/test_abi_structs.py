"""The ctypes structures of the Python binding against the C ABI's structs.

Every struct that crosses the ABI by pointer (stencil descriptor and plan,
run / CG / batch / Poisson statistics) is declared twice: in include/perks.h
and as a ctypes.Structure in paper_2204_02064_gb300/api.py.  A field added on
one side only would shift every later field.  This test compiles a small C
program against the header with gcc, prints sizeof and the offset of every
field the binding declares, and compares them with ctypes' layout.  CPU
only: nothing is launched."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2204_02064_gb300 import api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [
    (api.StencilDesc, "perks_stencil_desc"),
    (api.StencilPlan, "perks_stencil_plan"),
    (api.RunStats, "perks_run_stats"),
    (api.CgStats, "perks_cg_stats"),
    (api.BatchStats, "perks_batch_stats"),
    (api.PoissonStats, "perks_poisson_stats"),
]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "perks.h"', "int main(void) {"]
    for cls, cname in PAIRS:
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        layout[(cname, field)] = int(value)
    return layout


@pytest.mark.parametrize("cls,cname", PAIRS, ids=[c for _, c in PAIRS])
def test_ctypes_layout_matches_header(c_layout, cls, cname):
    assert ctypes.sizeof(cls) == c_layout[(cname, "sizeof")], cname
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[(cname, field)], (cname, field)
