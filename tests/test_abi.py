"""The C-ABI library loads and exports every entry point include/perks.h
declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "perks.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(perks_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("perks_context_create", "perks_stencil_create", "perks_stencil_run",
              "perks_csr_create", "perks_cg_solve"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_2204_02064_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2204_02064_gb300")
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle|#include\s+.*oracle)", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not pat.search(src), f
