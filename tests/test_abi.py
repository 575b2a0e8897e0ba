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


def test_noalloc_rejects_overflowing_extents_before_gpu_work():
    """perks_stencil_run_noalloc checks each extent before forming their
    product: 2^32 x 2^32 cells (whose product overflows int64 arithmetic on
    the way) is refused with INVALID_ARG by argument checks alone, before
    any CUDA call, so it runs without a GPU."""
    import ctypes as C
    from paper_2204_02064_gb300 import api, inputs
    lib = api.load()
    for shape in [(2 ** 32, 2 ** 32), (1, 2 ** 40, 2 ** 40), (2 ** 21, 1, 1)]:
        d = api._stencil_desc(shape, inputs.shape_offsets("3d7pt" if len(shape) == 3 else "2d5pt"),
                              [0.1] * (7 if len(shape) == 3 else 5), "f64", 0.0, None)
        dummy = C.c_void_p(16)     # never dereferenced: the call fails before using it
        st = lib.perks_stencil_run_noalloc(C.byref(d), dummy, dummy, 3, C.c_void_p(0), 1)
        assert api.STATUS[st] == "INVALID_ARG", shape
