"""ctypes front end of the CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py``; never by the product package.  It does
argument marshalling only; every step of the arithmetic is in ``oracle.c``.
The shared object is compiled with gcc on first use (``build()``), in
``oracle/_build/``, so the same source serves x86 and Arm hosts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
NOT_CONVERGED = -7
BREAKDOWN = -8


_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lib_omp = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (plain gcc, no -march);
    with openmp=True the same source with -fopenmp into liboracle_omp.so
    (the all-cores CPU baseline of the benchmark only)."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_OMP if openmp else _SO
    if (not force and os.path.exists(so)
            and os.path.getmtime(so) >= os.path.getmtime(_SRC)):
        return so
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def stencil_run_all_cores(field: np.ndarray, offsets, weights, steps: int, boundary: float = 0.0):
    """oracle_stencil_run from the OpenMP build (planes of a step in parallel
    on every host core; identical results).  Returns (field, threads)."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            lib = ctypes.CDLL(build(openmp=True))
            P = ctypes.c_void_p
            i64, f64 = ctypes.c_int64, ctypes.c_double
            lib.oracle_stencil_run.argtypes = [ctypes.c_int, i64, i64, i64, ctypes.c_int,
                                               ctypes.c_int, P, P, f64, i64, P, P]
            lib.oracle_stencil_run.restype = ctypes.c_int
            lib.oracle_threads.restype = ctypes.c_int
            _lib_omp = lib
    lib = _lib_omp
    f = np.ascontiguousarray(field, dtype=np.float64)
    dims = list(f.shape[::-1]) + [1, 1, 1]
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, 3))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
    out = np.empty_like(f)
    st = lib.oracle_stencil_run(f.ndim, dims[0], dims[1], dims[2], int(np.abs(off).max()), off.shape[0],
                                _ptr(off), _ptr(w), float(boundary), int(steps), _ptr(f), _ptr(out))
    if st != OK:
        raise ValueError(f"oracle_stencil_run failed with status {st}")
    return out, int(lib.oracle_threads())


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.oracle_stencil_run.argtypes = [ctypes.c_int, i64, i64, i64, ctypes.c_int,
                                           ctypes.c_int, P, P, f64, i64, P, P]
        lib.oracle_stencil_run.restype = ctypes.c_int
        lib.oracle_stencil_run_lowp.argtypes = [ctypes.c_int, i64, i64, i64, ctypes.c_int,
                                                ctypes.c_int, P, P, f64, i64, ctypes.c_int, P, P]
        lib.oracle_stencil_run_lowp.restype = ctypes.c_int
        lib.oracle_bf16_round.argtypes = [ctypes.c_float]
        lib.oracle_bf16_round.restype = ctypes.c_float
        lib.oracle_poisson_csr.argtypes = [i32, i32, P, P, P, P]
        lib.oracle_poisson_csr.restype = i64
        lib.oracle_conv2d.argtypes = [i32, i32, i32, i32, i32, P, P, P, P]
        lib.oracle_conv2d.restype = None
        lib.oracle_warmnet_forward.argtypes = [i32, i32, i32, i32, P, P, P, P]
        lib.oracle_warmnet_forward.restype = ctypes.c_int
        lib.oracle_warmnet_grad.argtypes = [i32, i32, i32, i32, i32, P, P, P, P, P, P]
        lib.oracle_warmnet_grad.restype = ctypes.c_int
        lib.oracle_csr_spmv.argtypes = [i32, P, P, P, P, P]
        lib.oracle_csr_spmv.restype = None
        lib.oracle_dot.argtypes = [i32, P, P]
        lib.oracle_dot.restype = f64
        lib.oracle_cg.argtypes = [i32, P, P, P, P, P, f64, i32, i32, P, P, P, i32]
        lib.oracle_cg.restype = ctypes.c_int
        lib.oracle_cg_fp32_ir.argtypes = [i32, P, P, P, P, P, f64, f64, i32, i32, P, P, P]
        lib.oracle_cg_fp32_ir.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def stencil_run(field: np.ndarray, offsets, weights, steps: int, boundary: float = 0.0,
                ndim: int | None = None, radius: int | None = None) -> np.ndarray:
    """Jacobi steps of Eq. (iterativeStencil) on a 1/2/3-D interior array.

    ``field`` has shape (nz, ny, nx) / (ny, nx) / (nx,) (x fastest, C order);
    ``offsets`` is a sequence of (dx, dy, dz) triples, ``weights`` the matching
    coefficients.  Returns the field after ``steps`` steps (new array).
    """
    lib = _load()
    f = np.ascontiguousarray(field, dtype=np.float64)
    nd = f.ndim if ndim is None else ndim
    dims = list(f.shape[::-1]) + [1, 1, 1]
    nx, ny, nz = dims[0], dims[1], dims[2]
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, 3))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
    if off.shape[0] != w.shape[0]:
        raise ValueError("offsets and weights differ in length")
    r = int(np.abs(off).max()) if radius is None else radius
    out = np.empty_like(f)
    st = lib.oracle_stencil_run(nd, nx, ny, nz, r, off.shape[0], _ptr(off), _ptr(w),
                                float(boundary), int(steps), _ptr(f), _ptr(out))
    if st != OK:
        raise ValueError(f"oracle_stencil_run failed with status {st}")
    return out


def stencil_run_lowp(field: np.ndarray, offsets, weights, steps: int, storage: str,
                     boundary: float = 0.0, ndim: int | None = None,
                     radius: int | None = None) -> np.ndarray:
    """fp32 / bf16 storage variant (fp32 FMA accumulation, table order).

    ``field`` holds values already of the storage type (as float32); returns
    float32 values of the storage type."""
    lib = _load()
    f = np.ascontiguousarray(field, dtype=np.float32)
    nd = f.ndim if ndim is None else ndim
    dims = list(f.shape[::-1]) + [1, 1, 1]
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, 3))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
    r = int(np.abs(off).max()) if radius is None else radius
    out = np.empty_like(f)
    code = {"f32": 1, "bf16": 2}[storage]
    st = lib.oracle_stencil_run_lowp(nd, dims[0], dims[1], dims[2], r, off.shape[0], _ptr(off),
                                     _ptr(w), float(boundary), int(steps), code, _ptr(f), _ptr(out))
    if st != OK:
        raise ValueError(f"oracle_stencil_run_lowp failed with status {st}")
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bf16 (nearest, ties to even), returned as float32."""
    lib = _load()
    xs = np.asarray(x, dtype=np.float32).ravel()
    return np.array([lib.oracle_bf16_round(float(v)) for v in xs], dtype=np.float32).reshape(np.shape(x))


def _csr(rowptr, col, val):
    return (np.ascontiguousarray(rowptr, dtype=np.int32),
            np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


def spmv(rowptr, col, val, x) -> np.ndarray:
    lib = _load()
    rp, c, v = _csr(rowptr, col, val)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    n = rp.shape[0] - 1
    y = np.empty(n, dtype=np.float64)
    lib.oracle_csr_spmv(n, _ptr(rp), _ptr(c), _ptr(v), _ptr(xx), _ptr(y))
    return y


def dot(u, v) -> float:
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    return float(lib.oracle_dot(uu.shape[0], _ptr(uu), _ptr(vv)))


def cg(rowptr, col, val, b, x0=None, rtol: float = 1e-10, max_iter: int = 10000,
       max_restarts: int = 4, trace_len: int = 0):
    """CG of Sec. 2.2.2.  Returns dict(x, status, iters, true_rel, trace)."""
    lib = _load()
    rp, c, v = _csr(rowptr, col, val)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    n = rp.shape[0] - 1
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it = ctypes.c_int32(0)
    tr = ctypes.c_double(0.0)
    trace = np.zeros((max(trace_len, 1), 3))
    st = lib.oracle_cg(n, _ptr(rp), _ptr(c), _ptr(v), _ptr(bb), _ptr(x), float(rtol),
                       int(max_iter), int(max_restarts), ctypes.byref(it), ctypes.byref(tr),
                       _ptr(trace) if trace_len > 0 else None, int(trace_len))
    k = min(it.value, trace_len)
    return dict(x=x, status=st, iters=it.value, true_rel=tr.value, trace=trace[:k].copy())


def cg_fp32_ir(rowptr, col, val, b, x0=None, rtol: float = 1e-10, inner_rtol: float = 1e-4,
               max_inner: int = 5000, max_outer: int = 50):
    """FP32-inner CG with fp64 iterative refinement.  Returns a dict."""
    lib = _load()
    rp, c, v = _csr(rowptr, col, val)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    n = rp.shape[0] - 1
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    inner = ctypes.c_int32(0)
    outer = ctypes.c_int32(0)
    tr = ctypes.c_double(0.0)
    st = lib.oracle_cg_fp32_ir(n, _ptr(rp), _ptr(c), _ptr(v), _ptr(bb), _ptr(x), float(rtol),
                               float(inner_rtol), int(max_inner), int(max_outer),
                               ctypes.byref(inner), ctypes.byref(outer), ctypes.byref(tr))
    return dict(x=x, status=st, inner_iters=inner.value, outer_iters=outer.value,
                true_rel=tr.value)


def poisson_csr(k: np.ndarray):
    """CSR of the finite-volume operator for the coefficient field k (ny, nx)."""
    lib = _load()
    kk = np.ascontiguousarray(k, dtype=np.float64)
    ny, nx = kk.shape
    n = nx * ny
    rp = np.empty(n + 1, dtype=np.int32)
    c = np.empty(5 * n, dtype=np.int32)
    v = np.empty(5 * n, dtype=np.float64)
    nnz = lib.oracle_poisson_csr(nx, ny, _ptr(kk), _ptr(rp), _ptr(c), _ptr(v))
    return rp, c[:nnz].copy(), v[:nnz].copy()


def conv2d(x: np.ndarray, w: np.ndarray, b=None, dil: int = 1) -> np.ndarray:
    """x: (cin, h, w); w: (cout, cin, 3, 3); returns (cout, h, w)."""
    lib = _load()
    xx = np.ascontiguousarray(x, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    cin, h, wd = xx.shape
    cout = ww.shape[0]
    bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    out = np.empty((cout, h, wd))
    lib.oracle_conv2d(cin, cout, h, wd, dil, _ptr(xx), _ptr(ww), _ptr(bb) if bb is not None else None,
                      _ptr(out))
    return out


def warmnet_forward(params: np.ndarray, x: np.ndarray, c1: int, dil=(1, 2, 4, 8)) -> np.ndarray:
    """Forward pass of the 4-layer warm-start network on one input (c0, h, w)."""
    lib = _load()
    xx = np.ascontiguousarray(x, dtype=np.float64)
    c0, h, w = xx.shape
    pp = np.ascontiguousarray(params, dtype=np.float64)
    dd = np.ascontiguousarray(dil, dtype=np.int32)
    out = np.empty((h, w))
    st = lib.oracle_warmnet_forward(c0, c1, h, w, _ptr(dd), _ptr(pp), _ptr(xx), _ptr(out))
    if st != OK:
        raise ValueError("oracle_warmnet_forward failed")
    return out


def warmnet_grad(params: np.ndarray, x: np.ndarray, t: np.ndarray, c1: int, dil=(1, 2, 4, 8)):
    """Loss mean((N(x) - t)^2) over a batch x (nimg, c0, h, w) with targets
    t (nimg, h, w), and its gradient (same layout as params)."""
    lib = _load()
    xx = np.ascontiguousarray(x, dtype=np.float64)
    nimg, c0, h, w = xx.shape
    tt = np.ascontiguousarray(t, dtype=np.float64).reshape(nimg, h, w)
    pp = np.ascontiguousarray(params, dtype=np.float64)
    dd = np.ascontiguousarray(dil, dtype=np.int32)
    g = np.empty_like(pp)
    loss = np.zeros(1)
    st = lib.oracle_warmnet_grad(nimg, c0, c1, h, w, _ptr(dd), _ptr(pp), _ptr(xx), _ptr(tt), _ptr(loss), _ptr(g))
    if st != OK:
        raise ValueError("oracle_warmnet_grad failed")
    return float(loss[0]), g
