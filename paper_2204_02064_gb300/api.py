"""Python binding of the C ABI in include/perks.h (argument marshalling only).

Every step of the solvers runs in libperks_gb300.so; this module converts
torch tensors / numpy arrays to pointers, passes the current CUDA stream and
turns status codes into exceptions.  There is no CPU path: if the library is
missing and cannot be built, importing fails.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MAX_POINTS = 125
F64, F32, BF16 = 0, 1, 2
PERSISTENT, PER_STEP = 0, 1
KERNEL_AUTO, KERNEL_RESIDENT, KERNEL_STREAMING, KERNEL_PER_STEP = 0, 1, 2, 3
BATCH_RING, BATCH_STRIP = 0, 1
KERNEL_NAMES = {KERNEL_RESIDENT: "resident", KERNEL_STREAMING: "streaming", KERNEL_PER_STEP: "per_step"}
CG_FP64, CG_FP32_IR, CG_FP64_MULTI = 0, 1, 2
SPMV_ROWVEC, SPMV_MERGE, SPMV_SEG = 0, 1, 2

STATUS = {
    0: "OK", -1: "INVALID_ARG", -2: "UNSUPPORTED", -3: "OUT_OF_MEMORY",
    -4: "LAUNCH_TOO_LARGE", -5: "CUDA", -6: "BARRIER_TIMEOUT", -7: "NOT_CONVERGED",
    -8: "BREAKDOWN",
}
DTYPES = {"f64": F64, "f32": F32, "bf16": BF16}


class PerksError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class StencilDesc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("nz", ctypes.c_int64), ("radius", ctypes.c_int32), ("npts", ctypes.c_int32),
                ("offsets", ctypes.c_int32 * (3 * MAX_POINTS)),
                ("weights", ctypes.c_double * MAX_POINTS), ("dtype", ctypes.c_int32),
                ("boundary", ctypes.c_double)]


class StencilPlan(ctypes.Structure):
    _fields_ = [("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32),
                ("tiles_z", ctypes.c_int32), ("smem_cache_planes", ctypes.c_int32),
                ("reg_cache", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4),
                ("balanced", ctypes.c_int32)]


class RunStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("variant", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32),
                ("tiles_z", ctypes.c_int32), ("reg_cache_planes", ctypes.c_int32),
                ("smem_cache_planes", ctypes.c_int32), ("prefetch_planes", ctypes.c_int32),
                ("smem_bytes_per_block", ctypes.c_int64), ("cells", ctypes.c_int64),
                ("cached_cells", ctypes.c_int64), ("halo_cells_per_step", ctypes.c_int64),
                ("algorithmic_bytes", ctypes.c_double), ("kernel", ctypes.c_int32),
                ("planes_per_sync", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class CgStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer_iterations", ctypes.c_int32),
                ("true_rel_residual", ctypes.c_double), ("status", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("bytes_per_iteration", ctypes.c_double),
                ("trace", ctypes.POINTER(ctypes.c_double)), ("trace_len", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k not in ("trace",)}


class BatchStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("grid_blocks", ctypes.c_int32), ("tiles", ctypes.c_int32),
                ("max_tiles_per_block", ctypes.c_int32), ("width_cap", ctypes.c_int32),
                ("smem_bytes_per_block", ctypes.c_int64), ("cells", ctypes.c_int64),
                ("cached_cells", ctypes.c_int64), ("halo_cells_per_step", ctypes.c_int64),
                ("granularity", ctypes.c_double), ("predicted_ms_per_step", ctypes.c_double),
                ("algorithmic_bytes", ctypes.c_double), ("kernel", ctypes.c_int32),
                ("strip_rows", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PoissonStats(ctypes.Structure):
    _fields_ = [("problems", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
                ("max_iterations", ctypes.c_int32), ("mean_iterations", ctypes.c_double),
                ("max_true_rel_residual", ctypes.c_double),
                ("iterations", ctypes.POINTER(ctypes.c_int32)),
                ("true_rel_residual", ctypes.POINTER(ctypes.c_double)), ("capacity", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()
P = ctypes.c_void_p


def _declare(lib):
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sigs = {
        "perks_context_create": ([ctypes.c_int, ctypes.POINTER(P)], i32),
        "perks_context_destroy": ([P], i32),
        "perks_last_error": ([P], ctypes.c_char_p),
        "perks_context_set_barrier_timeout": ([P, i64], i32),
        "perks_barrier_benchmark": ([P, i32, i32, i32, ctypes.POINTER(f64)], i32),
        "perks_context_info": ([P, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                ctypes.POINTER(i64)], i32),
        "perks_stencil_create": ([P, ctypes.POINTER(StencilDesc), ctypes.POINTER(P)], i32),
        "perks_stencil_destroy": ([P], i32),
        "perks_stencil_set_plan": ([P, ctypes.POINTER(StencilPlan)], i32),
        "perks_stencil_set_field": ([P, P, ctypes.c_int, P], i32),
        "perks_stencil_get_field": ([P, P, ctypes.c_int, P], i32),
        "perks_stencil_run": ([P, i64, i32, P, ctypes.POINTER(RunStats)], i32),
        "perks_stencil_describe": ([P, i64, i32, ctypes.POINTER(RunStats)], i32),
        "perks_stencil_check": ([P, P], i32),
        "perks_csr_create": ([P, i32, i64, P, P, P, ctypes.c_int, ctypes.POINTER(P)], i32),
        "perks_op_destroy": ([P], i32),
        "perks_csr_spmv": ([P, P, P, P], i32),
        "perks_cg_solve": ([P, P, P, f64, i32, i32, f64, ctypes.c_int, P,
                            ctypes.POINTER(CgStats)], i32),
        "perks_cg_last_result": ([P, P, ctypes.POINTER(CgStats)], i32),
        "perks_stencil_run_noalloc": ([ctypes.POINTER(StencilDesc), P, P, i64, P, i32], i32),
        "perks_fp64_fma_benchmark": ([P, i32, ctypes.POINTER(f64)], i32),
        "perks_batch_set_kernel": ([P, i32, i32], i32),
        "perks_gather_benchmark": ([P, i32, i32, i32, ctypes.POINTER(f64)], i32),
        "perks_op_set_spmv": ([P, i32], i32),
        "perks_op_set_vector_cache": ([P, i32], i32),
        "perks_op_vector_cache_active": ([P], i32),
        "perks_stencil_set_trace": ([P, i32], i32),
        "perks_stencil_autotune": ([P, i32, i32, P, ctypes.POINTER(StencilPlan), ctypes.POINTER(f64)], i32),
        "perks_stencil_get_trace": ([P, P, i64, ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
        "perks_poisson_create": ([P, i32, i32, i32, P, ctypes.c_int, ctypes.POINTER(P)], i32),
        "perks_poisson_destroy": ([P], i32),
        "perks_poisson_apply": ([P, P, P, P], i32),
        "perks_poisson_solve": ([P, P, P, f64, i32, P, ctypes.POINTER(PoissonStats)], i32),
        "perks_poisson_set_block_threads": ([P, i32], i32),
        "perks_poisson_scale_guess": ([P, P, P, P], i32),
        "perks_poisson_set_group": ([P, i32], i32),
        "perks_poisson_set_rows_per_pass": ([P, i32], i32),
        "perks_warmnet_create": ([P, P, i32, ctypes.c_uint64, ctypes.POINTER(P)], i32),
        "perks_warmnet_destroy": ([P], i32),
        "perks_warmnet_num_params": ([P], i32),
        "perks_warmnet_get_params": ([P, P], i32),
        "perks_warmnet_set_params": ([P, P], i32),
        "perks_warmnet_set_scale": ([P, ctypes.c_float], i32),
        "perks_warmnet_get_scale": ([P], ctypes.c_float),
        "perks_warmnet_set_pool": ([P, i32], i32),
        "perks_warmnet_set_tensor_cores": ([P, i32], i32),
        "perks_warmnet_predict": ([P, i32, i32, i32, P, P, P, P], i32),
        "perks_warmnet_gradient": ([P, i32, i32, i32, P, P, P, P, P, P], i32),
        "perks_warmnet_train_step": ([P, i32, i32, i32, P, P, P, ctypes.c_float, P, P], i32),
        "perks_warmnet_fit": ([P, i32, i32, i32, P, P, P, i32, i32, ctypes.c_float, i32,
                               ctypes.c_uint64, P, P], i32),
        "perks_batch_create": ([P, i32, ctypes.POINTER(StencilDesc), ctypes.POINTER(P)], i32),
        "perks_batch_destroy": ([P], i32),
        "perks_batch_set_field": ([P, i32, P, ctypes.c_int, P], i32),
        "perks_batch_get_field": ([P, i32, P, ctypes.c_int, P], i32),
        "perks_batch_run": ([P, i64, i32, P, ctypes.POINTER(BatchStats)], i32),
        "perks_batch_autotune": ([P, i64, P, ctypes.POINTER(BatchStats)], i32),
        "perks_batch_set_plan": ([P, f64, i32], i32),
    }
    for name, (args, res) in sigs.items():
        if not hasattr(lib, name):
            continue
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


def library_path() -> str:
    return _build.LIB


def load():
    """Loads libperks_gb300.so, building it with nvcc first if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path)
            _declare(lib)
            _lib = lib
        return _lib


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return P(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return P(0)
    if isinstance(stream, int):
        return P(stream)
    return P(stream.cuda_stream)


def _buffer(obj):
    """(pointer, on_device, nbytes) of a torch tensor or numpy array."""
    try:
        import torch
        if isinstance(obj, torch.Tensor):
            if not obj.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return P(obj.data_ptr()), 1 if obj.is_cuda else 0, obj.numel() * obj.element_size()
    except ImportError:
        pass
    if isinstance(obj, np.ndarray):
        if not obj.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return P(obj.ctypes.data), 0, obj.nbytes
    raise TypeError(f"unsupported buffer type {type(obj)}")


class Context:
    def __init__(self, device: int = 0):
        self._lib = load()
        h = P()
        st = self._lib.perks_context_create(int(device), ctypes.byref(h))
        if st != 0:
            raise PerksError(st, f"perks_context_create(device={device}) failed")
        self.handle = h
        self.device = device

    def check(self, st: int):
        if st != 0:
            raise PerksError(st, self.last_error)

    @property
    def last_error(self) -> str:
        return self._lib.perks_last_error(self.handle).decode()

    def barrier_benchmark(self, blocks: int, threads: int = 512, iterations: int = 2000) -> float:
        """Microseconds per grid barrier of a `blocks` x `threads` persistent grid."""
        us = ctypes.c_double()
        self.check(self._lib.perks_barrier_benchmark(self.handle, int(blocks), int(threads), int(iterations),
                                                     ctypes.byref(us)))
        return us.value

    def fp64_fma_benchmark(self, iterations: int = 20000) -> float:
        """Measured FP64 pipe throughput in TFLOP/s (independent FMA chains on every SM)."""
        t = ctypes.c_double()
        self.check(self._lib.perks_fp64_fma_benchmark(self.handle, int(iterations), ctypes.byref(t)))
        return t.value

    def gather_benchmark(self, log2_elems: int = 20, iterations: int = 2000, elem_bytes: int = 8) -> float:
        """Random gathers of elem_bytes (4 or 8) per second from an L2-resident
        vector of 2^log2_elems elements."""
        t = ctypes.c_double()
        self.check(self._lib.perks_gather_benchmark(self.handle, int(log2_elems), int(elem_bytes), int(iterations),
                                                    ctypes.byref(t)))
        return t.value

    def set_barrier_timeout(self, ns: int):
        self.check(self._lib.perks_context_set_barrier_timeout(self.handle, int(ns)))

    def info(self) -> dict:
        sm, smem, l2 = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        self.check(self._lib.perks_context_info(self.handle, ctypes.byref(sm), ctypes.byref(smem),
                                                ctypes.byref(l2)))
        return {"sm_count": sm.value, "smem_per_block": smem.value, "l2_bytes": l2.value}

    def close(self):
        if getattr(self, "handle", None):
            self._lib.perks_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stencil_desc(shape, offsets, weights, dtype, boundary, radius):
    shape = tuple(int(s) for s in shape)
    if len(shape) not in (2, 3):
        raise ValueError("shape must be 2-D or 3-D")
    offs = [tuple(int(v) for v in o) + (0,) * (3 - len(o)) for o in offsets]
    w = [float(v) for v in weights]
    if len(offs) != len(w) or not 1 <= len(w) <= MAX_POINTS:
        raise ValueError("offsets/weights mismatch or too many points")
    d = StencilDesc()
    d.ndim = len(shape)
    d.nx, d.ny, d.nz = shape[::-1] + (1,) * (3 - len(shape))
    d.radius = int(radius if radius is not None else max(max(abs(v) for v in o) for o in offs))
    d.npts = len(w)
    for i, o in enumerate(offs):
        d.offsets[3 * i:3 * i + 3] = list(o)
        d.weights[i] = w[i]
    d.dtype = DTYPES[dtype]
    d.boundary = float(boundary)
    return d


def stencil_run_noalloc(shape, offsets, weights, src, dst, steps: int, dtype: str = "f64",
                        boundary: float = 0.0, radius: int | None = None, stream=None,
                        sync: bool = True):
    """perks_stencil_run_noalloc: persistent run from device tensor `src` into
    device tensor `dst` with no allocation (scratch is a static device array)."""
    lib = load()
    d = _stencil_desc(shape, offsets, weights, dtype, boundary, radius)
    sp, sdev, sn = _buffer(src)
    dp, ddev, dn = _buffer(dst)
    if not (sdev and ddev):
        raise ValueError("src and dst must be device tensors")
    st = lib.perks_stencil_run_noalloc(ctypes.byref(d), sp, dp, int(steps), _stream(stream),
                                       1 if sync else 0)
    if st != 0:
        raise PerksError(st, "perks_stencil_run_noalloc failed")


class Stencil:
    """A Jacobi stencil over a device-resident grid (perks_stencil_*).

    ``shape`` is (ny, nx) or (nz, ny, nx) in C order (x fastest); ``offsets``
    are (dx, dy[, dz]) tuples and ``weights`` the matching coefficients.
    """

    def __init__(self, ctx: Context, shape, offsets, weights, dtype: str = "f64",
                 boundary: float = 0.0, radius: int | None = None):
        self.ctx = ctx
        self._lib = ctx._lib
        shape = tuple(int(s) for s in shape)
        if len(shape) not in (2, 3):
            raise ValueError("shape must be 2-D or 3-D")
        offs = [tuple(int(v) for v in o) + (0,) * (3 - len(o)) for o in offsets]
        w = [float(v) for v in weights]
        if len(offs) != len(w) or not 1 <= len(w) <= MAX_POINTS:
            raise ValueError("offsets/weights mismatch or too many points")
        d = StencilDesc()
        d.ndim = len(shape)
        dims = shape[::-1] + (1,) * (3 - len(shape))
        d.nx, d.ny, d.nz = dims
        d.radius = int(radius if radius is not None else max(max(abs(v) for v in o) for o in offs))
        d.npts = len(w)
        for i, o in enumerate(offs):
            d.offsets[3 * i:3 * i + 3] = list(o)
            d.weights[i] = w[i]
        d.dtype = DTYPES[dtype]
        d.boundary = float(boundary)
        h = P()
        ctx.check(self._lib.perks_stencil_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.shape = shape
        self.dtype = dtype
        self.cells = int(np.prod(shape))

    def set_plan(self, tiles=(0, 0, 0), smem_cache_planes: int = -1, reg_cache: int = 1,
                 scalar: bool = False, planes_per_barrier: int = 0, kernel: int = KERNEL_AUTO,
                 threads: int = 0, rows: int = 0, balanced: bool = False):
        """Plan override; ``scalar`` selects the one-cell-per-thread kernel
        instead of the 16-byte-vector kernel; ``planes_per_barrier`` (2 or 4,
        0 = automatic) picks how many planes the vector kernel computes
        between two block barriers; ``kernel`` = KERNEL_RESIDENT selects the
        resident-tile kernel (``tiles`` and ``threads`` 256/512 apply to
        it, 0 = automatic), KERNEL_STREAMING / KERNEL_AUTO the plane-streaming
        kernel; ``rows`` (1 or 2, 0 = automatic) is the resident kernel's
        rows per thread; ``balanced`` (cache-free plane streaming only) cuts
        the tile columns' planes into equal shares, one per co-resident
        block, instead of one tile per block."""
        p = StencilPlan()
        p.tiles_x, p.tiles_y, p.tiles_z = [int(t) for t in tiles]
        p.smem_cache_planes = int(smem_cache_planes)
        p.reg_cache = int(rows) if kernel == KERNEL_RESIDENT else int(reg_cache)
        p.reserved[0] = 1 if scalar else 0
        p.reserved[1] = int(planes_per_barrier)
        p.reserved[2] = int(kernel)
        p.reserved[3] = int(threads)
        p.balanced = 1 if balanced else 0
        self.ctx.check(self._lib.perks_stencil_set_plan(self.handle, ctypes.byref(p)))

    def autotune(self, variant: int = PERSISTENT, probe_steps: int = 10, stream=None) -> dict:
        """Times candidate plans on the current field (restored afterwards),
        installs the fastest and returns it with its time per step."""
        p = StencilPlan()
        ms = ctypes.c_double()
        self.ctx.check(self._lib.perks_stencil_autotune(self.handle, int(variant), int(probe_steps),
                                                        _stream(stream), ctypes.byref(p), ctypes.byref(ms)))
        return {"tiles": (p.tiles_x, p.tiles_y, p.tiles_z), "reg_cache": p.reg_cache,
                "smem_cache_planes": p.smem_cache_planes, "planes_per_barrier": p.reserved[1],
                "kernel": KERNEL_NAMES.get(p.reserved[2], "streaming"), "threads": p.reserved[3],
                "rows": p.reg_cache if p.reserved[2] == KERNEL_RESIDENT else 0,
                "balanced": bool(p.balanced), "ms_per_step": ms.value}

    def set_trace(self, steps: int):
        """Record per-block start/end times of the first ``steps`` steps of the
        next persistent runs (0 turns tracing off)."""
        self.ctx.check(self._lib.perks_stencil_set_trace(self.handle, int(steps)))
        self._trace_steps = int(steps)

    def trace(self) -> np.ndarray:
        """(steps + 1, blocks, 2) array of %globaltimer ns of the last traced
        run: [k + 1, block] = (start, end) of the block's work in step k
        (k = -1: prologue)."""
        steps = getattr(self, "_trace_steps", 0)
        cap = 2 * (steps + 1) * 4 * 1024
        buf = np.zeros(cap, dtype=np.uint64)
        g = ctypes.c_int32()
        n = ctypes.c_int32()
        self.ctx.check(self._lib.perks_stencil_get_trace(self.handle, buf.ctypes.data, cap, ctypes.byref(g),
                                                         ctypes.byref(n)))
        return buf[:2 * (n.value + 1) * g.value].reshape(n.value + 1, g.value, 2)

    def reset_plan(self):
        self.ctx.check(self._lib.perks_stencil_set_plan(self.handle, None))

    def set_field(self, src, stream=None):
        ptr, dev, nbytes = _buffer(src)
        self._check_bytes(nbytes)
        self.ctx.check(self._lib.perks_stencil_set_field(self.handle, ptr, dev, _stream(stream)))

    def get_field(self, dst, stream=None):
        ptr, dev, nbytes = _buffer(dst)
        self._check_bytes(nbytes)
        self.ctx.check(self._lib.perks_stencil_get_field(self.handle, ptr, dev, _stream(stream)))
        return dst

    def _check_bytes(self, nbytes):
        es = {"f64": 8, "f32": 4, "bf16": 2}[self.dtype]
        if nbytes != self.cells * es:
            raise ValueError(f"buffer holds {nbytes} bytes, field needs {self.cells * es}")

    def run(self, steps: int, variant: int = PERSISTENT, stream=None, stats: bool = False):
        if stats:
            s = RunStats()
            self.ctx.check(self._lib.perks_stencil_run(self.handle, int(steps), int(variant),
                                                       _stream(stream), ctypes.byref(s)))
            return s.as_dict()
        self.ctx.check(self._lib.perks_stencil_run(self.handle, int(steps), int(variant),
                                                   _stream(stream), None))
        return None

    def describe(self, steps: int, variant: int = PERSISTENT) -> dict:
        s = RunStats()
        self.ctx.check(self._lib.perks_stencil_describe(self.handle, int(steps), int(variant),
                                                        ctypes.byref(s)))
        return s.as_dict()

    def check(self, stream=None):
        self.ctx.check(self._lib.perks_stencil_check(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            self._lib.perks_stencil_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CsrOperator:
    """A CSR matrix on the device (perks_csr_create) and its CG solver."""

    def __init__(self, ctx: Context, rowptr, col, val):
        self.ctx = ctx
        self._lib = ctx._lib
        self._keep = []
        rp_p, rp_dev, rp_n = _buffer(rowptr)
        c_p, c_dev, c_n = _buffer(col)
        v_p, v_dev, v_n = _buffer(val)
        if not (rp_dev == c_dev == v_dev):
            raise ValueError("rowptr, col and val must all be host or all device buffers")
        n = rp_n // 4 - 1
        nnz = c_n // 4
        if v_n != 8 * nnz:
            raise ValueError("val must hold nnz doubles")
        h = P()
        ctx.check(self._lib.perks_csr_create(ctx.handle, n, nnz, rp_p, c_p, v_p, rp_dev,
                                             ctypes.byref(h)))
        self.handle = h
        self.n = n
        self.nnz = nnz

    def set_spmv(self, kind: int):
        """SPMV_ROWVEC (default), SPMV_MERGE (thread-level merge walk) or
        SPMV_SEG (vector and nonzeros staged in shared memory one column
        segment at a time; its layout is built on first selection)."""
        self.ctx.check(self._lib.perks_op_set_spmv(self.handle, int(kind)))

    def set_vector_cache(self, level: int):
        """Vectors each block keeps in shared memory during a persistent
        solve with SPMV_ROWVEC: 0 none (default), 1 r, 2 x, r, q (fp32
        inner: r; r, d, q)."""
        self.ctx.check(self._lib.perks_op_set_vector_cache(self.handle, int(level)))

    @property
    def vector_cache_active(self) -> int:
        return int(self._lib.perks_op_vector_cache_active(self.handle))

    def spmv(self, x, y, stream=None):
        xp, xd, _ = _buffer(x)
        yp, yd, _ = _buffer(y)
        if not (xd and yd):
            raise ValueError("spmv takes device vectors")
        self.ctx.check(self._lib.perks_csr_spmv(self.handle, xp, yp, _stream(stream)))

    def solve(self, b, x, rtol: float = 1e-10, max_iter: int = 10000, mode: int = CG_FP64,
              inner_rtol: float = 0.0, stream=None, stats: bool = True, trace_len: int = 0,
              raise_on_error: bool = True):
        bp, bd, _ = _buffer(b)
        xp, xd, _ = _buffer(x)
        if bd != xd:
            raise ValueError("b and x must both be host or both device buffers")
        if not stats:
            self.ctx.check(self._lib.perks_cg_solve(self.handle, bp, xp, float(rtol), int(max_iter),
                                                    int(mode), float(inner_rtol), bd,
                                                    _stream(stream), None))
            return None
        s = CgStats()
        trace = None
        if trace_len > 0:
            trace = np.zeros(3 * trace_len)
            s.trace = trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            s.trace_len = trace_len
        st = self._lib.perks_cg_solve(self.handle, bp, xp, float(rtol), int(max_iter), int(mode),
                                      float(inner_rtol), bd, _stream(stream), ctypes.byref(s))
        out = s.as_dict()
        out["status_name"] = STATUS.get(st, str(st))
        if trace is not None:
            k = min(trace_len, s.iterations)
            out["trace"] = trace.reshape(-1, 3)[:k].copy()
        if st != 0 and raise_on_error:
            raise PerksError(st, self.ctx.last_error)
        return out

    def last_result(self, stream=None) -> dict:
        s = CgStats()
        st = self._lib.perks_cg_last_result(self.handle, _stream(stream), ctypes.byref(s))
        out = s.as_dict()
        out["status_name"] = STATUS.get(st, str(st))
        return out

    def close(self):
        if getattr(self, "handle", None):
            self._lib.perks_op_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many 2-D domains stepped together in one persistent launch (perks_batch_*).

    ``domains`` is a sequence of dicts with ``shape`` (ny, nx), ``offsets`` and
    ``weights`` (and optionally ``boundary``)."""

    def __init__(self, ctx: Context, domains, dtype: str = "f32"):
        self.ctx = ctx
        self._lib = ctx._lib
        n = len(domains)
        arr = (StencilDesc * n)()
        for i, d in enumerate(domains):
            arr[i] = _stencil_desc(d["shape"], d["offsets"], d["weights"], dtype,
                                   d.get("boundary", 0.0), d.get("radius"))
        h = P()
        ctx.check(self._lib.perks_batch_create(ctx.handle, n, arr, ctypes.byref(h)))
        self.handle = h
        self.shapes = [tuple(d["shape"]) for d in domains]
        self.dtype = dtype

    def set_field(self, i: int, src, stream=None):
        ptr, dev, _ = _buffer(src)
        self.ctx.check(self._lib.perks_batch_set_field(self.handle, int(i), ptr, dev, _stream(stream)))

    def get_field(self, i: int, dst, stream=None):
        ptr, dev, _ = _buffer(dst)
        self.ctx.check(self._lib.perks_batch_get_field(self.handle, int(i), ptr, dev, _stream(stream)))
        return dst

    def run(self, steps: int, variant: int = PERSISTENT, stream=None, stats: bool = False):
        s = BatchStats() if stats else None
        self.ctx.check(self._lib.perks_batch_run(self.handle, int(steps), int(variant), _stream(stream),
                                                 ctypes.byref(s) if stats else None))
        return s.as_dict() if stats else None

    def autotune(self, probe_steps: int = 5, stream=None) -> dict:
        s = BatchStats()
        self.ctx.check(self._lib.perks_batch_autotune(self.handle, int(probe_steps), _stream(stream),
                                                      ctypes.byref(s)))
        return s.as_dict()

    def set_plan(self, granularity: float = 1.0, width_cap: int = 0):
        """Ring kernel with this tile granularity and width cap."""
        self.ctx.check(self._lib.perks_batch_set_plan(self.handle, float(granularity), int(width_cap)))

    def set_kernel(self, kernel: int, strip_rows: int = 0):
        """BATCH_RING or BATCH_STRIP (rows per strip item, 0 = automatic)."""
        self.ctx.check(self._lib.perks_batch_set_kernel(self.handle, int(kernel), int(strip_rows)))

    def close(self):
        if getattr(self, "handle", None):
            self._lib.perks_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Poisson:
    """Batched variable-coefficient Poisson problems (perks_poisson_*).

    ``k`` is an array/tensor of shape (nprob, ny, nx) of positive coefficients."""

    def __init__(self, ctx: Context, k):
        self.ctx = ctx
        self._lib = ctx._lib
        shape = tuple(k.shape)
        if len(shape) != 3:
            raise ValueError("k must be (nprob, ny, nx)")
        self.nprob, self.ny, self.nx = (int(v) for v in shape)
        ptr, dev, nbytes = _buffer(k)
        if nbytes != 8 * self.nprob * self.ny * self.nx:
            raise ValueError("k must be float64")
        h = P()
        ctx.check(self._lib.perks_poisson_create(ctx.handle, self.nx, self.ny, self.nprob, ptr, dev,
                                                 ctypes.byref(h)))
        self.handle = h

    def apply(self, v, y, stream=None):
        vp, vd, _ = _buffer(v)
        yp, yd, _ = _buffer(y)
        if not (vd and yd):
            raise ValueError("apply takes device tensors")
        self.ctx.check(self._lib.perks_poisson_apply(self.handle, vp, yp, _stream(stream)))

    def scale_guess(self, b, x, stream=None):
        """x <- (<x,b> / <x,Ax>) x per problem, in place: the multiple of the
        guess closest to the solution in the A-norm."""
        bp, bd, _ = _buffer(b)
        xp, xd, _ = _buffer(x)
        if not (bd and xd):
            raise ValueError("scale_guess takes device tensors")
        self.ctx.check(self._lib.perks_poisson_scale_guess(self.handle, bp, xp, _stream(stream)))

    def set_block_threads(self, threads: int):
        """512 (one block per SM, default) or 256 threads per problem's block."""
        self.ctx.check(self._lib.perks_poisson_set_block_threads(self.handle, int(threads)))

    def set_rows_per_pass(self, rows: int):
        """4 (default: 128 registers, one 512-thread block per SM) or 1 (64
        registers, two blocks per SM)."""
        self.ctx.check(self._lib.perks_poisson_set_rows_per_pass(self.handle, int(rows)))

    def set_group(self, blocks: int):
        """Blocks per problem: 0 (automatic, default), 1, 2, 4 or 8 (rows split over the group)."""
        self.ctx.check(self._lib.perks_poisson_set_group(self.handle, int(blocks)))

    def solve(self, b, x, rtol: float = 1e-8, max_iter: int = 20000, stream=None, stats: bool = True):
        bp, bd, _ = _buffer(b)
        xp, xd, _ = _buffer(x)
        if not (bd and xd):
            raise ValueError("solve takes device tensors")
        if not stats:
            self.ctx.check(self._lib.perks_poisson_solve(self.handle, bp, xp, float(rtol), int(max_iter),
                                                         _stream(stream), None))
            return None
        it = np.zeros(self.nprob, dtype=np.int32)
        tr = np.zeros(self.nprob, dtype=np.float64)
        s = PoissonStats()
        s.iterations = it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        s.true_rel_residual = tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        s.capacity = self.nprob
        self.ctx.check(self._lib.perks_poisson_solve(self.handle, bp, xp, float(rtol), int(max_iter),
                                                     _stream(stream), ctypes.byref(s)))
        return {"iterations": it, "true_rel_residual": tr, "max_iterations": s.max_iterations,
                "mean_iterations": s.mean_iterations, "grid_blocks": s.grid_blocks,
                "max_true_rel_residual": s.max_true_rel_residual}

    def close(self):
        if getattr(self, "handle", None):
            self._lib.perks_poisson_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WarmNet:
    """The learned warm start (perks_warmnet_*): a 4-layer 3x3 conv network
    mapping (log k, f) to a first guess of u.  Images are device float64
    tensors of shape (nimg, ny, nx)."""

    def __init__(self, ctx: Context, storage: int = BF16, dilations=(1, 2, 4, 8), seed: int = 0, pool: int = 1):
        self.ctx = ctx
        self._lib = ctx._lib
        d = np.ascontiguousarray(dilations, dtype=np.int32)
        h = P()
        ctx.check(self._lib.perks_warmnet_create(ctx.handle, d.ctypes.data, int(storage), int(seed),
                                                 ctypes.byref(h)))
        self.handle = h
        self.num_params = int(self._lib.perks_warmnet_num_params(h))
        self.pool = int(pool)
        if self.pool != 1:
            ctx.check(self._lib.perks_warmnet_set_pool(h, self.pool))

    def set_tensor_cores(self, enable: bool):
        """BF16 storage: inner layers on the tensor cores (default) or CUDA cores."""
        self.ctx.check(self._lib.perks_warmnet_set_tensor_cores(self.handle, int(bool(enable))))

    def close(self):
        if getattr(self, "handle", None):
            self._lib.perks_warmnet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        self.ctx.check(self._lib.perks_warmnet_get_params(self.handle, out.ctypes.data))
        return out

    @params.setter
    def params(self, values):
        v = np.ascontiguousarray(values, dtype=np.float32)
        if v.size != self.num_params:
            raise ValueError("expected %d parameters" % self.num_params)
        self.ctx.check(self._lib.perks_warmnet_set_params(self.handle, v.ctypes.data))

    @property
    def scale(self) -> float:
        return float(self._lib.perks_warmnet_get_scale(self.handle))

    @scale.setter
    def scale(self, value: float):
        self.ctx.check(self._lib.perks_warmnet_set_scale(self.handle, float(value)))

    @staticmethod
    def _dims(t):
        shape = tuple(t.shape)
        if len(shape) != 3:
            raise ValueError("images must be (nimg, ny, nx)")
        return shape

    def _ptrs(self, *ts):
        out = []
        for t in ts:
            p, dev, nbytes = _buffer(t)
            if not dev:
                raise ValueError("warm-start network takes device tensors")
            if nbytes != 8 * int(np.prod(tuple(t.shape))) or tuple(t.shape) != tuple(ts[0].shape):
                raise ValueError("images must be float64 tensors of one shape")
            out.append(p)
        return out

    def predict(self, k, f, u, stream=None):
        nimg, ny, nx = self._dims(k)
        kp, fp, up = self._ptrs(k, f, u)
        self.ctx.check(self._lib.perks_warmnet_predict(self.handle, nimg, ny, nx, kp, fp, up, _stream(stream)))

    def gradient(self, k, f, u, stream=None):
        nimg, ny, nx = self._dims(k)
        kp, fp, up = self._ptrs(k, f, u)
        g = np.empty(self.num_params, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        self.ctx.check(self._lib.perks_warmnet_gradient(self.handle, nimg, ny, nx, kp, fp, up, g.ctypes.data,
                                                        loss.ctypes.data, _stream(stream)))
        return float(loss[0]), g

    def train_step(self, k, f, u, lr: float = 1e-3, stream=None) -> float:
        nimg, ny, nx = self._dims(k)
        kp, fp, up = self._ptrs(k, f, u)
        loss = np.zeros(1, dtype=np.float32)
        self.ctx.check(self._lib.perks_warmnet_train_step(self.handle, nimg, ny, nx, kp, fp, up, float(lr),
                                                          _stream(stream), loss.ctypes.data))
        return float(loss[0])

    def fit(self, k, f, u, batch: int = 16, epochs: int = 1, lr: float = 1e-3, auto_scale: bool = True,
            seed: int = 0, stream=None) -> np.ndarray:
        nimg, ny, nx = self._dims(k)
        kp, fp, up = self._ptrs(k, f, u)
        losses = np.zeros(max(epochs, 1), dtype=np.float32)
        self.ctx.check(self._lib.perks_warmnet_fit(self.handle, nimg, ny, nx, kp, fp, up, int(batch), int(epochs),
                                                   float(lr), int(bool(auto_scale)), int(seed), _stream(stream),
                                                   losses.ctypes.data))
        return losses[:epochs]
