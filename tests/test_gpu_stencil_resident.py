"""GPU parity of the resident-tile persistent stencil kernel (every block
keeps its whole tile in shared memory for all steps; Sec. 3's execution
model with D_uncache = 0) against the oracle, called through the C ABI.

fp64: normwise-per-element relative error <= 1e-12 against the fp64 oracle
(as in test_gpu_stencil.py).  fp32 / bf16 storage: bit for bit against the
low-precision oracle (fp32 FMA chain in table order, rounded to the storage
type every step).  The cases cover every compiled thread count, ragged y
and z splits (tiles of different sizes in one grid), segments of uneven
length (dummy plane slots), tiles of one row or one plane, and the 2-D
orientation.
"""
import numpy as np
import pytest

from paper_2204_02064_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def rel_err(g, o):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    floor = 1e-3 * max(np.max(np.abs(o)), 1e-300)
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), floor)))


@pytest.fixture(scope="module")
def ctx():
    from paper_2204_02064_gb300 import api
    return api.Context(0)


def _run(ctx, name, f, steps, dtype, plan=None, boundary=0.0, trace=0):
    from paper_2204_02064_gb300 import api
    offs = inputs.shape_offsets(name)
    w = inputs.workload_weights(name, seed=5)
    st = api.Stencil(ctx, f.shape, offs, w, dtype=dtype, boundary=boundary)
    if plan is not None:
        st.set_plan(kernel=api.KERNEL_RESIDENT, **plan)
    if trace:
        st.set_trace(trace)
    src = torch.from_numpy(np.ascontiguousarray(f)).to(TT[dtype]).cuda()
    st.set_field(src)
    stats = st.run(steps, stats=True)
    out = torch.empty_like(src)
    st.get_field(out)
    torch.cuda.synchronize()
    tr = st.trace() if trace else None
    st.close()
    return src, out, stats, tr


def _check(oracle, name, src, out, steps, dtype, boundary=0.0):
    offs = inputs.shape_offsets(name)
    w = inputs.workload_weights(name, seed=5)
    if dtype == "f64":
        ref = oracle.stencil_run(src.cpu().numpy(), offs, w, steps, boundary=boundary)
        err = rel_err(out.cpu().numpy(), ref)
        assert err <= 1e-12, err
    else:
        ref = oracle.stencil_run_lowp(src.float().cpu().numpy(), offs, w, steps, dtype, boundary=boundary)
        got = out.float().cpu().numpy()
        assert np.array_equal(got, ref), float(np.max(np.abs(got - ref)))


CASES = [
    # (name, grid shape (C order), steps, plan)
    ("3d7pt", (48, 32, 64), 9, dict(threads=512, rows=1)),
    ("3d7pt", (48, 32, 64), 10, dict(threads=256, rows=2)),
    ("3d7pt", (37, 29, 64), 7, dict(threads=512, rows=1)),               # ragged y and z splits
    ("3d7pt", (37, 29, 64), 8, dict(threads=256, rows=2, tiles=(2, 3, 5))),   # odd rows: a half row group
    ("3d7pt", (61, 5, 32), 6, dict(threads=512, rows=1, tiles=(1, 5, 2))),    # one row per tile
    ("3d7pt", (61, 5, 32), 6, dict(threads=256, rows=2, tiles=(1, 5, 2))),    # one row: a row group half outside
    ("3d7pt", (13, 24, 32), 5, dict(threads=512, rows=1, tiles=(2, 2, 13))),  # one plane per tile
    ("3d7pt", (20, 12, 32), 5, dict(threads=512, rows=1, tiles=(4, 3, 2))),   # 8-cell rows: bf16 lanes own W and E
    ("3d7pt", (20, 3, 32), 5, dict(threads=256, rows=2, tiles=(4, 3, 2))),    # one-row tiles own both y-faces
    ("3d7pt", (7, 40, 16), 4, dict(threads=256, rows=2, tiles=(1, 1, 1))),    # one tile: no halo exchange
    ("2d5pt", (256, 256), 100, dict(threads=256, rows=1)),
    ("2d5pt", (131, 128), 17, dict(threads=512, rows=1)),
    ("2d5pt", (97, 64), 11, dict(threads=256, rows=1, tiles=(2, 1, 7))),
]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("name,shape,steps,plan", CASES)
def test_resident_matches_oracle(ctx, oracle, name, shape, steps, plan, dtype):
    f = inputs.stencil_field(shape, 41)
    src, out, stats, _ = _run(ctx, name, f, steps, dtype, plan=plan)
    assert stats["kernel"] == 1 and stats["cached_cells"] == stats["cells"]
    if "tiles" in plan:
        assert (stats["tiles_x"], stats["tiles_y"], stats["tiles_z"]) == tuple(plan["tiles"])
    assert stats["threads_per_block"] == plan["threads"]
    assert stats["reg_cache_planes"] == plan["rows"]
    _check(oracle, name, src, out, steps, dtype)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("steps", [1, 2, 3])
@pytest.mark.parametrize("rows", [1, 2])
def test_resident_few_steps_and_buffer_parity(ctx, oracle, dtype, steps, rows):
    """Odd step counts leave the result in the other ping-pong buffer, even
    ones in the buffer that was read (written only after every block read)."""
    f = inputs.stencil_field((24, 40, 32), 43)
    src, out, _, _ = _run(ctx, "3d7pt", f, steps, dtype, plan=dict(threads=512 if rows == 1 else 256, rows=rows))
    _check(oracle, "3d7pt", src, out, steps, dtype)


@pytest.mark.parametrize("dtype", ["f64", "bf16"])
def test_resident_nonzero_boundary(ctx, oracle, dtype):
    f = inputs.stencil_field((21, 19, 32), 44)
    src, out, _, _ = _run(ctx, "3d7pt", f, 13, dtype, plan=dict(threads=256, rows=2), boundary=0.625)
    _check(oracle, "3d7pt", src, out, 13, dtype, boundary=0.625)


def test_resident_composition_bitwise(ctx):
    """run(7) then run(6) equals run(13) bit for bit (resumable by
    construction: the state between runs is the field)."""
    from paper_2204_02064_gb300 import api
    f = torch.from_numpy(inputs.stencil_field((40, 41, 48), 45)).float().cuda()
    st = api.Stencil(ctx, f.shape, inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"), dtype="f32")
    st.set_plan(kernel=api.KERNEL_RESIDENT)
    st.set_field(f)
    st.run(7)
    st.run(6)
    a = torch.empty_like(f)
    st.get_field(a)
    st.set_field(f)
    st.run(13)
    b = torch.empty_like(f)
    st.get_field(b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_resident_equals_streaming_bitwise(ctx, dtype):
    """Both persistent kernels round the same fp32 chains: bit-identical."""
    from paper_2204_02064_gb300 import api
    shape = (40, 36, 64)
    f = torch.from_numpy(inputs.stencil_field(shape, 46)).to(TT[dtype]).cuda()
    outs = []
    for kernel in (api.KERNEL_RESIDENT, api.KERNEL_STREAMING):
        st = api.Stencil(ctx, shape, inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"), dtype=dtype)
        st.set_plan(kernel=kernel)
        st.set_field(f)
        d = st.run(21, stats=True)
        assert d["kernel"] == kernel
        o = torch.empty_like(f)
        st.get_field(o)
        outs.append(o)
        st.close()
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])


def test_resident_barrier_timeout_and_trace(ctx, oracle):
    """A grid-barrier wait that gives up ends the resident kernel with
    BARRIER_TIMEOUT and the context keeps working; the step trace shows
    every block's step k starting after every block ended step k-1."""
    from paper_2204_02064_gb300 import api
    f = inputs.stencil_field((32, 32, 64), 47)
    ctx.set_barrier_timeout(0)
    try:
        with pytest.raises(api.PerksError) as ei:
            _run(ctx, "3d7pt", f, 5, "f64", plan=dict(threads=512))
        assert ei.value.name == "BARRIER_TIMEOUT"
    finally:
        ctx.set_barrier_timeout(2_000_000_000)
    src, out, stats, tr = _run(ctx, "3d7pt", f, 8, "f64", plan=dict(threads=512), trace=5)
    _check(oracle, "3d7pt", src, out, 8, "f64")
    tr = tr.astype(np.int64)
    assert tr.shape == (6, stats["grid_blocks"], 2)
    assert np.all(tr[:, :, 1] >= tr[:, :, 0])
    assert np.all(tr[1:, :, 0].min(axis=1) >= tr[:-1, :, 1].max(axis=1))


def test_resident_refuses_what_it_cannot_hold(ctx):
    """Asked for explicitly, the resident kernel refuses a domain whose tiles
    cannot fit in shared memory, and a stencil it is not compiled for."""
    from paper_2204_02064_gb300 import api
    st = api.Stencil(ctx, (384, 384, 384), inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"))
    st.set_plan(kernel=api.KERNEL_RESIDENT)
    with pytest.raises(api.PerksError) as ei:
        st.describe(10)
    assert ei.value.name == "UNSUPPORTED"
    st.close()
    st = api.Stencil(ctx, (32, 32, 32), inputs.shape_offsets("3d27pt"), inputs.workload_weights("3d27pt"))
    st.set_plan(kernel=api.KERNEL_RESIDENT)
    with pytest.raises(api.PerksError) as ei:
        st.describe(10)
    assert ei.value.name == "UNSUPPORTED"
    st.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_resident_default_at_192_cubed(ctx, dtype):
    """With no plan, the 3d7pt 192^3 domain in fp32 or bf16 fits the blocks'
    shared memory whole and runs the resident kernel (cached fraction 1)."""
    from paper_2204_02064_gb300 import api
    st = api.Stencil(ctx, (192, 192, 192), inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"),
                     dtype=dtype)
    d = st.describe(1000)
    st.close()
    assert d["kernel"] == 1 and d["cached_cells"] == d["cells"]
    assert d["algorithmic_bytes"] < 0.25 * 2 * 1000 * d["cells"] * {"f32": 4, "bf16": 2}[dtype]
