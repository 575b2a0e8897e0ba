"""The allocation-free stencil entry point (perks_stencil_run_noalloc),
called through the C ABI, against the regular entry point
(perks_stencil_run on a stencil object).  Its scratch is a static device
array shared by all calls, so several calls in a row must each give the
regular result, whatever the previous call left in the array."""
import numpy as np
import pytest

from paper_2204_02064_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rel_err(g, o):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    floor = 1e-3 * max(np.max(np.abs(o)), 1e-300)
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), floor)))


TOL = {"f64": 1e-12, "f32": 1e-5}
TT = {"f64": torch.float64, "f32": torch.float32}


def _regular(ctx, name, f, steps, dtype):
    from paper_2204_02064_gb300 import api
    st = api.Stencil(ctx, f.shape, inputs.shape_offsets(name), inputs.workload_weights(name, seed=5),
                     dtype=dtype)
    st.set_field(f)
    st.run(steps, api.PERSISTENT, stats=True)
    out = torch.empty_like(f)
    st.get_field(out)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_regular_entry_point_on_consecutive_calls(dtype):
    from paper_2204_02064_gb300 import api
    ctx = api.Context(0)
    cases = [("3d7pt", (40, 36, 52), 25, 1), ("2d5pt", (256, 256), 100, 2),
             ("3d7pt", (33, 47, 29), 12, 3)]
    for name, shape, steps, seed in cases:
        f = torch.from_numpy(inputs.stencil_field(shape, seed)).to(TT[dtype]).cuda()
        keep = f.clone()
        ref = _regular(ctx, name, f, steps, dtype)
        out = torch.full_like(f, float("nan"))
        api.stencil_run_noalloc(shape, inputs.shape_offsets(name), inputs.workload_weights(name, seed=5),
                                f, out, steps, dtype=dtype, sync=True)
        torch.cuda.synchronize()
        assert torch.equal(f, keep)                      # the input is only read
        assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) <= TOL[dtype]


def test_noalloc_rejects_too_large():
    from paper_2204_02064_gb300 import api
    shape = (1025, 1024)                                 # 2^20 + 1024 cells > 2^20
    f = torch.zeros(shape, dtype=torch.float64, device="cuda")
    out = torch.empty_like(f)
    with pytest.raises(api.PerksError) as ei:
        api.stencil_run_noalloc(shape, inputs.shape_offsets("2d5pt"), [0.2] * 5, f, out, 3)
    assert ei.value.name == "INVALID_ARG"


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_in_place_odd_and_even_steps(dtype):
    """in == out: a sequence of in-place calls with odd and even step counts
    (the odd ones end in the scratch field and copy back) gives the regular
    entry point's result for the total number of steps."""
    from paper_2204_02064_gb300 import api
    ctx = api.Context(0)
    name, shape = "3d7pt", (24, 30, 36)
    w = inputs.workload_weights(name, seed=5)
    f = torch.from_numpy(inputs.stencil_field(shape, 9)).to(TT[dtype]).cuda()
    ref = _regular(ctx, name, f, 3 + 4 + 5, dtype)
    x = f.clone()
    for steps in (3, 4, 5):
        api.stencil_run_noalloc(shape, inputs.shape_offsets(name), w, x, x, steps, dtype=dtype, sync=True)
    torch.cuda.synchronize()
    assert rel_err(x.cpu().numpy(), ref.cpu().numpy()) <= TOL[dtype]


def test_noalloc_zero_steps_copies_the_input():
    from paper_2204_02064_gb300 import api
    shape = (20, 24)
    f = torch.from_numpy(inputs.stencil_field(shape, 10)).cuda()
    out = torch.full_like(f, float("nan"))
    api.stencil_run_noalloc(shape, inputs.shape_offsets("2d5pt"), [0.2] * 5, f, out, 0)
    torch.cuda.synchronize()
    assert torch.equal(out, f)


def test_noalloc_unsupported_dtype_and_radius():
    from paper_2204_02064_gb300 import api
    shape = (32, 32)
    f = torch.zeros(shape, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(api.PerksError) as ei:
        api.stencil_run_noalloc(shape, inputs.shape_offsets("2d5pt"), [0.2] * 5, f, f.clone(), 2, dtype="bf16")
    assert ei.value.name == "UNSUPPORTED"
    g = torch.zeros(shape, dtype=torch.float64, device="cuda")
    offs = inputs.shape_offsets("2d13pt")                  # radius 3
    with pytest.raises(api.PerksError) as ei:
        api.stencil_run_noalloc(shape, offs, [1.0 / len(offs)] * len(offs), g, g.clone(), 2)
    assert ei.value.name == "INVALID_ARG"


def test_noalloc_rejects_edge_buffers_beyond_the_scratch():
    """A domain within the cell limit whose plan needs more than the 4 MiB of
    x-edge buffers the scratch holds: tall, narrow 3-D slabs split into many
    tiles of large y-z faces.  The size of the edge buffers is computed from
    the regular entry point's plan (perks_stencil_describe) for the same
    descriptor, so the case is known to exceed the limit before the call."""
    from paper_2204_02064_gb300 import api
    ctx = api.Context(0)
    w = inputs.workload_weights("3d7pt")
    chosen = None
    for shape in [(1024, 1024, 1), (512, 1024, 2), (256, 512, 8), (2048, 512, 1)]:
        st = api.Stencil(ctx, shape, inputs.shape_offsets("3d7pt"), w)
        try:
            d = st.describe(10, api.PERSISTENT)
        except api.PerksError:
            st.close()
            continue
        st.close()
        nz, ny, nx = shape
        tz = -(-nz // d["tiles_z"])
        ty = -(-ny // d["tiles_y"])
        width = 2 if nx % 2 == 0 else 1
        face_bytes = d["grid_blocks"] * 2 * width * tz * ty * 8
        if 2 * face_bytes > (4 << 20):
            chosen = shape
            break
    assert chosen is not None, "no candidate shape exceeds the edge-buffer limit"
    f = torch.zeros(chosen, dtype=torch.float64, device="cuda")
    with pytest.raises(api.PerksError) as ei:
        api.stencil_run_noalloc(chosen, inputs.shape_offsets("3d7pt"), w, f, f.clone(), 3)
    assert ei.value.name == "INVALID_ARG"
