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
