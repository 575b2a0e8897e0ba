"""Balanced shares of the cache-free plane-streaming body (C ABI -> CUDA)
against the oracle.

With `balanced` the plan's tile columns (each all of its planes in z) are laid
end to end and cut into one equal share of column-planes per co-resident
block, so a block may finish one column and start the next inside a step.
The cases below make the shares cross column ends at ragged positions and
leave each share only a few planes deep, so every piece's z-halos and the
ring refill between two pieces of one block are exercised.  fp64: within
1e-12 of the local value (floored at 1e-3 of the field maximum); fp32 / bf16
storage: bit for bit against the low-precision oracle."""
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


CASES = [
    # (shape name, grid shape (z, y, x) or (y, x), steps, tiles (x, y), threads, planes per barrier)
    ("3d7pt", (203, 24, 40), 9, (2, 4), 256, 4),
    ("3d7pt", (203, 24, 40), 9, (2, 4), 0, 2),
    ("3d7pt", (157, 40, 40), 6, (2, 4), 0, 4),
    ("2d5pt", (2600, 64), 13, (2, 1), 0, 2),
    ("2d25pt", (2600, 96), 7, (3, 1), 0, 4),
    ("poisson", (131, 20, 24), 5, (2, 4), 0, 2),
]


def _plan(tiles, threads, P):
    return dict(tiles=(tiles[0], tiles[1], 0), smem_cache_planes=0, reg_cache=0, planes_per_barrier=P,
                threads=threads, balanced=True)


def _run(ctx, name, src, steps, plan, variant, dtype):
    from paper_2204_02064_gb300 import api
    st = api.Stencil(ctx, tuple(src.shape), inputs.shape_offsets(name), inputs.workload_weights(name, seed=5),
                     dtype=dtype)
    st.set_plan(**plan)
    st.set_field(src)
    stats = st.run(steps, variant=variant, stats=True)
    out = torch.empty_like(src)
    st.get_field(out)
    torch.cuda.synchronize()
    st.close()
    return out, stats


@pytest.mark.parametrize("variant", [0, 1], ids=["persistent", "per_step"])
@pytest.mark.parametrize("name,shape,steps,tiles,threads,P", CASES)
def test_balanced_fp64(ctx, oracle, name, shape, steps, tiles, threads, P, variant):
    f = inputs.stencil_field(shape, 41)
    src = torch.from_numpy(f).cuda()
    out, stats = _run(ctx, name, src, steps, _plan(tiles, threads, P), variant, "f64")
    if variant == 0:  # more blocks than tile columns: the columns really are shared out
        assert stats["grid_blocks"] > tiles[0] * tiles[1]
    ref = oracle.stencil_run(f, inputs.shape_offsets(name), inputs.workload_weights(name, seed=5), steps)
    assert rel_err(out.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("name,shape,steps,tiles,threads,P", [c for c in CASES if c[4] == 0])
def test_balanced_lowp_bit_exact(ctx, oracle, name, shape, steps, tiles, threads, P, dtype):
    f = inputs.stencil_field(shape, 43).astype(np.float32)
    src = torch.from_numpy(f).to(TT[dtype]).cuda()
    f_store = src.float().cpu().numpy()
    out, stats = _run(ctx, name, src, steps, _plan(tiles, threads, P), 0, dtype)
    assert stats["grid_blocks"] > tiles[0] * tiles[1]
    ref = oracle.stencil_run_lowp(f_store, inputs.shape_offsets(name), inputs.workload_weights(name, seed=5),
                                  steps, dtype)
    got = out.float().cpu().numpy()
    assert np.array_equal(got, ref), float(np.max(np.abs(got - ref)))


def test_balanced_needs_the_cache_free_body(ctx):
    from paper_2204_02064_gb300 import api
    st = api.Stencil(ctx, (203, 24, 40), inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"))
    with pytest.raises(api.PerksError) as ei:
        st.set_plan(tiles=(2, 4, 0), smem_cache_planes=-1, reg_cache=1, balanced=True)
        st.run(2, stats=True)
    assert ei.value.name == "UNSUPPORTED"
    st.close()


def test_balanced_equals_one_tile_per_block_bitwise(ctx):
    """The cut of a domain into blocks does not change what a cell computes:
    the balanced run and a one-tile-per-block run of the same columns give the
    same bits (fp64, 20 steps, persistent)."""
    f = inputs.stencil_field((203, 24, 40), 44)
    src = torch.from_numpy(f).cuda()
    a, _ = _run(ctx, "3d7pt", src, 20, _plan((2, 4), 256, 4), 0, "f64")
    b, _ = _run(ctx, "3d7pt", src, 20, dict(tiles=(2, 4, 3), smem_cache_planes=0, reg_cache=0,
                                            planes_per_barrier=4, threads=256), 0, "f64")
    assert torch.equal(a, b)


@pytest.mark.parametrize("balanced", [False, True])
@pytest.mark.parametrize("threads,P", [(256, 2), (256, 4), (0, 2)])
def test_fp64_3d7pt_unequal_neighbour_weights(ctx, oracle, threads, P, balanced):
    """fp64 3d7pt whose neighbour weights differ takes the cache-free body's
    table-order sum (equal weights take the neighbour-sum form with a pair
    sum carried between planes); both agree with the oracle."""
    from paper_2204_02064_gb300 import api
    shape, steps = (203, 24, 40), 11
    w = np.array([0.31, 0.07, 0.13, 0.09, 0.11, 0.12, 0.17])
    f = inputs.stencil_field(shape, 45)
    src = torch.from_numpy(f).cuda()
    st = api.Stencil(ctx, shape, inputs.shape_offsets("3d7pt"), w)
    st.set_plan(tiles=(2, 4, 0 if balanced else 3), smem_cache_planes=0, reg_cache=0, planes_per_barrier=P,
                threads=threads, balanced=balanced)
    st.set_field(src)
    st.run(steps, stats=True)
    out = torch.empty_like(src)
    st.get_field(out)
    torch.cuda.synchronize()
    st.close()
    ref = oracle.stencil_run(f, inputs.shape_offsets("3d7pt"), w, steps)
    assert rel_err(out.cpu().numpy(), ref) <= 1e-12
