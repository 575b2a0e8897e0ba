"""GPU parity of the batched persistent stencil (many uneven 2-D domains in
one launch) against the oracle, per domain.  fp32 / bf16 storage is checked
bit for bit against the low-precision oracle (same fp32 FMA order), fp64 to
1e-12 (normwise) against the fp64 oracle."""
import numpy as np
import pytest

from paper_2204_02064_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def rel_err(g, o):
    floor = 1e-3 * max(np.max(np.abs(o)), 1e-300)
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), floor)))


@pytest.fixture(scope="module")
def ctx():
    from paper_2204_02064_gb300 import api
    return api.Context(0)


def small_domains():
    specs = [((40, 64), "2d5pt"), ((57, 128), "2d9pt"), ((33, 256), "2d25pt"), ((128, 72), "2ds9pt"),
             ((9, 16), "2d9pt"), ((200, 1200), "2d25pt"), ((64, 2056), "2d9pt")]
    out = []
    for i, (shape, name) in enumerate(specs):
        out.append(dict(shape=shape, name=name, offsets=inputs.shape_offsets(name),
                        weights=inputs.workload_weights(name, seed=40 + i), seed=500 + i))
    return out


def _run(ctx, doms, steps, dtype, variant=0, plan=None, autotune=0):
    from paper_2204_02064_gb300 import api
    b = api.Batch(ctx, doms, dtype=dtype)
    srcs = []
    for i, d in enumerate(doms):
        f = torch.from_numpy(inputs.stencil_field(d["shape"], d["seed"])).to(TT[dtype]).cuda()
        srcs.append(f)
        b.set_field(i, f)
    if plan is not None:
        b.set_plan(**plan)
    if autotune:
        b.autotune(autotune)
    stats = b.run(steps, variant=variant, stats=True)
    outs = []
    for i, f in enumerate(srcs):
        o = torch.empty_like(f)
        b.get_field(i, o)
        outs.append(o)
    torch.cuda.synchronize()
    return [s.float().double().cpu().numpy() if dtype != "f64" else s.cpu().numpy() for s in srcs], \
           [o.double().cpu().numpy() for o in outs], stats


@pytest.mark.parametrize("plan", [None, dict(granularity=0.05, width_cap=0), dict(granularity=4.0, width_cap=256)])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batch_lowp_bit_exact(ctx, oracle, dtype, plan):
    doms = small_domains()
    srcs, outs, stats = _run(ctx, doms, 13, dtype, plan=plan)
    assert stats["tiles"] >= len(doms)
    for d, s, o in zip(doms, srcs, outs):
        ref = oracle.stencil_run_lowp(s.astype(np.float32), d["offsets"], d["weights"], 13, dtype)
        assert np.array_equal(o.astype(np.float32), ref), d["name"]


def test_batch_fp64(ctx, oracle):
    doms = small_domains()
    srcs, outs, _ = _run(ctx, doms, 11, "f64", plan=dict(granularity=0.2, width_cap=0))
    for d, s, o in zip(doms, srcs, outs):
        ref = oracle.stencil_run(s, d["offsets"], d["weights"], 11)
        assert rel_err(o, ref) <= 1e-12, d["name"]


def test_batch_per_step_and_autotune_agree(ctx):
    doms = small_domains()
    _, a, _ = _run(ctx, doms, 9, "f32", variant=0)
    _, b, _ = _run(ctx, doms, 9, "f32", variant=1)
    _, c, st = _run(ctx, doms, 9, "f32", variant=0, autotune=2)
    assert st["granularity"] > 0
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_batch_full_size_workload(ctx, oracle):
    """The 64-domain workload (sides 128..2048, 3x3 / 5x5 boxes, fp32, 500
    steps): the smallest domains against the oracle bit for bit, every domain
    against the per-domain per-step baseline bit for bit."""
    doms = inputs.batch_domains()
    srcs, outs, stats = _run(ctx, doms, 500, "f32")
    assert stats["grid_blocks"] > 0
    _, base, _ = _run(ctx, doms, 500, "f32", variant=1)
    for o, bo in zip(outs, base):
        assert np.array_equal(o, bo)
    small = sorted(range(len(doms)), key=lambda i: doms[i]["shape"][0])[:3]
    for i in small:
        d = doms[i]
        ref = oracle.stencil_run_lowp(srcs[i].astype(np.float32), d["offsets"], d["weights"], 500, "f32")
        assert np.array_equal(outs[i].astype(np.float32), ref)


@pytest.mark.parametrize("rows", [0, 1, 3, 7, 64])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_strip_kernel_matches_oracle(ctx, oracle, dtype, rows):
    """The column-strip kernel (each warp streams 32-vector strips of rows
    through its own ring): items of 1 row (every row a new pipeline), odd
    heights (ragged row splits), narrow domains (a strip wider than the
    domain: idle lanes read the Dirichlet value) and a 2056-wide one (a
    strip of two vectors after the full ones); fp32 bit for bit against the
    low-precision oracle, fp64 within 1e-12."""
    from paper_2204_02064_gb300 import api
    doms = small_domains()
    b = api.Batch(ctx, doms, dtype=dtype)
    b.set_kernel(api.BATCH_STRIP, rows)
    srcs = []
    for i, d in enumerate(doms):
        f = torch.from_numpy(inputs.stencil_field(d["shape"], d["seed"])).to(TT[dtype]).cuda()
        srcs.append(f)
        b.set_field(i, f)
    st = b.run(12, stats=True)
    assert st["kernel"] == api.BATCH_STRIP and st["strip_rows"] == rows
    for i, (d, f) in enumerate(zip(doms, srcs)):
        o = torch.empty_like(f)
        b.get_field(i, o)
        torch.cuda.synchronize()
        if dtype == "f32":
            ref = oracle.stencil_run_lowp(f.cpu().numpy(), d["offsets"], d["weights"], 12, "f32")
            assert np.array_equal(o.cpu().numpy(), ref), d["name"]
        else:
            ref = oracle.stencil_run(f.cpu().numpy(), d["offsets"], d["weights"], 12)
            assert rel_err(o.cpu().numpy(), ref) <= 1e-12, d["name"]
    b.close()


def test_batch_strip_equals_ring_bitwise(ctx):
    """Both persistent batch kernels add the same fp32 FMA chains: identical
    fields after 21 steps, and the default kernel is the strip kernel."""
    from paper_2204_02064_gb300 import api
    doms = small_domains()
    _, a, sa = _run(ctx, doms, 21, "f32")
    _, r, sr = _run(ctx, doms, 21, "f32", plan=dict(granularity=1.0, width_cap=0))
    assert sa["kernel"] == api.BATCH_STRIP and sr["kernel"] == api.BATCH_RING
    for x, y in zip(a, r):
        assert np.array_equal(x, y)
