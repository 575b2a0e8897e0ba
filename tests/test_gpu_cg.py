"""GPU parity of the CG path (merge-path SpMV + persistent CG) against the oracle.

CG iterates diverge chaotically from any other implementation after many
steps because the dot products are summed in a different order, so parity is
checked as:
  (1) SpMV elementwise (1e-13 relative to the row's absolute sum);
  (2) alpha_k, beta_k, <r,r>_k of the first 20 iterations within 1e-11 (fp64);
  (3) iteration counts within +-2 of the oracle's;
  (4) final x within 1e-7 relative of the oracle's x (rtol 1e-10, kappa ~ 1e2);
  (5) the true residual, recomputed in fp64, at or below the tolerance on both.
"""
import numpy as np
import pytest
import scipy.sparse

from paper_2204_02064_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2204_02064_gb300 import api
    return api.Context(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _op(ctx, rp, c, v):
    from paper_2204_02064_gb300 import api
    return api.CsrOperator(ctx, _dev(rp), _dev(c), _dev(v))


def _rows_abs(rp, c, v, x):
    A = scipy.sparse.csr_matrix((np.abs(v), c, rp), shape=(len(rp) - 1, len(x)))
    return A @ np.abs(x)


def _spmv_case(ctx, oracle, rp, c, v, seed, kind=0):
    n = len(rp) - 1
    x = inputs.cg_rhs(n, seed)
    op = _op(ctx, rp, c, v)
    op.set_spmv(kind)
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    op.spmv(_dev(x), y)
    torch.cuda.synchronize()
    ref = oracle.spmv(rp, c, v, x)
    scale = np.maximum(_rows_abs(rp, c, v, x), 1e-300)
    assert np.max(np.abs(y.cpu().numpy() - ref) / scale) <= 1e-13


@pytest.mark.parametrize("kind", [0, 1, 2], ids=["rowvec", "merge", "seg"])
@pytest.mark.parametrize("n,seed", [(7, 1), (2000, 2), (50000, 3), (300001, 4)])
def test_spmv_synthetic(ctx, oracle, n, seed, kind):
    rp, c, v = inputs.csr_spd_matrix(n, seed)
    _spmv_case(ctx, oracle, rp, c, v, seed, kind)


@pytest.mark.parametrize("kind", [0, 1, 2], ids=["rowvec", "merge", "seg"])
def test_spmv_long_rows_and_empty_rows(ctx, oracle, kind):
    """Rows longer than a tile (4096 path items) and empty rows exercise the
    thread- and tile-level carry fix-up."""
    rng = np.random.default_rng(5)
    n = 30000
    lengths = rng.integers(0, 40, size=n)
    lengths[::97] = 0
    if kind == 2:
        # the segmented layout caps a block's nonzeros per 4096-column segment
        # at 2048: long rows spread over the segments
        lengths[123] = 12000
        lengths[5000] = 6000
        lengths[5001] = 4097
    else:
        lengths[123] = 20000
        lengths[5000] = 9000
        lengths[5001] = 4097
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=rp[1:])
    nnz = int(rp[-1])
    c = rng.integers(0, n, size=nnz).astype(np.int32)
    v = rng.standard_normal(nnz)
    _spmv_case(ctx, oracle, rp.astype(np.int32), c, v, 6, kind)


@pytest.fixture(scope="module")
def system_4k():
    n = 4000
    rp, c, v = inputs.csr_spd_matrix(n, 31)
    return rp, c, v, inputs.cg_rhs(n, 31)


def _solve(ctx, rp, c, v, b, mode, rtol=1e-10, x0=None, host=False, trace_len=0, spmv=0, **kw):
    from paper_2204_02064_gb300 import api
    op = _op(ctx, rp, c, v)
    op.set_spmv(spmv)
    n = len(b)
    if host:
        x = np.zeros(n) if x0 is None else np.array(x0)
        res = op.solve(np.ascontiguousarray(b), x, rtol=rtol, mode=mode, trace_len=trace_len, **kw)
        return x, res
    x = torch.zeros(n, dtype=torch.float64, device="cuda") if x0 is None else _dev(x0)
    res = op.solve(_dev(b), x, rtol=rtol, mode=mode, trace_len=trace_len, **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy(), res


@pytest.mark.parametrize("spmv", [0, 1, 2], ids=["rowvec", "merge", "seg"])
@pytest.mark.parametrize("mode", [0, 2], ids=["persistent", "multi_launch"])
def test_cg_fp64_trace_and_solution(ctx, oracle, system_4k, mode, spmv):
    rp, c, v, b = system_4k
    ref = oracle.cg(rp, c, v, b, rtol=1e-10, trace_len=20)
    x, res = _solve(ctx, rp, c, v, b, mode, trace_len=20, spmv=spmv)
    tr = res["trace"]
    assert tr.shape == ref["trace"].shape
    assert np.max(np.abs(tr - ref["trace"]) / np.abs(ref["trace"])) <= 1e-11
    assert abs(res["iterations"] - ref["iters"]) <= 2
    assert res["true_rel_residual"] <= 1e-10
    assert np.linalg.norm(x - ref["x"]) <= 1e-7 * np.linalg.norm(ref["x"])


@pytest.mark.parametrize("spmv", [0, 1, 2], ids=["rowvec", "merge", "seg"])
def test_cg_fp32_ir(ctx, oracle, system_4k, spmv):
    from paper_2204_02064_gb300 import api
    rp, c, v, b = system_4k
    ref = oracle.cg(rp, c, v, b, rtol=1e-10)
    ir = oracle.cg_fp32_ir(rp, c, v, b, rtol=1e-10, inner_rtol=1e-4)
    x, res = _solve(ctx, rp, c, v, b, api.CG_FP32_IR, inner_rtol=1e-4, spmv=spmv)
    assert res["true_rel_residual"] <= 1e-10
    assert res["outer_iterations"] >= 2
    assert abs(res["outer_iterations"] - ir["outer_iters"]) <= 1
    assert np.linalg.norm(x - ref["x"]) <= 1e-7 * np.linalg.norm(ref["x"])


def test_cg_host_buffers_and_initial_guess(ctx, oracle, system_4k):
    rp, c, v, b = system_4k
    x0 = 0.1 * inputs.cg_rhs(len(b), 77)
    ref = oracle.cg(rp, c, v, b, x0=x0, rtol=1e-10)
    x, res = _solve(ctx, rp, c, v, b, 0, x0=x0, host=True)
    assert res["true_rel_residual"] <= 1e-10
    assert np.linalg.norm(x - ref["x"]) <= 1e-7 * np.linalg.norm(ref["x"])


@pytest.mark.parametrize("spmv", [0, 1, 2], ids=["rowvec", "merge", "seg"])
def test_cg_cached_and_streamed_agree(ctx, oracle, spmv):
    # n=2000: every block's slice fits in shared memory (cached A, merge path);
    # n=60000: several tiles per block, streamed each iteration.
    for n in (2000, 60000):
        rp, c, v = inputs.csr_spd_matrix(n, 8)
        b = inputs.cg_rhs(n, 8)
        ref = oracle.cg(rp, c, v, b, rtol=1e-10, trace_len=10)
        x, res = _solve(ctx, rp, c, v, b, 0, trace_len=10, spmv=spmv)
        assert np.max(np.abs(res["trace"] - ref["trace"]) / np.abs(ref["trace"])) <= 1e-11
        assert res["true_rel_residual"] <= 1e-10


def test_cg_breakdown_reported(ctx):
    from paper_2204_02064_gb300 import api
    A = scipy.sparse.csr_matrix(np.diag([1.0, -1.0]))
    with pytest.raises(api.PerksError) as ei:
        _solve(ctx, A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data, np.ones(2), 0)
    assert ei.value.name == "BREAKDOWN"


def test_cg_zero_rhs(ctx):
    rp, c, v = inputs.csr_spd_matrix(100, 1)
    x, res = _solve(ctx, rp, c, v, np.zeros(100), 0)
    assert res["iterations"] == 0 and np.all(x == 0)


def test_cg_not_converged(ctx, system_4k):
    from paper_2204_02064_gb300 import api
    rp, c, v, b = system_4k
    with pytest.raises(api.PerksError) as ei:
        _solve(ctx, rp, c, v, b, 0, max_iter=3)
    assert ei.value.name == "NOT_CONVERGED"


def test_cg_barrier_timeout(ctx, system_4k):
    from paper_2204_02064_gb300 import api
    rp, c, v, b = system_4k
    ctx.set_barrier_timeout(0)
    try:
        with pytest.raises(api.PerksError) as ei:
            _solve(ctx, rp, c, v, b, 0)
        assert ei.value.name == "BARRIER_TIMEOUT"
    finally:
        ctx.set_barrier_timeout(2_000_000_000)
    x, res = _solve(ctx, rp, c, v, b, 0)
    assert res["true_rel_residual"] <= 1e-10


@pytest.fixture(scope="module")
def system_full():
    n = 1 << 20
    rp, c, v = inputs.csr_spd_matrix(n, inputs.SEED_CG)
    return rp, c, v, inputs.cg_rhs(n, inputs.SEED_CG)


@pytest.mark.parametrize("spmv", [0, 2], ids=["rowvec", "seg"])
def test_cg_full_size(ctx, oracle, system_full, spmv):
    """The CG workload at full size (n = 2^20, rtol 1e-10): trace of the first
    5 iterations against the oracle, true residual on the GPU side, both
    modes."""
    from paper_2204_02064_gb300 import api
    rp, c, v, b = system_full
    ref = oracle.cg(rp, c, v, b, rtol=1e-10, max_iter=5, max_restarts=0, trace_len=5)
    _, res5 = _solve(ctx, rp, c, v, b, 0, max_iter=5, trace_len=5, raise_on_error=False, spmv=spmv)
    assert np.max(np.abs(res5["trace"] - ref["trace"]) / np.abs(ref["trace"])) <= 1e-11
    x, res = _solve(ctx, rp, c, v, b, 0, spmv=spmv)
    assert res["true_rel_residual"] <= 1e-10
    x2, res2 = _solve(ctx, rp, c, v, b, api.CG_FP32_IR, spmv=spmv)
    assert res2["true_rel_residual"] <= 1e-10
    assert np.linalg.norm(x - x2) <= 1e-7 * np.linalg.norm(x)


def test_seg_spmv_limits_reported(ctx):
    """A block whose nonzeros in one 4096-column segment exceed the 2048 the
    shared-memory buffers hold cannot use the segmented SpMV: UNSUPPORTED,
    and the operator keeps working with its previous kind."""
    from paper_2204_02064_gb300 import api
    n = 3000
    # row 0: its diagonal; row 1: 2500 nonzeros in columns 0..2499 (one
    # segment); rows 2..n-1: their diagonal
    lengths = np.ones(n, dtype=np.int64)
    lengths[1] = 2500
    rp = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
    cols = np.concatenate([[0], np.arange(2500), np.arange(2, n)]).astype(np.int32)
    vals = np.ones(cols.shape[0])
    op = api.CsrOperator(ctx, _dev(rp), _dev(cols), _dev(vals))
    with pytest.raises(api.PerksError) as ei:
        op.set_spmv(2)
    assert ei.value.name == "UNSUPPORTED"
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    op.spmv(_dev(np.ones(n)), y)
    torch.cuda.synchronize()
    assert y[1].item() == 2500.0


@pytest.mark.parametrize("rtol", [1e-8, 1e-10])
def test_fp32_ir_automatic_inner_tolerance(ctx, system_full, rtol):
    """inner_rtol = 0 picks sqrt(rtol): two refinement steps reach the
    tolerance (the true residual is recomputed in fp64 on the GPU)."""
    from paper_2204_02064_gb300 import api
    rp, c, v, b = system_full
    x, res = _solve(ctx, rp, c, v, b, api.CG_FP32_IR, rtol=rtol, inner_rtol=0.0)
    assert res["true_rel_residual"] <= rtol
    assert res["outer_iterations"] <= 3


def test_cg_nan_rhs_reports_breakdown(ctx):
    """A NaN in b makes <p, Ap> non-finite at the first iteration: the solver
    stops with BREAKDOWN instead of iterating on NaNs."""
    from paper_2204_02064_gb300 import api
    rp, c, v = inputs.csr_spd_matrix(500, 9)
    b = inputs.cg_rhs(500, 9)
    b[17] = np.nan
    with pytest.raises(api.PerksError) as ei:
        _solve(ctx, rp, c, v, b, 0)
    assert ei.value.name in ("BREAKDOWN", "NOT_CONVERGED")


@pytest.mark.parametrize("mode", [0, 1], ids=["fp64", "fp32_ir"])
def test_vector_cache_levels_identical(ctx, oracle, system_4k, mode):
    """The vector cache (each block's rows of r, or of x, r, q -- the inner
    r, or r, d, q -- in shared memory) changes where values live, not the
    arithmetic: solutions, iteration counts and traces are identical at
    every level."""
    rp, c, v, b = system_4k
    out = {}
    for level in (0, 1, 2):
        op = _op(ctx, rp, c, v)
        op.set_vector_cache(level)
        assert op.vector_cache_active == level
        x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        res = op.solve(_dev(b), x, rtol=1e-10, mode=mode, trace_len=10)
        torch.cuda.synchronize()
        out[level] = (x.cpu().numpy(), res)
        op.close()
    for level in (1, 2):
        assert np.array_equal(out[level][0], out[0][0])
        assert out[level][1]["iterations"] == out[0][1]["iterations"]
        assert np.array_equal(out[level][1]["trace"], out[0][1]["trace"])
    ref = oracle.cg(rp, c, v, b, rtol=1e-10)
    assert np.linalg.norm(out[2][0] - ref["x"]) <= 1e-7 * np.linalg.norm(ref["x"])


def test_vector_cache_full_size(ctx, system_full):
    """n = 2^20 with every vector the blocks own in shared memory: fp64 and
    fp32-IR reach 1e-10 with the same iteration counts as without."""
    from paper_2204_02064_gb300 import api
    rp, c, v, b = system_full
    for mode in (api.CG_FP64, api.CG_FP32_IR):
        its = {}
        for level in (0, 2):
            op = _op(ctx, rp, c, v)
            op.set_vector_cache(level)
            assert op.vector_cache_active == level
            x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
            res = op.solve(_dev(b), x, rtol=1e-10, mode=mode)
            assert res["true_rel_residual"] <= 1e-10
            its[level] = res["iterations"]
            op.close()
        assert its[0] == its[2]


def test_vector_cache_skipped_when_rows_do_not_fit(ctx):
    """2^21 rows of one nonzero each: a block's rows (about 6.9k, 166 KB of
    cache) no longer let two blocks share an SM, so the solve keeps its
    vectors in global memory and still converges (A = 2 I: one iteration)."""
    n = 1 << 21
    rp = np.arange(n + 1, dtype=np.int32)
    c = np.arange(n, dtype=np.int32)
    v = np.full(n, 2.0)
    b = inputs.cg_rhs(n, 21)
    op = _op(ctx, rp, c, v)
    op.set_vector_cache(2)
    assert op.vector_cache_active == 0
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = op.solve(_dev(b), x, rtol=1e-12)
    assert res["true_rel_residual"] <= 1e-12
    assert np.max(np.abs(x.cpu().numpy() - b / 2.0)) <= 1e-15
    op.close()
