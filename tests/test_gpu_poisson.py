"""GPU parity of the batched variable-coefficient Poisson operator and its
persistent CG against the oracle (CSR of the same finite-volume operator)."""
import numpy as np
import pytest

from paper_2204_02064_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2204_02064_gb300 import api
    return api.Context(0)


def _k(nprob, ny, nx, seed):
    return np.exp(2.0 * inputs.uniform(seed, nprob * ny * nx).reshape(nprob, ny, nx) - 1.0)


def test_apply_matches_oracle(ctx, oracle):
    from paper_2204_02064_gb300 import api
    nprob, ny, nx = 3, 37, 53
    k = _k(nprob, ny, nx, 1)
    v = inputs.uniform(2, nprob * ny * nx).reshape(nprob, ny, nx) - 0.5
    P = api.Poisson(ctx, torch.from_numpy(k).cuda())
    y = torch.zeros(nprob, ny, nx, dtype=torch.float64, device="cuda")
    P.apply(torch.from_numpy(v).cuda(), y)
    torch.cuda.synchronize()
    for i in range(nprob):
        rp, c, val = oracle.poisson_csr(k[i])
        ref = oracle.spmv(rp, c, val, v[i].ravel())
        assert np.max(np.abs(y[i].cpu().numpy().ravel() - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("nprob,ny,nx", [(5, 24, 31), (300, 16, 16)])
def test_batched_cg_matches_oracle(ctx, oracle, nprob, ny, nx):
    """Every problem reaches the tolerance; iterations and solutions agree
    with the oracle's CG on the CSR form of the same operator."""
    from paper_2204_02064_gb300 import api
    k = _k(nprob, ny, nx, 3)
    f = 2.0 * inputs.uniform(4, nprob * ny * nx).reshape(nprob, ny, nx) - 1.0
    P = api.Poisson(ctx, torch.from_numpy(k).cuda())
    x = torch.zeros(nprob, ny, nx, dtype=torch.float64, device="cuda")
    res = P.solve(torch.from_numpy(f).cuda(), x, rtol=1e-8)
    xs = x.cpu().numpy()
    assert res["max_true_rel_residual"] <= 1e-8
    for i in range(0, nprob, max(1, nprob // 7)):
        rp, c, val = oracle.poisson_csr(k[i])
        ref = oracle.cg(rp, c, val, f[i].ravel(), rtol=1e-8, max_iter=20000)
        assert abs(int(res["iterations"][i]) - ref["iters"]) <= 2
        assert np.linalg.norm(xs[i].ravel() - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])


def test_warm_start_with_exact_solution_needs_no_iteration(ctx, oracle):
    from paper_2204_02064_gb300 import api
    nprob, ny, nx = 2, 20, 20
    k = _k(nprob, ny, nx, 5)
    u = inputs.uniform(6, nprob * ny * nx).reshape(nprob, ny, nx)
    P = api.Poisson(ctx, torch.from_numpy(k).cuda())
    b = torch.zeros(nprob, ny, nx, dtype=torch.float64, device="cuda")
    P.apply(torch.from_numpy(u).cuda(), b)
    x = torch.from_numpy(u).cuda()
    res = P.solve(b, x, rtol=1e-8)
    assert res["max_iterations"] == 0


def test_block_shapes_agree(ctx):
    """256- and 512-thread blocks solve the same problems to the tolerance
    with the same iteration counts (+-2: block sums in another order)."""
    from paper_2204_02064_gb300 import api
    nprob, ny, nx = 7, 40, 52
    k = _k(nprob, ny, nx, 5)
    f = 2.0 * inputs.uniform(6, nprob * ny * nx).reshape(nprob, ny, nx) - 1.0
    res = []
    for threads in (256, 512):
        P = api.Poisson(ctx, torch.from_numpy(k).cuda())
        P.set_rows_per_pass(4)  # the block shape applies to the 4-row kernel
        P.set_block_threads(threads)
        x = torch.zeros(nprob, ny, nx, dtype=torch.float64, device="cuda")
        r = P.solve(torch.from_numpy(f).cuda(), x, rtol=1e-8)
        assert r["max_true_rel_residual"] <= 1e-8
        res.append(r["iterations"])
    assert np.max(np.abs(res[0] - res[1])) <= 2


def test_scale_guess_matches_oracle(ctx, oracle):
    """x <- (<x,b>/<x,Ax>) x per problem, with A the oracle's CSR form of the
    operator; a zero guess stays zero and an exact solution is left as is."""
    from paper_2204_02064_gb300 import api
    nprob, ny, nx = 4, 29, 41
    k = _k(nprob, ny, nx, 7)
    f = 2.0 * inputs.uniform(8, nprob * ny * nx).reshape(nprob, ny, nx) - 1.0
    x = inputs.uniform(9, nprob * ny * nx).reshape(nprob, ny, nx) - 0.3
    x[3] = 0.0
    rp, c, val = oracle.poisson_csr(k[2])
    x[2] = oracle.cg(rp, c, val, f[2].ravel(), rtol=1e-13, max_iter=20000)["x"].reshape(ny, nx)
    P = api.Poisson(ctx, torch.from_numpy(k).cuda())
    xd = torch.from_numpy(x.copy()).cuda()
    P.scale_guess(torch.from_numpy(f).cuda(), xd)
    xs = xd.cpu().numpy()
    for i in range(3):
        rp, c, val = oracle.poisson_csr(k[i])
        ax = oracle.spmv(rp, c, val, x[i].ravel())
        alpha = oracle.dot(x[i].ravel(), f[i].ravel()) / oracle.dot(x[i].ravel(), ax)
        want = alpha * x[i]
        assert np.max(np.abs(xs[i] - want)) <= 1e-12 * np.max(np.abs(want))
        if i == 2:
            assert abs(alpha - 1.0) <= 1e-10
        else:  # the A-norm error against the solution does not grow
            u = oracle.cg(rp, c, val, f[i].ravel(), rtol=1e-12, max_iter=20000)["x"]
            def anorm(e):
                return oracle.dot(e, oracle.spmv(rp, c, val, e))
            assert anorm(u - xs[i].ravel()) <= anorm(u - x[i].ravel())
    assert not xs[3].any()
    P.close()


@pytest.mark.parametrize("rows", [1, 4])
@pytest.mark.parametrize("group", [2, 4, 8])
@pytest.mark.parametrize("nprob,ny,nx", [(5, 24, 31), (40, 37, 16)])
def test_block_groups_match_oracle(ctx, oracle, group, nprob, ny, nx, rows):
    """Rows of each problem split over a group of blocks (37 rows over 8
    blocks leaves some blocks one row block or none): every problem reaches
    the tolerance and agrees with the oracle's CG."""
    from paper_2204_02064_gb300 import api
    k = _k(nprob, ny, nx, 11)
    f = 2.0 * inputs.uniform(12, nprob * ny * nx).reshape(nprob, ny, nx) - 1.0
    P = api.Poisson(ctx, torch.from_numpy(k).cuda())
    P.set_rows_per_pass(rows)
    P.set_group(group)
    x = torch.zeros(nprob, ny, nx, dtype=torch.float64, device="cuda")
    res = P.solve(torch.from_numpy(f).cuda(), x, rtol=1e-8)
    xs = x.cpu().numpy()
    assert res["max_true_rel_residual"] <= 1e-8
    assert res["grid_blocks"] % group == 0
    for i in range(0, nprob, max(1, nprob // 5)):
        rp, c, val = oracle.poisson_csr(k[i])
        ref = oracle.cg(rp, c, val, f[i].ravel(), rtol=1e-8, max_iter=20000)
        assert abs(int(res["iterations"][i]) - ref["iters"]) <= 2
        assert np.linalg.norm(xs[i].ravel() - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])
    P.close()


def test_block_group_barrier_timeout_reported(ctx):
    """A group barrier that gives up at its first wait (timeout 0) ends the
    solve with BARRIER_TIMEOUT; the context stays usable."""
    from paper_2204_02064_gb300 import api
    nprob, ny, nx = 6, 32, 32
    k = _k(nprob, ny, nx, 13)
    f = torch.from_numpy(2.0 * inputs.uniform(14, nprob * ny * nx).reshape(nprob, ny, nx) - 1.0).cuda()
    P = api.Poisson(ctx, torch.from_numpy(k).cuda())
    P.set_group(2)
    x = torch.zeros(nprob, ny, nx, dtype=torch.float64, device="cuda")
    ctx.set_barrier_timeout(0)
    try:
        with pytest.raises(api.PerksError) as ei:
            P.solve(f, x, rtol=1e-8)
        assert ei.value.name == "BARRIER_TIMEOUT"
    finally:
        ctx.set_barrier_timeout(2_000_000_000)
    x.zero_()
    assert P.solve(f, x, rtol=1e-8)["max_true_rel_residual"] <= 1e-8
    with pytest.raises(api.PerksError) as ei:
        P.set_group(3)
    assert ei.value.name == "INVALID_ARG"
    P.close()


def test_automatic_block_groups(ctx):
    """By default problems of 64K cells and more get groups of 8 blocks (two
    per SM, one row per pass), smaller ones one block each."""
    from paper_2204_02064_gb300 import api
    for ny, nx, per in ((256, 256, 8), (64, 64, 1)):
        nprob = 3
        k = _k(nprob, ny, nx, 15)
        f = torch.from_numpy(2.0 * inputs.uniform(16, nprob * ny * nx).reshape(nprob, ny, nx) - 1.0).cuda()
        P = api.Poisson(ctx, torch.from_numpy(k).cuda())
        x = torch.zeros(nprob, ny, nx, dtype=torch.float64, device="cuda")
        res = P.solve(f, x, rtol=1e-8)
        assert res["grid_blocks"] == nprob * per
        assert res["max_true_rel_residual"] <= 1e-8
        P.close()


@pytest.mark.parametrize("group", [1, 4])
def test_one_row_per_pass_matches_oracle(ctx, oracle, group):
    """The 64-register kernel (one row per pass, two blocks per SM), with one
    block or a group of four per problem, agrees with the oracle's CG."""
    from paper_2204_02064_gb300 import api
    nprob, ny, nx = 9, 37, 45
    k = _k(nprob, ny, nx, 17)
    f = 2.0 * inputs.uniform(18, nprob * ny * nx).reshape(nprob, ny, nx) - 1.0
    P = api.Poisson(ctx, torch.from_numpy(k).cuda())
    P.set_rows_per_pass(1)
    P.set_group(group)
    x = torch.zeros(nprob, ny, nx, dtype=torch.float64, device="cuda")
    res = P.solve(torch.from_numpy(f).cuda(), x, rtol=1e-8)
    xs = x.cpu().numpy()
    assert res["max_true_rel_residual"] <= 1e-8
    for i in range(0, nprob, 4):
        rp, c, val = oracle.poisson_csr(k[i])
        ref = oracle.cg(rp, c, val, f[i].ravel(), rtol=1e-8, max_iter=20000)
        assert abs(int(res["iterations"][i]) - ref["iters"]) <= 2
        assert np.linalg.norm(xs[i].ravel() - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])
    with pytest.raises(api.PerksError):
        P.set_rows_per_pass(3)
    P.close()
