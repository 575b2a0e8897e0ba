"""Pins of the CG oracle (Sec. 2.2.2) and of the sparse SPD generator against
textbook properties and library routines, not against the oracle itself:

* finite termination: on random SPD systems with n <= 8, n iterations give the
  dense-solve answer;
* the A-norm error ||x* - x_k||_A is non-increasing (x* by Cholesky);
* a diagonal matrix with k distinct eigenvalues converges in k iterations;
* the first iteration equals its closed form (alpha_0 = b.b / b.Ab);
* SpMV equals a dense matrix-vector product;
* on the synthetic SPD matrix, CG and the FP32-IR variant reach the requested
  true residual and agree with a sparse direct solve;
* an indefinite system reports breakdown.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from paper_2204_02064_gb300 import inputs


def _dense_to_csr(A):
    S = scipy.sparse.csr_matrix(A)
    S.sort_indices()
    return S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64)


def _rand_spd(n, seed, cond=20.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (Q * ev) @ Q.T


@pytest.mark.parametrize("n,seed", [(2, 0), (5, 1), (8, 2)])
def test_exact_in_n_steps(oracle, n, seed):
    A = _rand_spd(n, seed)
    A = 0.5 * (A + A.T)
    b = np.random.default_rng(seed + 10).standard_normal(n)
    rp, c, v = _dense_to_csr(A)
    res = oracle.cg(rp, c, v, b, rtol=0.0, max_iter=n, max_restarts=0)
    xs = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A), b)
    assert res["iters"] == n
    assert np.linalg.norm(res["x"] - xs) <= 1e-10 * np.linalg.norm(xs)
    assert res["true_rel"] <= 1e-10


def test_a_norm_error_monotone(oracle):
    n = 40
    A = _rand_spd(n, 7, cond=500.0)
    A = 0.5 * (A + A.T)
    b = np.random.default_rng(3).standard_normal(n)
    rp, c, v = _dense_to_csr(A)
    xs = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A), b)
    errs = []
    for k in range(0, 41):
        x = oracle.cg(rp, c, v, b, rtol=0.0, max_iter=k, max_restarts=0)["x"]
        e = xs - x
        errs.append(np.sqrt(e @ A @ e))
    errs = np.array(errs)
    assert np.all(errs[1:] <= errs[:-1] * (1 + 1e-10))
    assert errs[-1] < 1e-3 * errs[0]


def test_distinct_eigenvalues_bound_iterations(oracle):
    n = 30
    d = np.array([1.0, 4.0, 9.0] * 10)
    rp, c, v = _dense_to_csr(np.diag(d))
    b = inputs.cg_rhs(n, 5)
    res = oracle.cg(rp, c, v, b, rtol=1e-12, max_iter=100, max_restarts=0)
    assert res["iters"] <= 3 + 1 and res["status"] == 0
    assert np.max(np.abs(res["x"] - b / d)) <= 1e-12


def test_first_iteration_closed_form(oracle):
    A = _rand_spd(6, 4)
    A = 0.5 * (A + A.T)
    b = np.arange(1.0, 7.0)
    rp, c, v = _dense_to_csr(A)
    res = oracle.cg(rp, c, v, b, rtol=0.0, max_iter=1, max_restarts=0, trace_len=1)
    Ab = A @ b
    alpha0 = (b @ b) / (b @ Ab)
    r1 = b - alpha0 * Ab
    beta0 = (r1 @ r1) / (b @ b)
    assert res["trace"][0, 0] == pytest.approx(alpha0, rel=1e-14)
    assert res["trace"][0, 1] == pytest.approx(beta0, rel=1e-12)
    assert res["trace"][0, 2] == pytest.approx(r1 @ r1, rel=1e-12)
    assert np.allclose(res["x"], alpha0 * b, rtol=1e-14, atol=0)


def test_spmv_matches_dense(oracle):
    rp, c, v = inputs.csr_spd_matrix(300, 17)
    A = scipy.sparse.csr_matrix((v, c, rp), shape=(300, 300)).toarray()
    x = inputs.cg_rhs(300, 9)
    assert np.max(np.abs(oracle.spmv(rp, c, v, x) - A @ x)) <= 1e-12
    assert oracle.dot(x, x) == pytest.approx(float(x @ x), rel=1e-14)


def test_generator_is_symmetric_and_dominant():
    n = 5000
    rp, c, v = inputs.csr_spd_matrix(n, 123)
    A = scipy.sparse.csr_matrix((v, c, rp), shape=(n, n))
    assert (A - A.T).count_nonzero() == 0
    diag = A.diagonal()
    off = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(diag)
    assert np.allclose(diag, 1.05 * off, rtol=1e-12)
    assert np.all(v[c == np.repeat(np.arange(n), np.diff(rp))] > 0)
    offd = v[c != np.repeat(np.arange(n), np.diff(rp))]
    assert offd.min() >= -1.0 and offd.max() < 0.0
    counts = np.diff(rp) - 1
    assert counts.min() >= 3 and 30 <= counts.mean() <= 40
    # columns sorted within rows
    for i in range(0, n, 997):
        assert np.all(np.diff(c[rp[i]:rp[i + 1]]) > 0)


@pytest.fixture(scope="module")
def small_system():
    n = 4000
    rp, c, v = inputs.csr_spd_matrix(n, 31)
    b = inputs.cg_rhs(n, 31)
    A = scipy.sparse.csr_matrix((v, c, rp), shape=(n, n)).tocsc()
    xs = scipy.sparse.linalg.spsolve(A, b)
    return rp, c, v, b, xs


def test_cg_synthetic_reaches_tolerance(oracle, small_system):
    rp, c, v, b, xs = small_system
    res = oracle.cg(rp, c, v, b, rtol=1e-10, max_iter=2000)
    assert res["status"] == 0
    assert res["true_rel"] <= 1e-10
    assert np.linalg.norm(res["x"] - xs) <= 1e-8 * np.linalg.norm(xs)


def test_cg_fp32_ir_reaches_tolerance(oracle, small_system):
    rp, c, v, b, xs = small_system
    res = oracle.cg_fp32_ir(rp, c, v, b, rtol=1e-10, inner_rtol=1e-4)
    assert res["status"] == 0
    assert res["true_rel"] <= 1e-10
    assert res["outer_iters"] >= 2
    assert np.linalg.norm(res["x"] - xs) <= 1e-8 * np.linalg.norm(xs)


def test_breakdown_on_indefinite(oracle):
    rp, c, v = _dense_to_csr(np.diag([1.0, -1.0]))
    res = oracle.cg(rp, c, v, np.array([1.0, 1.0]), rtol=1e-12, max_iter=10)
    assert res["status"] == oracle.BREAKDOWN


def test_zero_rhs_converges_immediately(oracle):
    rp, c, v = inputs.csr_spd_matrix(50, 1)
    res = oracle.cg(rp, c, v, np.zeros(50), rtol=1e-10, max_iter=10)
    assert res["status"] == 0 and res["iters"] == 0 and np.all(res["x"] == 0)
