"""Pins of the variable-coefficient Poisson operator and of the warm-start
network's forward pass in the oracle, against independent formulations."""
import numpy as np
import pytest
import scipy.signal
import scipy.sparse
import scipy.sparse.linalg

from paper_2204_02064_gb300 import inputs


def test_constant_k_is_scaled_laplacian(oracle):
    nx, ny, kc = 7, 5, 2.5
    rp, c, v = oracle.poisson_csr(np.full((ny, nx), kc))
    A = scipy.sparse.csr_matrix((v, c, rp), shape=(nx * ny, nx * ny)).toarray()
    # Dirichlet 0 through ghost cells at distance 1: the 1-D operator is tridiag(-1, 2, -1)
    T = lambda m: 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    L = np.kron(np.eye(ny), T(nx)) + np.kron(T(ny), np.eye(nx))
    assert np.allclose(A, kc * L, rtol=0, atol=1e-14)


def test_operator_symmetric_spd_and_harmonic_faces(oracle):
    k = np.exp(inputs.uniform(3, 6 * 9).reshape(6, 9) * 3 - 1.5)
    rp, c, v = oracle.poisson_csr(k)
    A = scipy.sparse.csr_matrix((v, c, rp), shape=(54, 54)).toarray()
    assert np.allclose(A, A.T, rtol=0, atol=0)
    assert np.min(np.linalg.eigvalsh(A)) > 0
    # off-diagonal between (1,2) and (2,2): harmonic mean of the two k
    c1, c2 = 2 * 9 + 1, 2 * 9 + 2
    assert A[c1, c2] == pytest.approx(-2 * k[2, 1] * k[2, 2] / (k[2, 1] + k[2, 2]), rel=1e-15)
    # a row's entries sum to the boundary-face coefficients (zero inside)
    rs = A.sum(axis=1).reshape(6, 9)
    assert np.allclose(rs[2:4, 2:7], 0, atol=1e-13)
    assert rs[0, 4] == pytest.approx(k[0, 4], rel=1e-12)


def test_manufactured_solution(oracle):
    """A u = f with f assembled from a known u: CG recovers u."""
    k = np.exp(inputs.uniform(4, 24 * 20).reshape(20, 24) - 0.5)
    rp, c, v = oracle.poisson_csr(k)
    u = inputs.uniform(5, 480)
    f = oracle.spmv(rp, c, v, u)
    res = oracle.cg(rp, c, v, f, rtol=1e-12, max_iter=5000)
    assert np.max(np.abs(res["x"] - u)) <= 1e-9


def test_conv2d_matches_scipy(oracle):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 11, 13))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    for dil in (1, 2, 3):
        out = oracle.conv2d(x, w, b, dil)
        for co in range(4):
            ref = np.full((11, 13), b[co])
            for ci in range(3):
                kk = np.zeros((2 * dil + 1, 2 * dil + 1))
                kk[::dil, ::dil] = w[co, ci]
                ref += scipy.signal.correlate2d(x[ci], kk, mode="same", boundary="fill")
            assert np.allclose(out[co], ref, atol=1e-12)


def test_warmnet_forward_composes_layers(oracle):
    rng = np.random.default_rng(1)
    c0, c1, h, w = 2, 4, 9, 10
    dil = (1, 2, 1, 3)
    shapes = [(c1, c0), (c1, c1), (c1, c1), (1, c1)]
    params, layers = [], []
    for co, ci in shapes:
        W = rng.standard_normal((co, ci, 3, 3)) * 0.3
        B = rng.standard_normal(co) * 0.1
        params += [W.ravel(), B]
        layers.append((W, B))
    params = np.concatenate(params)
    x = rng.standard_normal((c0, h, w))
    out = oracle.warmnet_forward(params, x, c1, dil)
    y = x
    for l, (W, B) in enumerate(layers):
        y = oracle.conv2d(y, W, B, dil[l])
        if l < 3:
            y = np.maximum(y, 0)
    assert np.allclose(out, y[0], atol=1e-13)


def _tiny_net(rng, c0, c1, scale=0.4):
    shapes = [(c1, c0), (c1, c1), (c1, c1), (1, c1)]
    parts = []
    for co, ci in shapes:
        parts += [rng.standard_normal(co * ci * 9) * scale, rng.standard_normal(co) * 0.1]
    return np.concatenate(parts)


def test_warmnet_grad_matches_central_differences(oracle):
    """Every parameter's derivative of the mean squared error, by central
    finite differences of the oracle's forward pass in fp64 (the network is
    piecewise linear in each parameter, so away from a ReLU kink the central
    difference is exact up to rounding), on a 2x8x8 input."""
    rng = np.random.default_rng(11)
    c0, c1, h, w = 2, 4, 8, 8
    dil = (1, 2, 1, 2)
    params = _tiny_net(rng, c0, c1)
    x = rng.standard_normal((2, c0, h, w))
    t = rng.standard_normal((2, h, w))
    loss, g = oracle.warmnet_grad(params, x, t, c1, dil)

    def L(p):
        return sum(np.mean((oracle.warmnet_forward(p, x[i], c1, dil) - t[i]) ** 2) for i in range(2)) / 2

    assert loss == pytest.approx(L(params), rel=1e-13)
    eps = 1e-6
    fd = np.empty_like(params)
    for i in range(params.size):
        e = np.zeros_like(params)
        e[i] = eps
        fd[i] = (L(params + e) - L(params - e)) / (2 * eps)
    err = np.abs(fd - g)
    assert np.max(err) <= 1e-7 * np.max(np.abs(g))
    assert np.count_nonzero(g) > 0.9 * g.size


def test_warmnet_grad_zero_at_exact_fit(oracle):
    """Targets produced by the network itself: loss 0, gradient 0."""
    rng = np.random.default_rng(12)
    c0, c1, h, w = 2, 3, 6, 7
    params = _tiny_net(rng, c0, c1)
    x = rng.standard_normal((3, c0, h, w))
    t = np.stack([oracle.warmnet_forward(params, x[i], c1) for i in range(3)])
    loss, g = oracle.warmnet_grad(params, x, t, c1)
    assert loss == 0.0 and np.all(g == 0.0)
