"""The Gaussian-random-field generator behind the Poisson coefficients:
sample variance and correlation against the squared-exponential covariance
it is built to have."""
import numpy as np

from paper_2204_02064_gb300 import inputs


def test_grf_variance_and_correlation():
    ell, sigma = 6.0, 1.3
    g = inputs.grf(48, 300, seed=9, ell=ell, sigma=sigma)
    assert abs(g.mean()) < 0.05 * sigma
    assert abs(g.var() / sigma ** 2 - 1.0) < 0.05
    for lag in (3, 6, 12):
        cx = np.mean(g[:, :, :-lag] * g[:, :, lag:]) / sigma ** 2
        cy = np.mean(g[:, :-lag, :] * g[:, lag:, :]) / sigma ** 2
        expect = np.exp(-lag ** 2 / (2 * ell ** 2))
        assert abs(cx - expect) < 0.05 and abs(cy - expect) < 0.05


def test_grf_is_seeded_and_pairs_independent():
    a = inputs.grf(32, 4, seed=1, ell=4.0)
    b = inputs.grf(32, 4, seed=1, ell=4.0)
    assert np.array_equal(a, b)
    assert abs(np.corrcoef(a[0].ravel(), a[1].ravel())[0, 1]) < 0.2


def test_poisson_problem_ranges():
    k, f = inputs.poisson_problems(32, 3, ell=4.0)
    assert k.shape == f.shape == (3, 32, 32)
    assert np.all(k > 0) and np.all(f >= -1) and np.all(f < 1)
