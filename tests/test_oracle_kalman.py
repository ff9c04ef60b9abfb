"""Pins the Kalman-filter likelihood (exact Z for linear-Gaussian models) to the
closed-form joint Gaussian density of y_{1:T}, evaluated by scipy."""
import numpy as np

import synth
from oracle import kalman


def test_scalar_kalman_matches_joint_gaussian():
    y = synth.ar1_observations(12, seed=1)
    for th in ([0.9, 1.0, 1.0, 1.0], [0.3, 0.7, 1.4, 2.0], [-0.8, 1.2, 0.5, 0.6]):
        a, sv, sw, s0 = th
        want = kalman.joint_gaussian_loglik([[a]], [[1.0]], [[sv * sv]], [[sw * sw]], [0.0],
                                            [[s0 * s0]], y.reshape(-1, 1))
        assert np.isclose(kalman.ar1_loglik(th, y), want, rtol=1e-11)


def test_multivariate_kalman_matches_joint_gaussian():
    dx, dy = 3, 2
    A, C, md = synth.lg_model(dx, dy, seed=3)
    th = synth.lg_theta(A, q=0.2, r=0.6)
    y = synth.lg_observations(A, C, 0.2, 0.6, 8, seed=3)
    want = kalman.joint_gaussian_loglik(A, C, 0.2 * np.eye(dx), 0.6 * np.eye(dy), np.zeros(dx),
                                        np.eye(dx), y.reshape(-1, dy))
    assert np.isclose(kalman.lg_loglik(th, md, y, dx, dy), want, rtol=1e-11)


def test_posterior_grid_is_normalised():
    y = synth.ar1_observations(100, seed=1)
    grid, dens, mean, var = kalman.ar1_posterior_grid(y)
    assert np.isclose(np.trapezoid(dens, grid), 1.0)
    assert 0.0 < var < 0.05 and -1.0 < mean < 1.0


def test_grid_recursion_matches_matrix_kalman():
    y = synth.ar1_observations(50, seed=1)
    a = np.array([-0.7, 0.1, 0.9])
    got = kalman.ar1_loglik_grid(a, y)
    want = [kalman.ar1_loglik([v, 1.0, 1.0, 1.0], y) for v in a]
    assert np.allclose(got, want, rtol=1e-12)
