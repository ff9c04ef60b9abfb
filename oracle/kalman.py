"""Exact marginal likelihoods of linear-Gaussian state-space models -- TEST INFRASTRUCTURE.

For linear-Gaussian models the Feynman-Kac normalising constant gamma_T(1) of
Section 1.2 (eq. (2)) is the Gaussian marginal likelihood p(y_{1:T}), computed
exactly by the Kalman filter.  Theorem 1 states E[Z^N_T] = Z_T, so these
values are the targets of the lack-of-bias checks.

Time indexing follows the rest of the repository: x_0 ~ prior, y_t observed
at x_t for t = 1..T.
"""
from __future__ import annotations

import numpy as np


def kalman_loglik(A, C, Q, R, m0, P0, y) -> float:
    """log p(y_{1:T}) for x_t = A x_{t-1} + N(0,Q), y_t = C x_t + N(0,R), x_0 ~ N(m0,P0).

    y has shape (T, dy)."""
    A, C, Q, R = (np.atleast_2d(np.asarray(v, dtype=np.float64)) for v in (A, C, Q, R))
    m = np.atleast_1d(np.asarray(m0, dtype=np.float64)).copy()
    P = np.atleast_2d(np.asarray(P0, dtype=np.float64)).copy()
    y = np.asarray(y, dtype=np.float64).reshape(len(y), -1)
    ll = 0.0
    for yt in y:
        m = A @ m                       # predict
        P = A @ P @ A.T + Q
        S = C @ P @ C.T + R             # innovation covariance
        e = yt - C @ m
        L = np.linalg.cholesky(S)
        z = np.linalg.solve(L, e)
        ll += -0.5 * (len(yt) * np.log(2 * np.pi) + 2 * np.sum(np.log(np.diag(L))) + z @ z)
        K = np.linalg.solve(S, C @ P).T  # gain P C^T S^-1 (S symmetric)
        m = m + K @ e
        P = P - K @ C @ P
        P = 0.5 * (P + P.T)
    return float(ll)


def ar1_loglik(theta, y) -> float:
    """AR(1) model of synth: theta = [a, sigma_v, sigma_w, sigma_0]."""
    a, sv, sw, s0 = (float(v) for v in theta)
    return kalman_loglik([[a]], [[1.0]], [[sv * sv]], [[sw * sw]], [0.0], [[s0 * s0]],
                         np.asarray(y).reshape(-1, 1))


def lg_loglik(theta, model_data, y, dx, dy) -> float:
    """LGSSM of synth: theta = [diag(A), log q, log r], model_data = [A, C]."""
    theta = np.asarray(theta, dtype=np.float64)
    A = np.asarray(model_data[: dx * dx], dtype=np.float64).reshape(dx, dx).copy()
    C = np.asarray(model_data[dx * dx: dx * dx + dy * dx], dtype=np.float64).reshape(dy, dx)
    A[np.diag_indices(dx)] = theta[:dx]
    q, r = np.exp(theta[dx]), np.exp(theta[dx + 1])
    return kalman_loglik(A, C, q * np.eye(dx), r * np.eye(dy), np.zeros(dx), np.eye(dx),
                         np.asarray(y).reshape(-1, dy))


def joint_gaussian_loglik(A, C, Q, R, m0, P0, y) -> float:
    """Closed form used to pin kalman_loglik: stack y_{1:T} as one Gaussian
    vector, build its mean and covariance from the model equations directly,
    and evaluate the density with scipy."""
    from scipy.stats import multivariate_normal
    A, C, Q, R = (np.atleast_2d(np.asarray(v, dtype=np.float64)) for v in (A, C, Q, R))
    y = np.asarray(y, dtype=np.float64).reshape(len(y), -1)
    T, dy = y.shape
    dx = A.shape[0]
    # x_t = A^t x_0 + sum_{s=1..t} A^{t-s} v_s
    Apow = [np.eye(dx)]
    for _ in range(T):
        Apow.append(A @ Apow[-1])
    cov_x = np.zeros((T, T, dx, dx))
    for t in range(1, T + 1):
        for u in range(1, T + 1):
            c = Apow[t] @ np.asarray(P0) @ Apow[u].T
            for s in range(1, min(t, u) + 1):
                c = c + Apow[t - s] @ Q @ Apow[u - s].T
            cov_x[t - 1, u - 1] = c
    mean = np.concatenate([C @ (Apow[t] @ np.asarray(m0, dtype=np.float64)) for t in range(1, T + 1)])
    cov = np.zeros((T * dy, T * dy))
    for t in range(T):
        for u in range(T):
            blk = C @ cov_x[t, u] @ C.T
            if t == u:
                blk = blk + R
            cov[t * dy:(t + 1) * dy, u * dy:(u + 1) * dy] = blk
    return float(multivariate_normal(mean=mean, cov=cov).logpdf(y.ravel()))


def ar1_loglik_grid(a_values, y, sv=1.0, sw=1.0, s0=1.0) -> np.ndarray:
    """The scalar Kalman recursion of kalman_loglik run for many AR coefficients at once."""
    a = np.asarray(a_values, dtype=np.float64)
    m = np.zeros_like(a)
    P = np.full_like(a, s0 * s0)
    ll = np.zeros_like(a)
    for yt in np.asarray(y, dtype=np.float64).ravel():
        m = a * m
        P = a * a * P + sv * sv
        S = P + sw * sw
        e = yt - m
        ll += -0.5 * (np.log(2 * np.pi * S) + e * e / S)
        K = P / S
        m = m + K * e
        P = P - K * P
    return ll


def ar1_posterior_grid(y, lo=-1.0, hi=1.0, n=4001, theta_rest=(1.0, 1.0, 1.0)):
    """Posterior of the AR coefficient a under a U(lo, hi) prior, by quadrature
    of the exact likelihood on a grid.  Returns (grid, density, mean, var)."""
    grid = np.linspace(lo, hi, n)
    ll = ar1_loglik_grid(grid, y, *theta_rest)
    w = np.exp(ll - ll.max())
    dens = w / np.trapezoid(w, grid)
    mean = np.trapezoid(grid * dens, grid)
    var = np.trapezoid((grid - mean) ** 2 * dens, grid)
    return grid, dens, float(mean), float(var)
