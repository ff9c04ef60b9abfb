"""Seeded synthetic inputs for the AIRPF workloads.

This module is shared by the CUDA path, its tests, the bench and the CPU
oracle.  It only *simulates data* from the state-space models (the problem
statement of Section 1.2, eq. (1)) with NumPy's PCG64 generator; it holds none
of the particle filter's arithmetic (no weighting, resampling, interaction or
likelihood estimation).

Model parameter vectors (theta) are laid out per model as follows; the same
layout is used by the C-ABI and by the oracle:

    AR1   : [a, sigma_v, sigma_w, sigma_0]
            x_0 ~ N(0, sigma_0^2), x_t = a x_{t-1} + sigma_v v_t, y_t = x_t + sigma_w w_t
    SV    : [mu, phi, sigma]
            x_0 ~ N(mu, sigma^2/(1-phi^2)), x_t = mu + phi (x_{t-1}-mu) + sigma v_t,
            y_t = exp(x_t/2) w_t
    NGM   : [q, r, p0]   (variances)
            x_0 ~ N(0, p0), x_t = x/2 + 25 x/(1+x^2) + 8 cos(1.2 t) + sqrt(q) v_t,
            y_t = x_t^2/20 + sqrt(r) w_t
    LGSSM : [A_11, ..., A_dd, log q, log r]  with model data [A (dx*dx), C (dy*dx)]
            x_0 ~ N(0, I), x_t = A_theta x_{t-1} + sqrt(q) v_t, y_t = C x_t + sqrt(r) w_t,
            A_theta = A with its diagonal replaced by theta[:dx]
    TOY   : [p_stay, p_correct]  (binary HMM of Section 4.1)
            x_0 ~ U{0,1}, x_t = x_{t-1} w.p. p_stay, y_t = x_t w.p. p_correct

Observations are indexed t = 1..T (array index t-1); x_0 is the prior draw.
"""
from __future__ import annotations

import numpy as np

MODEL_AR1, MODEL_SV, MODEL_NGM, MODEL_LGSSM, MODEL_TOY, MODEL_CP = 0, 1, 2, 3, 4, 5
MODEL_NAMES = {MODEL_AR1: "ar1", MODEL_SV: "sv", MODEL_NGM: "ngm",
               MODEL_LGSSM: "lgssm", MODEL_TOY: "toy", MODEL_CP: "changepoint"}

AR1_THETA = np.array([0.9, 1.0, 1.0, 1.0])
SV_THETA = np.array([-1.0, 0.95, 0.3])
NGM_THETA = np.array([10.0, 1.0, 5.0])
TOY_THETA = np.array([0.75, 0.75])
# change-point model (p, alpha, beta): a jump every 50 days on average to a rate drawn from
# Beta(2, 20) (mean 0.09)
CP_THETA = np.array([0.02, 2.0, 20.0])


def theta_dim(model: int, dx: int = 1) -> int:
    return {MODEL_AR1: 4, MODEL_SV: 3, MODEL_NGM: 3, MODEL_TOY: 2, MODEL_CP: 3}.get(model, dx + 2)


def ar1_observations(T: int, seed: int = 1, theta=AR1_THETA) -> np.ndarray:
    a, sv, sw, s0 = (float(v) for v in theta)
    rng = np.random.default_rng(seed)
    x = s0 * rng.standard_normal()
    y = np.empty(T)
    for t in range(T):
        x = a * x + sv * rng.standard_normal()
        y[t] = x + sw * rng.standard_normal()
    return y


def sv_observations(T: int, seed: int = 2, theta=SV_THETA) -> np.ndarray:
    mu, phi, sigma = (float(v) for v in theta)
    rng = np.random.default_rng(seed)
    x = mu + sigma / np.sqrt(1.0 - phi * phi) * rng.standard_normal()
    y = np.empty(T)
    for t in range(T):
        x = mu + phi * (x - mu) + sigma * rng.standard_normal()
        y[t] = np.exp(0.5 * x) * rng.standard_normal()
    return y


def ngm_observations(T: int, seed: int = 5, theta=NGM_THETA) -> np.ndarray:
    q, r, p0 = (float(v) for v in theta)
    rng = np.random.default_rng(seed)
    x = np.sqrt(p0) * rng.standard_normal()
    y = np.empty(T)
    for t in range(1, T + 1):
        x = 0.5 * x + 25.0 * x / (1.0 + x * x) + 8.0 * np.cos(1.2 * t) + np.sqrt(q) * rng.standard_normal()
        y[t - 1] = x * x / 20.0 + np.sqrt(r) * rng.standard_normal()
    return y


def lg_model(dx: int = 8, dy: int = 4, seed: int = 4, rho: float = 0.95):
    """A = (0.8 I + 0.05 G) rescaled to spectral radius rho, C ~ N(0, 1/dx).

    Returns (A, C, model_data) with model_data = concat(A.ravel(), C.ravel())."""
    rng = np.random.default_rng(seed)
    A = 0.8 * np.eye(dx) + 0.05 * rng.standard_normal((dx, dx))
    A *= rho / np.max(np.abs(np.linalg.eigvals(A)))
    C = rng.standard_normal((dy, dx)) / np.sqrt(dx)
    return A, C, np.concatenate([A.ravel(), C.ravel()])


def lg_theta(A: np.ndarray, q: float = 0.1, r: float = 0.5) -> np.ndarray:
    return np.concatenate([np.diag(A), [np.log(q), np.log(r)]])


def lg_observations(A, C, q: float, r: float, T: int, seed: int = 4) -> np.ndarray:
    """y[t-1, :] for t = 1..T, flattened row-major to T*dy."""
    rng = np.random.default_rng(seed + 1000)
    dx, dy = A.shape[0], C.shape[0]
    x = rng.standard_normal(dx)
    y = np.empty((T, dy))
    for t in range(T):
        x = A @ x + np.sqrt(q) * rng.standard_normal(dx)
        y[t] = C @ x + np.sqrt(r) * rng.standard_normal(dy)
    return y.ravel()


def toy_observations(T: int, seed: int = 3, theta=TOY_THETA) -> np.ndarray:
    stay, correct = (float(v) for v in theta)
    rng = np.random.default_rng(seed)
    x = int(rng.random() < 0.5)
    y = np.empty(T)
    for t in range(T):
        if rng.random() >= stay:
            x = 1 - x
        y[t] = float(x if rng.random() < correct else 1 - x)
    return y


def cp_observations(T: int, seed: int = 6, theta=CP_THETA, n_lo: int = 400, n_hi: int = 1200) -> np.ndarray:
    """Synthetic daily counts for the change-point model: n_t articles a day, uniform on
    [n_lo, n_hi], of which k_t ~ Binomial(n_t, x_t) carry the keyword; x_0 ~ Beta(alpha, beta),
    and each day x jumps with probability p to a fresh Beta(alpha, beta) draw.  Returns
    (k_1, n_1, k_2, n_2, ...) (d_y = 2)."""
    p, a, b = (float(v) for v in theta)
    rng = np.random.default_rng(seed)
    x = rng.beta(a, b)
    y = np.empty((T, 2))
    for t in range(T):
        if rng.random() < p:
            x = rng.beta(a, b)
        n = int(rng.integers(n_lo, n_hi + 1))
        y[t] = (rng.binomial(n, x), n)
    return y.ravel()


def batched_sv_thetas(B: int, seed: int = 7) -> tuple[np.ndarray, int]:
    """theta_c ~ N((-1, .95, .3), diag(.1, .01, .05)^2), redrawn until |phi|<1, sigma>0.

    Returns (theta[B, 3], number of redraws)."""
    rng = np.random.default_rng(seed)
    mean, sd = SV_THETA, np.array([0.1, 0.01, 0.05])
    out = np.empty((B, 3))
    redraws = 0
    for c in range(B):
        while True:
            th = mean + sd * rng.standard_normal(3)
            if abs(th[1]) < 1.0 and th[2] > 0.0:
                break
            redraws += 1
        out[c] = th
    return out, redraws


def batched_sizes(B: int, seed: int = 8) -> tuple[np.ndarray, np.ndarray]:
    """m_c ~ U{64,256,1024,4096}, M_c ~ U{32,128,512,1024}."""
    rng = np.random.default_rng(seed)
    m = rng.choice(np.array([64, 256, 1024, 4096]), size=B)
    M = rng.choice(np.array([32, 128, 512, 1024]), size=B)
    return m.astype(np.int32), M.astype(np.int32)


# Workloads quoted by the benchmark configurations, with their sizes.
WORKLOADS = {
    "ar1_m16_M64_T100": dict(model=MODEL_AR1, dx=1, dy=1, m=16, M=64, T=100,
                             theta=AR1_THETA, y=lambda: ar1_observations(100, 1)),
    "sv_m1024_M256_T1000": dict(model=MODEL_SV, dx=1, dy=1, m=1024, M=256, T=1000,
                                theta=SV_THETA, y=lambda: sv_observations(1000, 2)),
    "ngm_m65536_M256_T1000": dict(model=MODEL_NGM, dx=1, dy=1, m=65536, M=256, T=1000,
                                  theta=NGM_THETA, y=lambda: ngm_observations(1000, 5)),
    "changepoint_m64_M200_T523": dict(model=MODEL_CP, dx=1, dy=2, m=64, M=200, T=523,
                                      theta=CP_THETA, y=lambda: cp_observations(523, 6)),
    "changepoint_m64_M500_T523": dict(model=MODEL_CP, dx=1, dy=2, m=64, M=500, T=523,
                                      theta=CP_THETA, y=lambda: cp_observations(523, 6)),
}
