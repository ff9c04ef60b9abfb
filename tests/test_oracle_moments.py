"""Pins the oracle's output measures (the paper's output-measure equation): on the AR(1)
model the prediction filter p(x_t | y_1..t-1) and the filter p(x_t | y_1..t) are Gaussian
with the Kalman recursion's means and variances (written here, independently of the
oracle).  The particle estimates of E[x_t] and E[x_t^2], averaged over independent runs, match
them within Monte-Carlo error; a filter of one island (m = 1) gives the same kind of estimate;
and the prediction moments at t = 1 are the prior's."""
import numpy as np

import oracle
import synth


def _kalman_moments(theta, y):
    a, sv, sw, s0 = (float(v) for v in theta)
    mean, var = 0.0, s0 * s0
    out = np.zeros((len(y), 2, 2))
    for t, yt in enumerate(y):
        mean, var = a * mean, a * a * var + sv * sv          # predict x_t
        out[t, 0] = (mean, var + mean * mean)
        k = var / (var + sw * sw)                             # update with y_t
        mean, var = mean + k * (yt - mean), (1 - k) * var
        out[t, 1] = (mean, var + mean * mean)
    return out


def test_moments_match_kalman_ar1():
    th = synth.AR1_THETA
    y = synth.ar1_observations(15, seed=1)
    ref = _kalman_moments(th, y)
    runs = np.array([oracle.airpf(synth.MODEL_AR1, th, y, m=16, M=128, mode=oracle.MODE_ADAPTIVE, tau=0.5,
                                  seed=3, chain=r, record=False, moments=True)["moments"][:, :, :, 0]
                     for r in range(24)])
    mean = runs.mean(axis=0)
    se = runs.std(axis=0, ddof=1) / np.sqrt(runs.shape[0])
    assert np.all(np.abs(mean - ref) < 5 * se + 2e-3), np.max(np.abs(mean - ref) / (se + 1e-12))


def test_prediction_at_step_one_is_the_prior():
    th = np.array([0.9, 1.0, 1.0, 2.0])
    y = synth.ar1_observations(3, seed=1)
    mom = oracle.airpf(synth.MODEL_AR1, th, y, m=64, M=256, seed=1, record=False, moments=True)["moments"]
    # x_1 = 0.9 x_0 + v with x_0 ~ N(0, 4): mean 0, variance 0.81 * 4 + 1
    n = 64 * 256
    assert abs(mom[0, 0, 0, 0]) < 5 * np.sqrt(4.24 / n)
    assert abs(mom[0, 0, 1, 0] - 4.24) < 5 * 4.24 * np.sqrt(2.0 / n)


def test_single_island_moments_match_kalman():
    th = synth.AR1_THETA
    y = synth.ar1_observations(10, seed=1)
    ref = _kalman_moments(th, y)
    runs = np.array([oracle.airpf(synth.MODEL_AR1, th, y, m=1, M=2048, seed=5, chain=r, record=False,
                                  moments=True)["moments"][:, :, :, 0] for r in range(16)])
    mean = runs.mean(axis=0)
    se = runs.std(axis=0, ddof=1) / np.sqrt(runs.shape[0])
    assert np.all(np.abs(mean - ref) < 5 * se + 2e-3)
