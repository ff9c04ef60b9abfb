"""Pins the oracle's gradient references: the transition and prior densities, log Z with a
fixed lineage, its central-difference gradient, and the Fisher-identity score along the
lineages.

* log f and log pi_0 equal scipy's normal densities for every differentiable model;
* log Z with the run's own lineage and s* held fixed reproduces the run's log Z
  (stage-by-stage cascade against block means: rounding only);
* with one island of one particle the filter is a single path: log Z with the lineage
  fixed is the sum of the path's observation log-densities, whose theta-gradient follows
  from differentiating the AR(1) recursion by hand, and the Fisher score is the
  closed-form score of the path's joint density;
* the Fisher score estimates the Kalman score (its expectation over runs, within
  Monte-Carlo error) on the AR(1) model.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
import synth
from oracle import kalman


@pytest.mark.parametrize("model,theta,xp,x", [
    (synth.MODEL_AR1, [0.9, 1.3, 0.7, 2.0], [0.4], [1.1]),
    (synth.MODEL_SV, [-1.0, 0.95, 0.3], [-0.7], [-1.2]),
    (synth.MODEL_NGM, [10.0, 1.0, 5.0], [2.5], [4.0]),
])
def test_scalar_transition_and_prior_densities(model, theta, xp, x):
    th = np.asarray(theta)
    if model == synth.MODEL_AR1:
        mean, sd, pm, psd = th[0] * xp[0], th[1], 0.0, th[3]
    elif model == synth.MODEL_SV:
        mean, sd = th[0] + th[1] * (xp[0] - th[0]), th[2]
        pm, psd = th[0], th[2] / np.sqrt(1 - th[1] ** 2)
    else:
        t = 3
        mean = xp[0] / 2 + 25 * xp[0] / (1 + xp[0] ** 2) + 8 * np.cos(1.2 * t)
        sd, pm, psd = np.sqrt(th[0]), 0.0, np.sqrt(th[2])
    t = 3
    assert oracle.model_logf(model, th, xp, x, t=t) == pytest.approx(stats.norm.logpdf(x[0], mean, sd), rel=1e-12)
    assert oracle.model_logmu(model, th, x) == pytest.approx(stats.norm.logpdf(x[0], pm, psd), rel=1e-12)


def test_lgssm_transition_and_prior_densities():
    A, C, md = synth.lg_model(3, 2, seed=11)
    th = synth.lg_theta(A, q=0.1, r=0.5)
    Ad = A.copy()
    np.fill_diagonal(Ad, th[:3])
    xp = np.array([0.3, -0.2, 0.5])
    x = np.array([0.1, 0.4, -0.3])
    ref = stats.multivariate_normal.logpdf(x, Ad @ xp, 0.1 * np.eye(3))
    assert oracle.model_logf(synth.MODEL_LGSSM, th, xp, x, dx=3, dy=2, model_data=md) == pytest.approx(ref, rel=1e-12)
    ref0 = stats.multivariate_normal.logpdf(x, np.zeros(3), np.eye(3))
    assert oracle.model_logmu(synth.MODEL_LGSSM, th, x, dx=3, dy=2, model_data=md) == pytest.approx(ref0, rel=1e-12)


@pytest.mark.parametrize("mode", [oracle.MODE_ADAPTIVE, oracle.MODE_ALWAYS, oracle.MODE_NEVER])
def test_fixed_lineage_reproduces_the_run(mode):
    y = synth.ar1_observations(40, seed=1)
    kw = dict(m=8, M=16, seed=5, chain=2, iter=1)
    r = oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, mode=mode, tau=0.5, **kw)
    lz = oracle.logz_fixed(synth.MODEL_AR1, synth.AR1_THETA, y, r["anc"], r["sstar"], **kw)
    assert lz == pytest.approx(r["log_z"], rel=1e-12)


def _single_path(theta, y, seed=3):
    """x_0..x_T of one particle (m = M = 1) from the oracle's pinned model calls."""
    T = len(y)
    xs = [oracle.model_prior(synth.MODEL_AR1, theta, unit=0, seed=seed)]
    for t in range(1, T + 1):
        xs.append(oracle.model_step(synth.MODEL_AR1, theta, xs[-1], unit=0, t=t, seed=seed))
    return np.array([v[0] for v in xs])


def test_single_path_gradient_and_score_closed_form():
    y = synth.ar1_observations(25, seed=4)
    th = np.array([0.8, 1.2, 0.9, 1.5])
    a, sv, sw, s0 = th
    T = len(y)
    anc = np.zeros((T, 1), np.int32)
    sstar = np.ones(T, np.int32)
    kw = dict(m=1, M=1, seed=3)
    x = _single_path(th, y)
    # log Z with the lineage fixed: sum_t log g(y_t | x_t)
    lz = oracle.logz_fixed(synth.MODEL_AR1, th, y, anc, sstar, **kw)
    assert lz == pytest.approx(np.sum(stats.norm.logpdf(y, x[1:], sw)), rel=1e-12)
    # its gradient: x_t = a x_{t-1} + sv z_t, x_0 = s0 z_0 with z fixed
    z = (x[1:] - a * x[:-1]) / sv
    dx = np.zeros((4, T + 1))
    dx[3, 0] = x[0] / s0
    for t in range(1, T + 1):
        dx[:, t] = a * dx[:, t - 1]
        dx[0, t] += x[t - 1]
        dx[1, t] += z[t - 1]
    r = y - x[1:]
    grad = (dx[:, 1:] * (r / sw ** 2)).sum(axis=1)
    grad[2] += np.sum(-1 / sw + r ** 2 / sw ** 3)
    np.testing.assert_allclose(oracle.logz_fixed_gradient(synth.MODEL_AR1, th, y, anc, sstar, **kw), grad,
                               rtol=1e-7, atol=1e-9)
    # Fisher score of the single path: grad log p(x_0:T, y_1:T)
    e = x[1:] - a * x[:-1]
    score = np.array([np.sum(e * x[:-1]) / sv ** 2,
                      np.sum(-1 / sv + e ** 2 / sv ** 3),
                      np.sum(-1 / sw + r ** 2 / sw ** 3),
                      -1 / s0 + x[0] ** 2 / s0 ** 3])
    np.testing.assert_allclose(oracle.fisher_score(synth.MODEL_AR1, th, y, anc, sstar, **kw), score,
                               rtol=1e-7, atol=1e-8)


def test_fisher_score_estimates_the_kalman_score():
    y = synth.ar1_observations(30, seed=1)
    th = np.array(synth.AR1_THETA, float)
    kw = dict(m=4, M=256, seed=9)
    runs = []
    for c in range(16):
        r = oracle.airpf(synth.MODEL_AR1, th, y, mode=oracle.MODE_ADAPTIVE, tau=0.5, chain=c, **kw)
        runs.append(oracle.fisher_score(synth.MODEL_AR1, th, y, r["anc"], r["sstar"], chain=c, **kw))
    runs = np.array(runs)
    ref = np.zeros(4)
    for d in range(4):
        h = 1e-5
        tp, tm = th.copy(), th.copy()
        tp[d] += h
        tm[d] -= h
        ref[d] = (kalman.ar1_loglik(tp, y) - kalman.ar1_loglik(tm, y)) / (2 * h)
    mean = runs.mean(axis=0)
    se = runs.std(axis=0, ddof=1) / np.sqrt(len(runs))
    assert np.all(np.abs(mean - ref) < 4 * se + 0.05 * np.abs(ref) + 0.2), (mean, ref, se)


def test_gradient_reference_converges_on_ngm():
    """The gradient reference (central differences with one Richardson step at h = 1e-5)
    equals plain central differences at a hundred times smaller step on the nonlinear growth
    model, whose log Z bends sharply in q (the plain difference's h^2 error is below 1e-8
    there): the reference carries no truncation error at the 1e-6 level the GPU comparison
    uses."""
    y = synth.ngm_observations(25, 5)
    th = np.array([10.0, 1.0, 5.0])
    for chain in (1, 2):
        kw = dict(m=8, M=32, seed=6, chain=chain, iter=2)
        r = oracle.airpf(synth.MODEL_NGM, th, y, mode=oracle.MODE_ADAPTIVE, tau=0.5, **kw)
        ref = oracle.logz_fixed_gradient(synth.MODEL_NGM, th, y, r["anc"], r["sstar"], **kw)
        fine = np.zeros(3)
        for d in range(3):
            hd = 1e-7 * max(1.0, abs(th[d]))
            tp, tm = th.copy(), th.copy()
            tp[d] += hd
            tm[d] -= hd
            fine[d] = (oracle.logz_fixed(synth.MODEL_NGM, tp, y, r["anc"], r["sstar"], **kw)
                       - oracle.logz_fixed(synth.MODEL_NGM, tm, y, r["anc"], r["sstar"], **kw)) / (2 * hd)
        # the fine step's own rounding error: a few ulps of log Z over 1e-7
        atol = 4 * np.finfo(float).eps * abs(r["log_z"]) / 1e-7
        np.testing.assert_allclose(ref, fine, rtol=1e-7, atol=atol)
