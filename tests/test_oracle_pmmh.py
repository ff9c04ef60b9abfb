"""Pins the oracle's PMMH (Andrieu et al. 2010, used with AIRPF per Theorem 1's remark).

* the chain's posterior mean and variance of the AR coefficient agree with quadrature of
  the exact (Kalman) likelihood under the U(-1, 1) prior, within Monte-Carlo error;
* the chain is counter-based, so two runs of K iterations resume into one of 2K exactly.
"""
import numpy as np

import oracle
import synth
from oracle import kalman


def _batch_means_se(x, nb=20):
    b = np.array_split(x, nb)
    mu = np.array([v.mean() for v in b])
    return mu.std(ddof=1) / np.sqrt(nb)


def test_pmmh_posterior_matches_quadrature():
    y = synth.ar1_observations(100, seed=1)
    _, _, mean, var = kalman.ar1_posterior_grid(y)
    step = [0.05, 0, 0, 0]
    lo, hi = [-1, 0, 0, 0], [1, 0, 0, 0]
    r = oracle.pmmh(synth.MODEL_AR1, [0.5, 1.0, 1.0, 1.0], y, m=8, M=32, step=step, lo=lo, hi=hi,
                    iters=3000, mode=oracle.MODE_ADAPTIVE, tau=0.3, seed=31)
    a = r["theta"][500:, 0]
    se = _batch_means_se(a)
    assert abs(a.mean() - mean) < 4.5 * se + 1e-3, (a.mean(), mean, se)
    assert 0.4 * var < a.var() < 2.5 * var
    assert 0.05 < r["n_accept"] / 3000 < 0.95


def test_pmmh_resume_is_exact():
    y = synth.ar1_observations(30, seed=1)
    kw = dict(m=4, M=16, step=[0.05, 0, 0, 0], lo=[-1, 0, 0, 0], hi=[1, 0, 0, 0],
              mode=oracle.MODE_ALWAYS, seed=8, chain=5)
    full = oracle.pmmh(synth.MODEL_AR1, [0.5, 1, 1, 1], y, iters=40, **kw)
    h1 = oracle.pmmh(synth.MODEL_AR1, [0.5, 1, 1, 1], y, iters=20, **kw)
    h2 = oracle.pmmh(synth.MODEL_AR1, h1["theta_final"], y, iters=20, iter0=20,
                     state_logz=h1["logz_final"], **kw)
    assert np.array_equal(full["theta"], np.concatenate([h1["theta"], h2["theta"]]))
    assert np.array_equal(full["logz"], np.concatenate([h1["logz"], h2["logz"]]))


def test_langevin_pmmh_posterior_matches_quadrature():
    """The Langevin proposal (driven by the Fisher score of each estimate) targets the same
    posterior of the AR coefficient as quadrature of the Kalman likelihood under U(-1, 1)."""
    y = synth.ar1_observations(100, seed=1)
    _, _, mean, var = kalman.ar1_posterior_grid(y)
    step = [0.06, 0, 0, 0]
    lo, hi = [-1, 0, 0, 0], [1, 0, 0, 0]
    r = oracle.pmmh_langevin(synth.MODEL_AR1, [0.5, 1.0, 1.0, 1.0], y, m=4, M=64, step=step, lo=lo, hi=hi,
                             iters=1500, mode=oracle.MODE_ADAPTIVE, tau=0.3, seed=41)
    a = r["theta"][300:, 0]
    se = _batch_means_se(a)
    assert abs(a.mean() - mean) < 4.5 * se + 1e-3, (a.mean(), mean, se)
    assert 0.4 * var < a.var() < 2.5 * var
    assert 0.1 < r["n_accept"] / 1500 < 0.99


def test_langevin_pmmh_resume_is_exact():
    y = synth.ar1_observations(30, seed=1)
    kw = dict(m=4, M=16, step=[0.05, 0.05, 0, 0], lo=[-1, 0.1, 0, 0], hi=[1, 3, 0, 0],
              mode=oracle.MODE_ALWAYS, seed=8, chain=5)
    full = oracle.pmmh_langevin(synth.MODEL_AR1, [0.5, 1, 1, 1], y, iters=12, **kw)
    h1 = oracle.pmmh_langevin(synth.MODEL_AR1, [0.5, 1, 1, 1], y, iters=6, **kw)
    h2 = oracle.pmmh_langevin(synth.MODEL_AR1, h1["theta_final"], y, iters=6, iter0=6,
                              state_logz=h1["logz_final"], state_grad=h1["grad_final"], **kw)
    assert np.array_equal(full["theta"], np.concatenate([h1["theta"], h2["theta"]]))
    assert np.array_equal(full["logz"], np.concatenate([h1["logz"], h2["logz"]]))
