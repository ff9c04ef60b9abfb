"""Pins the oracle's adaptive internal resampling (an island resamples only when the ESS of
its particle weights omega_i g_t(x_i) falls below tau_int M; otherwise it carries the
normalised weights).

* Z-hat stays unbiased: its mean over independent runs matches the Kalman likelihood of the
  AR(1) model.
* With a threshold no ESS can fall below, no island ever resamples: each particle follows its
  own path and Z-hat is the sequential importance sampling estimate
  M^-1 sum_i prod_t g_t(x^i_t) (m = 1), recomputed here from the single-particle model calls.
* tau_int = 1 resamples whenever the weights are not all equal, i.e. at every step of a
  continuous model: the same run as tau_int = 0.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import kalman


@pytest.mark.parametrize("tau_int,mode,runs", [(0.5, oracle.MODE_ADAPTIVE, 1500), (0.9, oracle.MODE_ADAPTIVE, 1500),
                                                (0.2, oracle.MODE_ALWAYS, 4000)])
def test_unbiased_against_kalman(tau_int, mode, runs):
    """(The last case interacts at every stage while most islands carry unequal weights: an
    island that inherits a block must inherit its weights too; keeping its own was 54 standard
    errors off.)"""
    y = synth.ar1_observations(20, seed=1)
    th = synth.AR1_THETA
    lz = oracle.airpf_batch(synth.MODEL_AR1, th, y, m=4, M=16, runs=runs, mode=mode, tau=0.5,
                            seed=3, tau_int=tau_int)
    ratio = np.exp(lz - kalman.ar1_loglik(th, y))
    se = ratio.std(ddof=1) / np.sqrt(ratio.size)
    assert abs(ratio.mean() - 1.0) < 4 * se, (ratio.mean(), se)


def test_never_resampling_is_sequential_importance_sampling():
    y = synth.ar1_observations(8, seed=1)
    th = synth.AR1_THETA
    M, seed, chain, it = 64, 5, 2, 1
    r = oracle.airpf(synth.MODEL_AR1, th, y, m=1, M=M, seed=seed, chain=chain, iter=it, tau_int=1e-9)
    lpath = np.zeros(M)
    for i in range(M):
        x = oracle.model_prior(synth.MODEL_AR1, th, unit=i, seed=seed, chain=chain, iter=it)
        for t in range(1, len(y) + 1):
            x = oracle.model_step(synth.MODEL_AR1, th, x, unit=i, t=t, seed=seed, chain=chain, iter=it)
            lpath[i] += oracle.model_logg(synth.MODEL_AR1, th, y[t - 1:t], x)
    mx = lpath.max()
    ref = mx + np.log(np.exp(lpath - mx).sum()) - np.log(M)
    assert r["log_z"] == pytest.approx(ref, rel=1e-12)
    assert np.array_equal(r["anc"], np.tile(np.arange(M, dtype=np.int32), (len(y), 1)))


def test_threshold_one_equals_resampling_every_step():
    y = synth.sv_observations(15, seed=2)
    kw = dict(m=8, M=32, mode=oracle.MODE_ADAPTIVE, tau=0.5, seed=4, chain=1)
    a = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, tau_int=1.0, **kw)
    b = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, tau_int=0.0, **kw)
    assert np.array_equal(a["anc"], b["anc"])
    assert a["log_z"] == pytest.approx(b["log_z"], rel=1e-13)
