"""Pins the oracle's state-space models (Section 1.2, eq. (1)) and random streams.

Observation densities are compared with scipy's densities (the special cases reduce to
library routines); transitions and priors by their exact first two moments over many
independent stream units; the stream normals by a Kolmogorov-Smirnov test.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
import synth


def test_logg_matches_scipy_densities():
    rng = np.random.default_rng(0)
    for _ in range(20):
        x, y = rng.normal(), rng.normal()
        th = np.array([0.7, 1.3, 0.8, 1.1])
        assert np.isclose(oracle.model_logg(synth.MODEL_AR1, th, [y], [x]),
                          stats.norm.logpdf(y, loc=x, scale=0.8), rtol=1e-13, atol=1e-13)
        th = synth.SV_THETA
        assert np.isclose(oracle.model_logg(synth.MODEL_SV, th, [y], [x]),
                          stats.norm.logpdf(y, loc=0.0, scale=np.exp(x / 2)), rtol=1e-13, atol=1e-13)
        th = np.array([10.0, 1.7, 5.0])
        assert np.isclose(oracle.model_logg(synth.MODEL_NGM, th, [y], [x]),
                          stats.norm.logpdf(y, loc=x * x / 20, scale=np.sqrt(1.7)), rtol=1e-13, atol=1e-13)
    for xv in (0.0, 1.0):
        for yv in (0.0, 1.0):
            want = np.log(0.75 if xv == yv else 0.25)
            assert np.isclose(oracle.model_logg(synth.MODEL_TOY, synth.TOY_THETA, [yv], [xv]), want)
    dx, dy = 3, 2
    A, C, md = synth.lg_model(dx, dy, seed=1)
    th = synth.lg_theta(A, q=0.2, r=0.4)
    x, y = rng.normal(size=dx), rng.normal(size=dy)
    want = stats.multivariate_normal(mean=C @ x, cov=0.4 * np.eye(dy)).logpdf(y)
    assert np.isclose(oracle.model_logg(synth.MODEL_LGSSM, th, y, x, dx=dx, dy=dy, model_data=md),
                      want, rtol=1e-12)


def _moments(fn, n):
    v = np.array([fn(u) for u in range(n)])
    return v.mean(axis=0), v.var(axis=0)


@pytest.mark.parametrize("model,theta,xp,mean,var", [
    (synth.MODEL_AR1, [0.6, 1.5, 1.0, 1.0], 2.0, 1.2, 2.25),
    (synth.MODEL_SV, [-1.0, 0.9, 0.4], 0.5, -1.0 + 0.9 * 1.5, 0.16),
    (synth.MODEL_NGM, [10.0, 1.0, 5.0], 1.5, 0.75 + 37.5 / 3.25 + 8 * np.cos(1.2 * 3), 10.0),
])
def test_transition_moments(model, theta, xp, mean, var):
    n = 40000
    m_, v_ = _moments(lambda u: oracle.model_step(model, theta, [xp], unit=u, t=3, seed=9)[0], n)
    assert abs(m_ - mean) < 5 * np.sqrt(var / n)
    assert abs(v_ - var) < 5 * var * np.sqrt(2.0 / n)


@pytest.mark.parametrize("model,theta,mean,var", [
    (synth.MODEL_AR1, [0.9, 1.0, 1.0, 1.3], 0.0, 1.69),
    (synth.MODEL_SV, [-1.0, 0.95, 0.3], -1.0, 0.09 / (1 - 0.95 ** 2)),
    (synth.MODEL_NGM, [10.0, 1.0, 5.0], 0.0, 5.0),
    (synth.MODEL_TOY, [0.75, 0.75], 0.5, 0.25),
])
def test_prior_moments(model, theta, mean, var):
    n = 40000
    m_, v_ = _moments(lambda u: oracle.model_prior(model, theta, unit=u, seed=4)[0], n)
    assert abs(m_ - mean) < 5 * np.sqrt(var / n)
    assert abs(v_ - var) < 5 * var * np.sqrt(2.0 / n) + 1e-12


def test_toy_transition_flip_rate():
    n = 40000
    flips = np.array([oracle.model_step(synth.MODEL_TOY, [0.75, 0.75], [1.0], unit=u, t=2)[0] == 0.0
                      for u in range(n)])
    assert abs(flips.mean() - 0.25) < 5 * np.sqrt(0.25 * 0.75 / n)


def test_lg_transition_moments():
    dx, dy = 3, 2
    A, C, md = synth.lg_model(dx, dy, seed=2)
    th = synth.lg_theta(A, q=0.3, r=0.5)
    xp = np.array([1.0, -0.5, 2.0])
    n = 20000
    v = np.array([oracle.model_step(synth.MODEL_LGSSM, th, xp, unit=u, t=1, dx=dx, dy=dy,
                                    model_data=md) for u in range(n)])
    assert np.all(np.abs(v.mean(0) - A @ xp) < 5 * np.sqrt(0.3 / n))
    cov = np.cov(v.T)
    assert np.all(np.abs(cov - 0.3 * np.eye(dx)) < 5 * 0.3 * np.sqrt(2.0 / n))


def test_stream_normals_are_standard_normal():
    z = np.array([oracle.model_step(synth.MODEL_AR1, [0.0, 1.0, 1.0, 1.0], [0.0], unit=u, t=7,
                                    seed=77)[0] for u in range(20000)])
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_stream_keying_spec():
    """A one-normal transition of particle g at time t takes the Box-Muller pair of
    Philox(counter=(g >> 1, t, iter, chain<<8 | 1<<5 | 0), key=seed): the cosine normal
    for even g, the sine normal for odd g (particles 2j and 2j+1 share block j)."""
    seed, chain, it = 0x1234_5678_9ABC_DEF0, 3, 11
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for g, t in [(0, 1), (1, 1), (5, 2), (1000, 99), (1001, 99)]:
        w = oracle.philox([g >> 1, t, it, (chain << 8) | (1 << 5)], key)
        u0, u1 = (w[0] + 0.5) * 2.0 ** -32, (w[1] + 0.5) * 2.0 ** -32
        r, a = np.sqrt(-2 * np.log(u0)), 2 * np.pi * u1
        z = r * (np.sin(a) if g & 1 else np.cos(a))
        x = oracle.model_step(synth.MODEL_AR1, [0.0, 1.0, 1.0, 1.0], [0.0], unit=g, t=t,
                              seed=seed, chain=chain, iter=it)[0]
        assert x == pytest.approx(z, rel=1e-15, abs=1e-15)


def test_stream_keying_spec_several_normals():
    """A transition with d_x >= 2 normals keeps a block of its own: normal d of particle g is
    component d & 1 of the pair of Philox(counter=(g, t, iter, chain<<8 | 1<<5 | d >> 1))."""
    seed, chain, it = 99, 1, 4
    key = [seed & 0xFFFFFFFF, seed >> 32]
    dx = 3
    th = np.array([0.0, 0.0, 0.0, 0.0, 0.0])          # A = 0 (no off-diagonal data), q = e^0 = 1
    md = np.zeros(dx * dx + 1 * dx)
    for g, t in [(0, 1), (7, 3)]:
        x = oracle.model_step(synth.MODEL_LGSSM, th, np.zeros(dx), unit=g, t=t, dx=dx, dy=1, model_data=md,
                              seed=seed, chain=chain, iter=it)
        for d in range(dx):
            w = oracle.philox([g, t, it, (chain << 8) | (1 << 5) | (d >> 1)], key)
            u0, u1 = (w[0] + 0.5) * 2.0 ** -32, (w[1] + 0.5) * 2.0 ** -32
            r, a = np.sqrt(-2 * np.log(u0)), 2 * np.pi * u1
            assert x[d] == pytest.approx(r * (np.sin(a) if d & 1 else np.cos(a)), rel=1e-14, abs=1e-14)


def test_paired_transition_normals_are_independent():
    """Particles 2j and 2j+1 share one block: their normals are the two halves of one
    Box-Muller pair, so (z_2j, z_2j+1) is standard bivariate normal: correlation 0 and
    (z_2j^2 + z_2j+1^2) / 2 exponential with mean 1."""
    z = np.array([oracle.model_step(synth.MODEL_AR1, [0.0, 1.0, 1.0, 1.0], [0.0], unit=u, t=4,
                                    seed=5)[0] for u in range(20000)])
    a, b = z[0::2], z[1::2]
    assert abs(np.corrcoef(a, b)[0, 1]) < 4.0 / np.sqrt(a.size)
    assert stats.kstest((a * a + b * b) / 2, "expon").pvalue > 1e-3
    assert stats.kstest(b, "norm").pvalue > 1e-3
