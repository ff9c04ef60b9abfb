"""Pins the oracle's change-point model (Section 4.2): x_0 ~ Beta(alpha, beta), K(x, .) =
(1 - p) delta_x + p Beta(alpha, beta), k_t ~ Binomial(n_t, x_t).

* The Beta draws (a ratio of two Marsaglia-Tsang gammas, both branches: alpha >= 1 and the
  boosted alpha < 1) against scipy's Beta law by Kolmogorov-Smirnov tests, and their mean.
* The transition: jumps with probability p, keeps x exactly otherwise, and the jumped values
  follow the Beta law.
* The observation density against scipy's binomial pmf.
* The whole filter at the two closed-form ends: with p = 0 the rate never changes and the
  likelihood is the beta-binomial Prod_t C(n_t, k_t) B(alpha + K, beta + N - K) / B(alpha,
  beta); with p = 1 the rate is redrawn every day and the likelihood is the product of the
  daily beta-binomials.  Z-hat is unbiased, so its mean over independent runs matches.
"""
import numpy as np
import pytest
from scipy import special, stats

import oracle
import synth

CP = synth.MODEL_CP


@pytest.mark.parametrize("alpha,beta", [(2.0, 20.0), (0.5, 3.0), (1.0, 1.0)])
def test_prior_is_beta(alpha, beta):
    th = [0.1, alpha, beta]
    x = np.array([oracle.model_prior(CP, th, unit=u, seed=3)[0] for u in range(20000)])
    assert np.all((x > 0) & (x < 1))
    assert stats.kstest(x, stats.beta(alpha, beta).cdf).pvalue > 1e-3
    mean = alpha / (alpha + beta)
    sd = np.sqrt(alpha * beta / ((alpha + beta) ** 2 * (alpha + beta + 1)))
    assert abs(x.mean() - mean) < 5 * sd / np.sqrt(x.size)


def test_transition_jumps_with_probability_p():
    p, alpha, beta = 0.3, 2.0, 5.0
    xp = 0.123456789
    n = 20000
    x = np.array([oracle.model_step(CP, [p, alpha, beta], [xp], unit=u, t=4, seed=8)[0] for u in range(n)])
    stay = x == xp
    jumps = x[~stay]
    assert abs(jumps.size / n - p) < 5 * np.sqrt(p * (1 - p) / n)
    assert stats.kstest(jumps, stats.beta(alpha, beta).cdf).pvalue > 1e-3


def test_transition_never_and_always():
    xp = 0.4
    never = [oracle.model_step(CP, [0.0, 2.0, 5.0], [xp], unit=u, t=2)[0] for u in range(500)]
    assert all(v == xp for v in never)
    always = np.array([oracle.model_step(CP, [1.0, 2.0, 5.0], [xp], unit=u, t=2)[0] for u in range(500)])
    assert not np.any(always == xp)


def test_logg_is_binomial_pmf():
    rng = np.random.default_rng(0)
    for _ in range(50):
        n = int(rng.integers(1, 2000))
        k = int(rng.integers(0, n + 1))
        x = float(rng.uniform(1e-6, 1 - 1e-6))
        got = oracle.model_logg(CP, synth.CP_THETA, [k, n], [x], dy=2)
        assert got == pytest.approx(stats.binom.logpmf(k, n, x), rel=1e-11, abs=1e-9)
    assert oracle.model_logg(CP, synth.CP_THETA, [0, 10], [0.0], dy=2) == 0.0
    assert oracle.model_logg(CP, synth.CP_THETA, [3, 10], [0.0], dy=2) == -np.inf


def _log_beta_binomial_joint(y, alpha, beta):
    k, n = y[0::2], y[1::2]
    logc = special.gammaln(n + 1) - special.gammaln(k + 1) - special.gammaln(n - k + 1)
    return logc.sum() + special.betaln(alpha + k.sum(), beta + (n - k).sum()) - special.betaln(alpha, beta)


def _log_beta_binomial_daily(y, alpha, beta):
    k, n = y[0::2], y[1::2]
    logc = special.gammaln(n + 1) - special.gammaln(k + 1) - special.gammaln(n - k + 1)
    return (logc + special.betaln(alpha + k, beta + n - k) - special.betaln(alpha, beta)).sum()


@pytest.mark.parametrize("p,exact", [(0.0, _log_beta_binomial_joint), (1.0, _log_beta_binomial_daily)])
@pytest.mark.parametrize("mode", [oracle.MODE_ADAPTIVE, oracle.MODE_ALWAYS])
def test_filter_is_unbiased_at_closed_form_ends(p, exact, mode):
    alpha, beta = 2.0, 5.0
    y = synth.cp_observations(6, seed=11, theta=[0.3, alpha, beta], n_lo=5, n_hi=15)
    lz_exact = exact(y, alpha, beta)
    lz = oracle.airpf_batch(CP, [p, alpha, beta], y, m=4, M=32, runs=400, mode=mode, tau=0.5, dy=2, seed=2)
    ratio = np.exp(lz - lz_exact)
    se = ratio.std(ddof=1) / np.sqrt(ratio.size)
    assert abs(ratio.mean() - 1.0) < 4 * se + 1e-3, (ratio.mean(), se)
