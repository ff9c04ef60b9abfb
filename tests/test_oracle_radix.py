"""Pins the oracle's radix-r interactions (r = 2^b; m a power of r).

* The r-way island choice: with one r-ary stage that interacts (m = r = 4, one step), island
  0 takes the block of island c with probability W_c / sum W, where W_c = M^-1 sum_i
  g(y_1 | x^{c,i}_1) is recomputed here from the single-particle model calls.
* The adaptive decision is taken per r-ary stage: every recorded s* is the first binary stage
  of a group (1, b + 1, 2b + 1, ...) or S + 1.
* Z-hat stays unbiased against the Kalman likelihood.
* Radix 2 is the binary algorithm.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import kalman


def test_four_way_choice_is_proportional_to_the_weights():
    th = synth.AR1_THETA
    y = synth.ar1_observations(1, seed=1)
    m, M, seed = 4, 4, 21
    hits = np.zeros(m)
    expect = np.zeros(m)
    var = np.zeros(m)
    for chain in range(3000):
        r = oracle.airpf(synth.MODEL_AR1, th, y, m=m, M=M, mode=oracle.MODE_ALWAYS, seed=seed, chain=chain,
                         radix=4)
        lw = np.zeros(m)
        for c in range(m):
            lg = []
            for i in range(M):
                u = c * M + i
                x0 = oracle.model_prior(synth.MODEL_AR1, th, unit=u, seed=seed, chain=chain)
                x1 = oracle.model_step(synth.MODEL_AR1, th, x0, unit=u, t=1, seed=seed, chain=chain)
                lg.append(oracle.model_logg(synth.MODEL_AR1, th, y, x1))
            lg = np.array(lg)
            lw[c] = lg.max() + np.log(np.exp(lg - lg.max()).mean())
        pc = np.exp(lw - lw.max())
        pc /= pc.sum()
        hits[r["src"][0, 0]] += 1
        expect += pc
        var += pc * (1 - pc)
    z = (hits - expect) / np.sqrt(var)
    assert np.all(np.abs(z) < 4), z


@pytest.mark.parametrize("radix", [4, 8])
def test_adaptive_decision_per_radix_stage(radix):
    y = synth.ngm_observations(40, seed=5)
    r = oracle.airpf(synth.MODEL_NGM, synth.NGM_THETA, y, m=64, M=16, mode=oracle.MODE_ADAPTIVE, tau=0.7,
                     seed=2, radix=radix)
    b = int(np.log2(radix))
    assert np.all((r["sstar"] - 1) % b == 0), r["sstar"]
    assert len(set(r["sstar"].tolist())) > 1          # the decision varies over the run


def test_unbiased_against_kalman_radix4():
    y = synth.ar1_observations(20, seed=1)
    th = synth.AR1_THETA
    lz = oracle.airpf_batch(synth.MODEL_AR1, th, y, m=16, M=8, runs=3000, mode=oracle.MODE_ADAPTIVE, tau=0.7,
                            seed=3, radix=4)
    ratio = np.exp(lz - kalman.ar1_loglik(th, y))
    se = ratio.std(ddof=1) / np.sqrt(ratio.size)
    assert abs(ratio.mean() - 1.0) < 4 * se, (ratio.mean(), se)


def test_radix_two_is_binary():
    y = synth.sv_observations(20, seed=2)
    kw = dict(m=16, M=16, mode=oracle.MODE_ADAPTIVE, tau=0.6, seed=4)
    a = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, radix=2, **kw)
    b = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, **kw)
    assert np.array_equal(a["anc"], b["anc"]) and a["log_z"] == b["log_z"]


def test_m_not_a_power_of_the_radix_is_refused():
    with pytest.raises(ValueError):
        oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, synth.ar1_observations(3, 1), m=8, M=4, radix=4)
