"""Pins the oracle's radix-r interactions (r = 2^b; m a power of r; Section 2's A_s with
r^-1 1_r in place of 1/2 1_2).

At an r-ary stage every island draws one member of its group of r islands, with probability
proportional to the members' weights and independently of the other islands (the selection
line of Algorithm 1).  Pinned by:

* the exact pair-moment recursion extended to r-ary stages equals brute-force enumeration of
  every random outcome in rational arithmetic (m = r = 4, M = 1, T = 3), and gives E[Z] = Z;
* the oracle's Monte-Carlo E[(Z^N)^2] on the binary HMM (m = 4, r = 4, M = 2, T = 16, always
  interacting) lies inside a 4.5-sigma band around the r-ary exact value and outside it around
  the value of two binary butterfly stages (the r-way choice built from chained pair choices,
  which has the right marginal but correlated islands);
* the joint law of the island choices: after one interacting 4-ary stage, islands k != l pick
  the same member with probability sum_c p_c^2 (p_c = W_c / sum W recomputed here from single-
  particle model calls), and each island's marginal is p;
* adaptive decisions per r-ary stage: s* is the first stage whose recorded ENF reaches tau;
* Z stays unbiased against the Kalman likelihood; radix 2 is the binary algorithm.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import exact_variance as ev
from oracle import kalman


@pytest.fixture(scope="module")
def toy():
    return ev.toy_model(0.75, 0.75)


def test_radix_pair_moments_equal_brute_force(toy):
    pi0, K, g = toy
    ys = synth.toy_observations(3, seed=3)
    gs = [g(y) for y in ys]
    z = np.exp(ev.forward_z(pi0, K, gs))
    ez, ez2 = ev.pair_moments(pi0, K, gs, 4, 1, True, radix=4)
    bz, bz2 = ev.brute_force_moments(0.75, 0.75, ys, 4, 1, 1, radix=4)
    assert ez == pytest.approx(float(bz), rel=1e-13)
    assert ez2 == pytest.approx(float(bz2), rel=1e-13)
    assert ez == pytest.approx(z, rel=1e-13)
    # the r-ary value differs from two binary stages (same m, M, y)
    _, bin2 = ev.brute_force_moments(0.75, 0.75, ys, 4, 1, 1, radix=2)
    assert abs(float(bin2) - float(bz2)) > 1e-6 * float(bz2)
    # adaptive r-ary interaction is unbiased too (Theorem 1)
    az, _ = ev.brute_force_moments(0.75, 0.75, ys, 4, 1, 2, Fraction(95, 100), radix=4)
    assert float(az) == pytest.approx(z, rel=1e-13)


def test_oracle_second_moment_matches_radix_exact(toy):
    pi0, K, g = toy
    ys = synth.toy_observations(16, seed=3)
    gs = [g(y) for y in ys]
    exact4 = ev.pair_moments(pi0, K, gs, 4, 2, True, radix=4)[1]
    binary = ev.pair_moments(pi0, K, gs, 4, 2, True, radix=2)[1]
    runs = 600_000
    lz = oracle.airpf_batch(synth.MODEL_TOY, synth.TOY_THETA, ys, m=4, M=2, runs=runs, mode=oracle.MODE_ALWAYS,
                            seed=21, radix=4)
    z2 = np.exp(2 * lz)
    mean, se = z2.mean(), z2.std() / np.sqrt(runs)
    assert abs(mean - exact4) < 4.5 * se, (mean, exact4, se)
    assert abs(mean - binary) > 4.5 * se, ("cannot tell r-ary from chained binary stages", mean, binary, se)


def _island_weights(th, y, m, M, seed, chain):
    """p_c = W_c / sum W after the first weighting, from single-particle model calls."""
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
    p = np.exp(lw - lw.max())
    return p / p.sum()


def test_four_way_choices_are_independent_and_proportional():
    th = synth.AR1_THETA
    y = synth.ar1_observations(1, seed=1)
    m, M, seed, runs = 4, 4, 21, 4000
    hits = np.zeros(m)
    expect = np.zeros(m)
    var = np.zeros(m)
    coll, coll_exp, coll_var = 0.0, 0.0, 0.0
    pairs = [(k, l) for k in range(m) for l in range(k + 1, m)]
    for chain in range(runs):
        r = oracle.airpf(synth.MODEL_AR1, th, y, m=m, M=M, mode=oracle.MODE_ALWAYS, seed=seed, chain=chain,
                         radix=4)
        src = r["src"][0]
        p = _island_weights(th, y, m, M, seed, chain)
        hits[src[0]] += 1
        expect += p
        var += p * (1 - p)
        q = float((p * p).sum())                 # P(two islands pick the same member)
        coll += sum(src[k] == src[l] for k, l in pairs)
        coll_exp += len(pairs) * q
        coll_var += len(pairs) * q * (1 - q)
    z = (hits - expect) / np.sqrt(var)
    assert np.all(np.abs(z) < 4), z
    # the pair indicators are not independent of each other, so the band is wider than 4 SD
    zc = (coll - coll_exp) / np.sqrt(3 * coll_var)
    assert abs(zc) < 4, (coll, coll_exp, zc)


@pytest.mark.parametrize("radix", [4, 8])
def test_adaptive_decision_per_radix_stage(radix):
    y = synth.ngm_observations(40, seed=5)
    tau = 0.7
    r = oracle.airpf(synth.MODEL_NGM, synth.NGM_THETA, y, m=64, M=16, mode=oracle.MODE_ADAPTIVE, tau=tau,
                     seed=2, radix=radix)
    Sr = int(round(np.log(64) / np.log(radix)))
    assert r["enf"].shape == (40, Sr + 1)
    for t in range(40):
        e = r["enf"][t, 1:]
        below = e < tau
        # interacting stages form a prefix; s* is the first stage with ENF >= tau
        want = Sr + 1 if below.all() else 1 + int(np.argmin(below))
        assert r["sstar"][t] == want, (t, r["sstar"][t], e)
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
