"""Pins the oracle's whole AIRPF run against exact results on the binary HMM of Section 4.1.

* the pair-moment recursion (from Theorem 3 and Lemmas 2-3) equals a brute-force
  enumeration of every random outcome in rational arithmetic;
* E[Z^N] equals the forward-algorithm Z in every mode (Theorem 1, lack of bias);
* the oracle's Monte-Carlo E[(Z^N)^2] lies inside a 4.5-sigma band around the exact value
  for always / never interaction, m = 1 and adaptive interaction, and the band is narrow
  enough to reject the exact value of the *other* interaction mode (so a wrong island
  choice rule or a dropped stage would fail).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import exact_variance as ev


@pytest.fixture(scope="module")
def toy():
    pi0, K, g = ev.toy_model(0.75, 0.75)
    return pi0, K, g


def test_pair_moments_equal_brute_force(toy):
    pi0, K, g = toy
    ys = synth.toy_observations(3, seed=3)
    gs = [g(y) for y in ys]
    for m, M, interact in [(2, 2, False), (2, 2, True), (1, 4, False), (1, 2, False)]:
        ez, ez2 = ev.pair_moments(pi0, K, gs, m, M, interact)
        bz, bz2 = ev.brute_force_moments(0.75, 0.75, ys, m, M, 1 if interact else 0)
        assert ez == pytest.approx(float(bz), rel=1e-13)
        assert ez2 == pytest.approx(float(bz2), rel=1e-13)


def test_expectation_equals_forward_algorithm(toy):
    """Theorem 1: E[Z^N_T] = Z_T, in every interaction mode."""
    pi0, K, g = toy
    ys = synth.toy_observations(3, seed=5)
    z = np.exp(ev.forward_z(pi0, K, [g(y) for y in ys]))
    for mode, tau in [(0, 1), (1, 1), (2, Fraction(9, 10)), (2, Fraction(99, 100))]:
        bz, _ = ev.brute_force_moments(0.75, 0.75, ys, 2, 2, mode, tau)
        assert float(bz) == pytest.approx(z, rel=1e-13)
    ys = synth.toy_observations(10, seed=6)
    z = np.exp(ev.forward_z(pi0, K, [g(y) for y in ys]))
    for m, M, inter in [(4, 2, True), (4, 2, False), (1, 8, False)]:
        ez, _ = ev.pair_moments(pi0, K, [g(y) for y in ys], m, M, inter)
        assert ez == pytest.approx(z, rel=1e-12)


def _mc_second_moment(ys, m, M, mode, tau=0.3, runs=200_000, seed=21):
    lz = oracle.airpf_batch(synth.MODEL_TOY, synth.TOY_THETA, ys, m=m, M=M, runs=runs,
                            mode=mode, tau=tau, seed=seed)
    z2 = np.exp(2 * lz)
    return z2.mean(), z2.std() / np.sqrt(runs)


def test_oracle_second_moment_matches_exact(toy):
    pi0, K, g = toy
    ys = synth.toy_observations(12, seed=3)
    gs = [g(y) for y in ys]
    exact = {
        "always": ev.pair_moments(pi0, K, gs, 4, 2, True)[1],
        "never": ev.pair_moments(pi0, K, gs, 4, 2, False)[1],
    }
    for name, mode in (("always", oracle.MODE_ALWAYS), ("never", oracle.MODE_NEVER)):
        mean, se = _mc_second_moment(ys, 4, 2, mode)
        assert abs(mean - exact[name]) < 4.5 * se, (name, mean, exact[name], se)
        other = exact["never" if name == "always" else "always"]
        assert abs(mean - other) > 4.5 * se, "test cannot tell the interaction modes apart"
    # m = 1: a single bootstrap filter of 8 particles
    bpf2 = ev.pair_moments(pi0, K, gs, 1, 8, False)[1]
    mean, se = _mc_second_moment(ys, 1, 8, oracle.MODE_ALWAYS)
    assert abs(mean - bpf2) < 4.5 * se
    assert abs(mean - exact["never"]) > 4.5 * se


def test_oracle_adaptive_second_moment_matches_brute_force():
    ys = synth.toy_observations(3, seed=3)
    tau = Fraction(9, 10)
    _, bz2 = ev.brute_force_moments(0.75, 0.75, ys, 2, 2, 2, tau)
    _, never2 = ev.brute_force_moments(0.75, 0.75, ys, 2, 2, 0)
    mean, se = _mc_second_moment(ys, 2, 2, oracle.MODE_ADAPTIVE, tau=0.9, runs=400_000)
    assert abs(mean - float(bz2)) < 4.5 * se
    assert abs(float(bz2) - float(never2)) > 0      # adaptive differs from never here


def test_relative_variance_ordering_at_long_horizon(toy):
    """Section 4.1: BPF < AIRPF < IBPF in relative variance for long data records."""
    pi0, K, g = toy
    ys = synth.toy_observations(24, seed=3)
    gs = [g(y) for y in ys]
    z = np.exp(ev.forward_z(pi0, K, gs))
    rv = {name: ev.pair_moments(pi0, K, gs, m, M, inter)[1] / z ** 2 - 1
          for name, m, M, inter in [("bpf", 1, 8, False), ("airpf", 4, 2, True),
                                    ("ibpf", 4, 2, False)]}
    assert rv["bpf"] < rv["airpf"] < rv["ibpf"]
