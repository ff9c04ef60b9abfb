"""Pins the oracle's AIRPF run (Algorithm 1) to what the paper and the mathematics fix.

* Theorem 1 (lack of bias): mean of Z^N / Z_Kalman over independent runs is 1 within a
  4.5-sigma band, on AR(1) and on a small multivariate linear-Gaussian model;
* Section 2: m = 1 is the bootstrap filter, alpha = I gives independent bootstrap filters
  (the BPF is a separately written function);
* the resampling and island-choice draws equal a re-derivation from the stream
  specification with numpy's searchsorted;
* the invariants of Algorithm 1: ENF non-decreasing over stages (Section 2.3), the
  interacting stages form a prefix, full interaction equalises the island weights.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import kalman


def test_unbiased_ar1_against_kalman():
    y = synth.ar1_observations(100, seed=1)
    z = kalman.ar1_loglik(synth.AR1_THETA, y)
    for mode in (oracle.MODE_ALWAYS, oracle.MODE_ADAPTIVE, oracle.MODE_NEVER):
        lz = oracle.airpf_batch(synth.MODEL_AR1, synth.AR1_THETA, y, m=16, M=64, runs=400,
                                mode=mode, tau=0.3, seed=5)
        r = np.exp(lz - z)
        assert abs(r.mean() - 1.0) < 4.5 * r.std() / np.sqrt(len(r)), (mode, r.mean(), r.std())
        # a mis-scaled weight would show up as a shift of log Z far beyond its spread
        assert abs(np.mean(lz - z)) < 0.5


def test_unbiased_small_lgssm_against_kalman():
    dx, dy = 2, 2
    A, C, md = synth.lg_model(dx, dy, seed=11)
    th = synth.lg_theta(A, q=0.1, r=0.5)
    y = synth.lg_observations(A, C, 0.1, 0.5, 30, seed=11)
    z = kalman.lg_loglik(th, md, y, dx, dy)
    lz = oracle.airpf_batch(synth.MODEL_LGSSM, th, y, m=8, M=32, runs=400, dx=dx, dy=dy,
                            model_data=md, mode=oracle.MODE_ADAPTIVE, tau=0.5, seed=6)
    r = np.exp(lz - z)
    assert abs(r.mean() - 1.0) < 4.5 * r.std() / np.sqrt(len(r))


def test_m1_is_bootstrap_filter():
    y = synth.sv_observations(40, seed=2)
    for M in (1, 37, 64):
        a = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, m=1, M=M, seed=3, chain=2, iter=4)
        lz, anc, _ = oracle.bpf(synth.MODEL_SV, synth.SV_THETA, y, M=M, seed=3, chain=2, iter=4)
        assert a["log_z"] == pytest.approx(lz, rel=1e-14, abs=1e-12)
        assert np.array_equal(a["anc"], anc)


def test_never_is_independent_bootstrap_filters():
    y = synth.ar1_observations(30, seed=1)
    m, M = 8, 16
    a = oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, m=m, M=M, mode=oracle.MODE_NEVER,
                     seed=9, chain=1)
    lzs = []
    for k in range(m):
        lz, anc, _ = oracle.bpf(synth.MODEL_AR1, synth.AR1_THETA, y, M=M, seed=9, chain=1,
                                unit0=k * M)
        lzs.append(lz)
        assert np.array_equal(a["anc"][:, k * M:(k + 1) * M], anc + k * M)
    lzs = np.array(lzs)
    want = np.log(np.mean(np.exp(lzs - lzs.max()))) + lzs.max()
    assert a["log_z"] == pytest.approx(want, rel=1e-13)
    assert np.array_equal(a["src"], np.tile(np.arange(m), (len(y), 1)))


def _unif(w):
    return (float(w) + 0.5) * 2.0 ** -32


def test_resampling_matches_searchsorted_rederivation():
    """Draw j of island k at t = 1 takes the first i with C_i > u_j C_{M-1}."""
    y = synth.sv_observations(1, seed=2)
    m, M, seed, chain, it = 2, 50, 17, 3, 8
    a = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, m=m, M=M, mode=oracle.MODE_NEVER,
                     seed=seed, chain=chain, iter=it)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for k in range(m):
        g = np.empty(M)
        u = np.empty(M)
        for i in range(M):
            unit = k * M + i
            x0 = oracle.model_prior(synth.MODEL_SV, synth.SV_THETA, unit=unit, seed=seed,
                                    chain=chain, iter=it)
            x1 = oracle.model_step(synth.MODEL_SV, synth.SV_THETA, x0, unit=unit, t=1,
                                   seed=seed, chain=chain, iter=it)
            g[i] = np.exp(oracle.model_logg(synth.MODEL_SV, synth.SV_THETA, y[:1], x1))
            w = oracle.philox([unit >> 1, 1, it, (chain << 8) | (1 << 5)], key)
            u[i] = _unif(w[3] if unit & 1 else w[2])
        cdf = np.cumsum(g)
        want = np.searchsorted(cdf, u * cdf[-1], side="right")
        assert np.array_equal(a["anc"][0, k * M:(k + 1) * M], k * M + want)


def test_island_choice_matches_rederivation():
    """Stage s: island k takes the lower island of {k, k^b} iff u (W_lo+W_hi) < W_lo."""
    y = synth.ar1_observations(1, seed=1)
    m, M, seed = 4, 8, 23
    a = oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, m=m, M=M, mode=oracle.MODE_ALWAYS,
                     seed=seed)
    key = [seed, 0]
    W = np.empty(m)
    for k in range(m):
        gs = []
        for i in range(M):
            x0 = oracle.model_prior(synth.MODEL_AR1, synth.AR1_THETA, unit=k * M + i, seed=seed)
            x1 = oracle.model_step(synth.MODEL_AR1, synth.AR1_THETA, x0, unit=k * M + i, t=1,
                                   seed=seed)
            gs.append(np.exp(oracle.model_logg(synth.MODEL_AR1, synth.AR1_THETA, y[:1], x1)))
        W[k] = np.mean(gs)
    idx = np.arange(m)
    for s in (1, 2):
        b = 1 << (s - 1)
        new_idx, new_W = idx.copy(), W.copy()
        for k in range(m):
            lo, hi = k & ~b, k | b
            u = _unif(oracle.philox([k, 1, 0, (2 << 5) | s], key)[0])
            new_idx[k] = idx[lo] if u * (W[lo] + W[hi]) < W[lo] else idx[hi]
            new_W[k] = 0.5 * (W[lo] + W[hi])
        idx, W = new_idx, new_W
    assert np.array_equal(a["src"][0], idx)
    assert np.allclose(W, W[0])       # the full butterfly equalises the weights


@pytest.mark.parametrize("mode", [oracle.MODE_ADAPTIVE, oracle.MODE_ALWAYS, oracle.MODE_NEVER])
def test_stage_invariants(mode):
    y = synth.sv_observations(60, seed=2)
    m, M, tau = 64, 16, 0.6
    a = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, m=m, M=M, mode=mode, tau=tau, seed=4)
    enf, sstar = a["enf"], a["sstar"]
    S = 6
    assert np.all(np.diff(enf[:, 1:], axis=1) >= -1e-12)        # ENF non-decreasing
    assert np.all((enf[:, 1:] >= 1.0 / m - 1e-12) & (enf[:, 1:] <= 1 + 1e-12))
    for t in range(len(y)):
        if mode == oracle.MODE_ADAPTIVE:
            below = enf[t, 1:] < tau
            want = 1 + int(np.argmin(below)) if not below.all() else S + 1
            assert sstar[t] == want
            assert np.all(below[: want - 1])                    # interacting stages: a prefix
        elif mode == oracle.MODE_ALWAYS:
            assert sstar[t] == S + 1
            if t > 0:
                assert enf[t, 0] == pytest.approx(1.0, abs=1e-12)   # equal weights
        else:
            assert sstar[t] == 1
    assert a["logz_trace"][-1] == pytest.approx(a["log_z"], rel=1e-15)


def test_dead_filter_gives_minus_infinity():
    y = np.full(5, 1e200)
    a = oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, m=4, M=8, mode=oracle.MODE_ADAPTIVE)
    assert a["log_z"] == -np.inf
    assert np.all(np.isfinite(a["xfinal"]))


def test_argument_checks():
    y = synth.ar1_observations(5)
    for kw in (dict(m=3, M=4), dict(m=4, M=0), dict(m=4, M=4, tau=0.0), dict(m=4, M=4, tau=1.5)):
        with pytest.raises(ValueError):
            oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, **kw)
