"""Radix-r interactions (r = 4, 8, 16; m a power of r) on the GPU against the oracle: FP64
ancestors, s*, ENF and log Z element by element in the adaptive and always modes and every
launch form, with groups that lie inside one CTA's islands and groups that span several CTAs;
the FP32-mixed path's island choices against the oracle's on the first step; Theorem 3's
second moment with 4-ary stages; and the configuration check."""
import numpy as np
import pytest

import oracle
import synth
from oracle import exact_variance as ev
from parity_util import compare_filter, compare_first_step, run_gpu

pytestmark = pytest.mark.gpu


def _check_stages(g, k, m, radix):
    Sr = int(round(np.log(m) / np.log(radix)))
    assert g["enf"].shape[-1] == Sr + 1
    assert np.all((g["sstar"][k] >= 1) & (g["sstar"][k] <= Sr + 1))


# (one CTA holds a filter of at most 16 islands of 32 threads)
@pytest.mark.parametrize("radix,m,launch", [(r, m, l) for r, m in [(4, 16), (4, 64), (8, 64), (16, 256)]
                                            for l in ("steps", "split", "cta") if l != "cta" or m <= 16])
def test_matches_oracle(radix, m, launch):
    y = synth.ngm_observations(30, seed=5)
    g = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, m=m, M=32, B=2, mode="adaptive", tau=0.7, seed=3, chain0=1,
                iter=2, launch=launch, radix=radix)
    for k in range(2):
        o = oracle.airpf(synth.MODEL_NGM, synth.NGM_THETA, y, m=m, M=32, mode=oracle.MODE_ADAPTIVE, tau=0.7, seed=3,
                         chain=1 + k, iter=2, radix=radix)
        compare_filter(g, k, o, m=m, what=f"radix {radix} m={m} {launch} b={k}", min_steps=10)
        _check_stages(g, k, m, radix)


# groups spanning several CTAs' records: G islands per CTA with log2 G not a multiple of log2 r
@pytest.mark.parametrize("radix,m,G,launch", [(4, 64, 2, "steps"), (4, 64, 8, "split"), (16, 256, 8, "steps"),
                                              (8, 64, 4, "split"), (4, 256, 2, "grid")])
def test_groups_spanning_ctas(radix, m, G, launch):
    y = synth.sv_observations(25, seed=2)
    g = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, m=m, M=32, B=2, mode="always", seed=7, launch=launch,
                radix=radix, islands_per_cta=G)
    for k in range(2):
        o = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, m=m, M=32, mode=oracle.MODE_ALWAYS, seed=7, chain=k,
                         radix=radix)
        compare_filter(g, k, o, m=m, what=f"radix {radix} m={m} G={G} {launch} b={k}", min_steps=10)
        _check_stages(g, k, m, radix)


def test_grid_launch_and_always_mode():
    y = synth.ar1_observations(30, seed=1)
    for mode, launch in [("always", "steps"), ("adaptive", "grid")]:
        g = run_gpu(synth.MODEL_AR1, synth.AR1_THETA, y, m=64, M=64, B=2, mode=mode, tau=0.9, seed=6, launch=launch,
                    radix=4)
        for k in range(2):
            o = oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, m=64, M=64,
                             mode={"always": 1, "adaptive": 2}[mode], tau=0.9, seed=6, chain=k, radix=4)
            compare_filter(g, k, o, m=64, what=f"radix 4 {mode} {launch} b={k}", min_steps=10)


def test_fp32_island_choices_first_step():
    """FP32-mixed: the first step's 4-way island choices (decided exactly in integers, also where
    a group spans CTAs) and its internal draws match the oracle's wherever the oracle is not
    within 1e-5 of a threshold."""
    y = synth.sv_observations(1, seed=2)
    m, M = 256, 64
    for G in (0, 2):
        g = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, m=m, M=M, B=4, mode="always", seed=9, precision="fp32",
                    radix=4, record=7, islands_per_cta=G)
        for k in range(4):
            o = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, m=m, M=M, mode=oracle.MODE_ALWAYS, seed=9, chain=k,
                             radix=4, tie_rel=1e-5, tie_masks=True)
            n = compare_first_step(g, k, o, M=M, what=f"radix 4 fp32 G={G} b={k}")
            assert n >= 0.95 * m * M


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_toy_second_moment_radix4(precision):
    """Theorem 3 with 4-ary stages: E[(Z^N)^2] over 10^6 filters (m = r = 4, M = 2, T = 16, every
    stage interacting) within 4.5 SE of the exact r-ary pair-moment value, and outside the band
    around the value of two binary stages."""
    pi0, K, gfun = ev.toy_model(0.75, 0.75)
    y = synth.toy_observations(16, seed=3)
    gs = [gfun(v) for v in y]
    exact4 = ev.pair_moments(pi0, K, gs, 4, 2, True, radix=4)[1]
    binary = ev.pair_moments(pi0, K, gs, 4, 2, True, radix=2)[1]
    R = 1_000_000
    g = run_gpu(synth.MODEL_TOY, synth.TOY_THETA, y, m=4, M=2, B=R, mode="always", seed=23, precision=precision,
                record=0, radix=4)
    z2 = np.exp(2 * g["log_z"])
    mean, se = z2.mean(), z2.std() / np.sqrt(R)
    assert abs(mean - exact4) < 4.5 * se, (mean, exact4, se)
    assert abs(mean - binary) > 4.5 * se, (mean, binary, se)


def test_m_not_a_power_of_the_radix_is_refused():
    import paper_2312_06484_gb300 as gp
    with pytest.raises(gp.AirpfError, match="ARG"):
        gp.AIRPF(synth.MODEL_AR1, m=8, M=16, T=4, radix=4)
