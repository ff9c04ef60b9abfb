"""Radix-r interactions (r = 4, 8; m a power of r) on the GPU against the oracle: FP64
ancestors, s*, ENF and log Z element by element in the adaptive and always modes and every
launch form, s* only at the first binary stage of a group, and the configuration check."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import compare_filter, run_gpu

pytestmark = pytest.mark.gpu


# (one CTA holds a filter of at most 16 islands of 32 threads)
@pytest.mark.parametrize("radix,m,launch", [(r, m, l) for r, m in [(4, 16), (4, 64), (8, 64), (16, 256)]
                                            for l in ("steps", "split", "cta") if l != "cta" or m <= 16])
def test_matches_oracle(radix, m, launch):
    y = synth.ngm_observations(30, seed=5)
    g = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, m=m, M=32, B=2, mode="adaptive", tau=0.7, seed=3, chain0=1,
                iter=2, launch=launch, radix=radix)
    b = int(np.log2(radix))
    for k in range(2):
        o = oracle.airpf(synth.MODEL_NGM, synth.NGM_THETA, y, m=m, M=32, mode=oracle.MODE_ADAPTIVE, tau=0.7, seed=3,
                         chain=1 + k, iter=2, radix=radix)
        compare_filter(g, k, o, m=m, what=f"radix {radix} m={m} {launch} b={k}")
        assert np.all((g["sstar"][k] - 1) % b == 0)


def test_grid_launch_and_always_mode():
    y = synth.ar1_observations(30, seed=1)
    for mode, launch in [("always", "steps"), ("adaptive", "grid")]:
        g = run_gpu(synth.MODEL_AR1, synth.AR1_THETA, y, m=64, M=64, B=2, mode=mode, tau=0.9, seed=6, launch=launch,
                    radix=4)
        for k in range(2):
            o = oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, m=64, M=64,
                             mode={"always": 1, "adaptive": 2}[mode], tau=0.9, seed=6, chain=k, radix=4)
            compare_filter(g, k, o, m=64, what=f"radix 4 {mode} {launch} b={k}")


def test_m_not_a_power_of_the_radix_is_refused():
    import paper_2312_06484_gb300 as gp
    with pytest.raises(gp.AirpfError, match="ARG"):
        gp.AIRPF(synth.MODEL_AR1, m=8, M=16, T=4, radix=4)
