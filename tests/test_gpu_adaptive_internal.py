"""Adaptive internal resampling (tau_int > 0: an island resamples only when the ESS of its
particle weights falls below tau_int M, otherwise it keeps its particles and their weights)
on the GPU.

* FP64 against the oracle element by element (ancestors, s*, ENF, log Z; the oracle flags a
  resample/keep decision within 1e-12 of its threshold as a tie) in every interaction mode and
  launch form.
* tau_int = 1 resamples at every step of a continuous model: the same run, bit for bit, as
  tau_int = 0.
* FP32-mixed: Z-hat unbiased against the Kalman likelihood.
* Refused with the gradient and output-measure records and in airpf_run_static.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import kalman
from parity_util import compare_filter, run_gpu

pytestmark = pytest.mark.gpu

MODES = {"never": oracle.MODE_NEVER, "always": oracle.MODE_ALWAYS, "adaptive": oracle.MODE_ADAPTIVE}


@pytest.mark.parametrize("tau_int", [0.5, 0.9])
@pytest.mark.parametrize("mode,launch", [("adaptive", "steps"), ("always", "steps"), ("adaptive", "cta"),
                                         ("adaptive", "split"), ("never", "grid")])
def test_ar1_matches_oracle(tau_int, mode, launch):
    y = synth.ar1_observations(40, seed=1)
    g = run_gpu(synth.MODEL_AR1, synth.AR1_THETA, y, m=16, M=64, B=2, mode=mode, tau=0.5, seed=7, chain0=3,
                iter=2, launch=launch, tau_int=tau_int)
    for b in range(2):
        o = oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, m=16, M=64, mode=MODES[mode], tau=0.5, seed=7,
                         chain=3 + b, iter=2, tau_int=tau_int)
        compare_filter(g, b, o, m=16, what=f"tau_int={tau_int} {mode} {launch} b={b}")


def test_sv_and_ngm_match_oracle():
    for model, th, y in [(synth.MODEL_SV, synth.SV_THETA, synth.sv_observations(30, 2)),
                         (synth.MODEL_NGM, synth.NGM_THETA, synth.ngm_observations(30, 5))]:
        g = run_gpu(model, th, y, m=32, M=100, B=2, mode="adaptive", tau=0.6, seed=5, tau_int=0.6)
        for b in range(2):
            o = oracle.airpf(model, th, y, m=32, M=100, mode=oracle.MODE_ADAPTIVE, tau=0.6, seed=5, chain=b,
                             tau_int=0.6)
            compare_filter(g, b, o, m=32, what=f"model {model} b={b}")


def test_threshold_one_is_resampling_every_step():
    y = synth.sv_observations(50, seed=2)
    kw = dict(m=64, M=128, B=3, mode="adaptive", tau=0.3, seed=2)
    a = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, tau_int=1.0, **kw)
    b = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, tau_int=0.0, **kw)
    np.testing.assert_array_equal(a["anc"], b["anc"])
    np.testing.assert_array_equal(a["log_z"], b["log_z"])


def test_fp32_unbiased_against_kalman():
    y = synth.ar1_observations(20, seed=1)
    th = synth.AR1_THETA
    g = run_gpu(synth.MODEL_AR1, th, y, m=4, M=16, B=4000, mode="always", tau=0.5, seed=3, precision="fp32",
                record=0, tau_int=0.2)
    ratio = np.exp(g["log_z"] - kalman.ar1_loglik(th, y))
    se = ratio.std(ddof=1) / np.sqrt(ratio.size)
    assert abs(ratio.mean() - 1.0) < 4 * se, (ratio.mean(), se)


def test_refused_combinations():
    import torch
    import paper_2312_06484_gb300 as gp
    for rec in (gp.RECORD_GRAD, gp.RECORD_MOMENTS):
        with pytest.raises(gp.AirpfError, match="UNSUPPORTED"):
            gp.AIRPF(synth.MODEL_AR1, m=4, M=16, T=5, record=rec, tau_int=0.5)
    y = torch.tensor(synth.ar1_observations(5, seed=1), device="cuda")
    th = torch.tensor(synth.AR1_THETA[None, :], device="cuda")
    lz = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gp.AirpfError, match="UNSUPPORTED"):
        gp.run_static(synth.MODEL_AR1, th, y, lz, m=4, M=16, tau_int=0.5)
