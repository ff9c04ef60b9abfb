"""Statistical checks of the CUDA path through the C ABI (both precisions):

* Theorem 1 (lack of bias): over 1000 independent filters of the AR(1) workload
  (m=16 x M=64 x T=100), mean Z^N / Z_Kalman lies within 4.5 standard errors of 1; also on
  a small linear-Gaussian model;
* the FP32-mixed path's log Z has the distribution of the FP64 path's (mean within 4.5
  standard errors of the difference, SD ratio within 15%);
* Theorem 3: on the binary HMM of Section 4.1 (m=4 x M=2, T=12) the empirical E[(Z^N)^2]
  over 10^6 filters lies within 4.5 standard errors of the exact pair-moment value, for
  always / never interaction and for the m=1 bootstrap filter, and the band excludes the
  other interaction mode's exact value."""
import numpy as np
import pytest

import synth
from oracle import exact_variance as ev
from oracle import kalman
from parity_util import run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mode", ["adaptive", "always", "never"])
def test_unbiased_against_kalman(gpu_lib, precision, mode):
    y = synth.ar1_observations(100, seed=1)
    z = kalman.ar1_loglik(synth.AR1_THETA, y)
    g = run_gpu(synth.MODEL_AR1, synth.AR1_THETA, y, m=16, M=64, B=1000, mode=mode, tau=0.3, seed=3,
                precision=precision, record=0)
    r = np.exp(g["log_z"] - z)
    assert np.all(np.isfinite(r))
    assert abs(r.mean() - 1.0) < 4.5 * r.std() / np.sqrt(len(r)), (r.mean(), r.std())


def test_unbiased_lgssm_fp32(gpu_lib):
    dx, dy = 3, 2
    A, C, md = synth.lg_model(dx, dy, seed=11)
    th = synth.lg_theta(A, q=0.1, r=0.5)
    y = synth.lg_observations(A, C, 0.1, 0.5, 30, seed=11)
    z = kalman.lg_loglik(th, md, y, dx, dy)
    g = run_gpu(synth.MODEL_LGSSM, th, y, m=16, M=32, B=1000, dx=dx, dy=dy, model_data=md,
                mode="adaptive", tau=0.5, seed=4, precision="fp32", record=0)
    r = np.exp(g["log_z"] - z)
    assert abs(r.mean() - 1.0) < 4.5 * r.std() / np.sqrt(len(r))


def test_fp32_distribution_matches_fp64(gpu_lib):
    y = synth.sv_observations(200, seed=2)
    kw = dict(m=64, M=64, B=1000, mode="adaptive", tau=0.3, record=0)
    a = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, seed=5, precision="fp32", **kw)["log_z"]
    b = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, seed=6, precision="fp64", **kw)["log_z"]
    se = np.sqrt(a.var() / len(a) + b.var() / len(b))
    assert abs(a.mean() - b.mean()) < 4.5 * se, (a.mean(), b.mean(), se)
    assert 0.85 < a.std() / b.std() < 1.15


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_toy_second_moment_matches_theorem3(gpu_lib, precision):
    pi0, K, gfun = ev.toy_model(0.75, 0.75)
    y = synth.toy_observations(12, seed=3)
    gs = [gfun(v) for v in y]
    exact = {"always": ev.pair_moments(pi0, K, gs, 4, 2, True)[1],
             "never": ev.pair_moments(pi0, K, gs, 4, 2, False)[1],
             "bpf": ev.pair_moments(pi0, K, gs, 1, 8, False)[1]}
    R = 1_000_000
    for name, m, M, mode, other in [("always", 4, 2, "always", "never"), ("never", 4, 2, "never", "always"),
                                    ("bpf", 1, 8, "always", "never")]:
        g = run_gpu(synth.MODEL_TOY, synth.TOY_THETA, y, m=m, M=M, B=R, mode=mode, seed=17,
                    precision=precision, record=0)
        z2 = np.exp(2 * g["log_z"])
        mean, se = z2.mean(), z2.std() / np.sqrt(R)
        assert abs(mean - exact[name]) < 4.5 * se, (name, mean, exact[name], se)
        assert abs(mean - exact[other]) > 4.5 * se, (name, "cannot separate from", other)
