"""The output measures (airpf_moments) against the oracle.

In FP64 the GPU and the oracle hold the same particles and island weights at every step
before the first flagged tie, so the moments E[x_d] and E[x_d^2] of the prediction filter
(the mutated particles with W_{t,0}) and of the filter (the internally resampled particles
with W_{t,1}) agree to rounding (the sums run in another order).  Every launch form gives the
same bits, and the FP32-mixed moments are close to the FP64 ones.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _gpu(model, theta, y, *, m, M, B, dx=1, dy=1, mode="adaptive", tau=0.3, seed=0, chain0=0, iter=0,
         precision="fp64", model_data=None, launch="auto"):
    import torch
    import paper_2312_06484_gb300 as gp
    f = gp.AIRPF(model, m=m, M=M, T=len(y) // dy, B=B, dx=dx, dy=dy, mode=mode, tau=tau, precision=precision,
                 seed=seed, record=gp.RECORD_MOMENTS, model_data=model_data, launch=launch)
    th = torch.tensor(np.tile(np.asarray(theta, np.float64), (B, 1)), device="cuda")
    out = f.run(th, torch.tensor(np.asarray(y, np.float64), device="cuda"), chain0=chain0, iter=iter)
    mom = f.moments()
    f.sync()
    res = mom.cpu().numpy(), out["log_z"].cpu().numpy(), f.launch_mode
    f.close()
    return res


def _check(model, theta, y, *, m, M, B=2, dx=1, dy=1, mode="adaptive", tau=0.3, seed=0, model_data=None):
    g, lz, _ = _gpu(model, theta, y, m=m, M=M, B=B, dx=dx, dy=dy, mode=mode, tau=tau, seed=seed, chain0=1,
                    iter=2, model_data=model_data)
    checked = 0
    for b in range(B):
        o = oracle.airpf(model, theta, y, m=m, M=M, dx=dx, dy=dy, mode={"adaptive": 2, "always": 1, "never": 0}[mode],
                         tau=tau, seed=seed, chain=1 + b, iter=2, model_data=model_data, moments=True)
        T = o["moments"].shape[0]
        upto = T if o["tie"][0] == 0 else o["tie"][0] - 1
        if upto == 0:
            continue
        ref = o["moments"][:upto]
        # rounding of sums in another order: relative to the value, and to E[x^2] where the
        # mean is near 0
        tol = 1e-9 * np.abs(ref) + 1e-12 * (np.abs(ref[:, :, 1:2, :]) + 1.0)
        err = np.abs(g[b, :upto] - ref)
        assert np.all(err <= tol), (b, float((err / tol).max()))
        checked += 1
    assert checked >= 1
    return g


@pytest.mark.parametrize("mode", ["adaptive", "always", "never"])
def test_ar1_moments_match_oracle(mode):
    y = synth.ar1_observations(30, seed=1)
    _check(synth.MODEL_AR1, synth.AR1_THETA, y, m=16, M=64, mode=mode, tau=0.5, seed=7)


def test_sv_ragged_island_moments_match_oracle():
    """M = 37: no particle run is a whole vector (the per-particle path)."""
    y = synth.sv_observations(25, seed=2)
    _check(synth.MODEL_SV, synth.SV_THETA, y, m=32, M=37, tau=0.8, seed=4)


def test_lgssm_moments_match_oracle():
    dx, dy = 3, 2
    A, C, md = synth.lg_model(dx, dy, seed=11)
    th = synth.lg_theta(A, q=0.1, r=0.5)
    y = synth.lg_observations(A, C, 0.1, 0.5, 20, seed=11)
    _check(synth.MODEL_LGSSM, th, y, m=8, M=32, dx=dx, dy=dy, tau=0.5, seed=2, model_data=md)


def test_changepoint_moments_match_oracle():
    y = synth.cp_observations(523, seed=6)[:2 * 30]
    _check(synth.MODEL_CP, synth.CP_THETA, y, m=64, M=200, dy=2, seed=3)


def test_moments_do_not_depend_on_the_launch_form():
    y = synth.ngm_observations(20, seed=5)
    kw = dict(m=16, M=64, B=2, mode="adaptive", tau=0.5, seed=9)
    ref, lz_ref, _ = _gpu(synth.MODEL_NGM, synth.NGM_THETA, y, launch="steps", **kw)
    for launch in ("cta", "grid", "split"):
        g, lz, mode = _gpu(synth.MODEL_NGM, synth.NGM_THETA, y, launch=launch, **kw)
        np.testing.assert_array_equal(g, ref, err_msg=launch)
        np.testing.assert_array_equal(lz, lz_ref, err_msg=launch)


def test_fp32_moments_close_to_fp64():
    """The SV workload's size on a shortened series: FP32-mixed moments within a small part
    of the filter's spread of the FP64 ones (same streams)."""
    y = synth.sv_observations(1000, seed=2)[:50]
    a, _, _ = _gpu(synth.MODEL_SV, synth.SV_THETA, y, m=1024, M=256, B=1, seed=1, precision="fp64")
    b, _, _ = _gpu(synth.MODEL_SV, synth.SV_THETA, y, m=1024, M=256, B=1, seed=1, precision="fp32")
    sd = np.sqrt(a[:, :, :, 1, :] - a[:, :, :, 0, :] ** 2)
    assert np.all(np.abs(b[:, :, :, 0, :] - a[:, :, :, 0, :]) < 0.1 * sd)
