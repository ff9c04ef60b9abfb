"""The gradient pass (airpf_grad) against the oracle.

In FP64 the GPU filter draws the same random numbers and, short of a flagged tie, takes the
same ancestors and s* as the oracle, so:
* the adjoint gradient equals the central differences of the oracle's log Z with the
  oracle's own lineage and s* held fixed;
* the Fisher-identity score equals the oracle's score along that lineage;
both to 1e-6 relative (the central differences' accuracy).  Keeping the states every few
steps and recomputing the rest gives the same results as keeping every step.  In FP32, on
the linear-Gaussian workload of the differentiation experiment (d_x = 8, d_y = 4), the
score's mean over runs matches the Kalman score.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import kalman

pytestmark = pytest.mark.gpu

MODES = {"never": oracle.MODE_NEVER, "always": oracle.MODE_ALWAYS, "adaptive": oracle.MODE_ADAPTIVE}


def _gpu_grad(model, theta, y, *, m, M, B=1, dx=1, dy=1, mode="adaptive", tau=0.5, seed=0, chain0=0, iter=0,
              precision="fp64", model_data=None, ckpt=0, launch="auto"):
    import torch
    import paper_2312_06484_gb300 as gp
    f = gp.AIRPF(model, m=m, M=M, T=len(y) // dy, B=B, dx=dx, dy=dy, mode=mode, tau=tau, precision=precision,
                 seed=seed, record=gp.RECORD_GRAD, model_data=model_data, ckpt=ckpt, launch=launch)
    th = torch.tensor(np.tile(np.asarray(theta, np.float64), (B, 1)), device="cuda")
    out = f.grad(th, torch.tensor(np.asarray(y, np.float64), device="cuda"), chain0=chain0, iter=iter)
    f.sync()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    f.close()
    return res


def _check_against_oracle(model, theta, y, *, m, M, mode, tau, seed, chain, iter, dx=1, dy=1,
                          model_data=None, g=None, b=0):
    kw = dict(m=m, M=M, dx=dx, dy=dy, seed=seed, chain=chain, iter=iter, model_data=model_data)
    r = oracle.airpf(model, theta, y, mode=MODES[mode], tau=tau, **kw)
    if r["tie"][0] != 0:
        return False
    ref_g = oracle.logz_fixed_gradient(model, theta, y, r["anc"], r["sstar"], **kw)
    ref_s = oracle.fisher_score(model, theta, y, r["anc"], r["sstar"], **kw)
    assert abs(g["log_z"][b] - r["log_z"]) <= 1e-10 * abs(r["log_z"])
    np.testing.assert_allclose(g["grad"][b], ref_g, rtol=1e-6, atol=1e-6 * (1 + np.abs(ref_g).max()))
    np.testing.assert_allclose(g["score"][b], ref_s, rtol=1e-6, atol=1e-6 * (1 + np.abs(ref_s).max()))
    return True


@pytest.mark.parametrize("mode", ["adaptive", "always", "never"])
def test_ar1_gradient_and_score_match_oracle(mode):
    y = synth.ar1_observations(30, seed=1)
    th = np.array([0.85, 1.1, 0.9, 1.3])
    B = 2
    g = _gpu_grad(synth.MODEL_AR1, th, y, m=8, M=32, B=B, mode=mode, tau=0.5, seed=5, chain0=3, iter=1)
    checked = sum(_check_against_oracle(synth.MODEL_AR1, th, y, m=8, M=32, mode=mode, tau=0.5, seed=5,
                                        chain=3 + b, iter=1, g=g, b=b) for b in range(B))
    assert checked >= 1


def test_lgssm_gradient_and_score_match_oracle():
    dx, dy = 3, 2
    A, C, md = synth.lg_model(dx, dy, seed=11)
    th = synth.lg_theta(A, q=0.1, r=0.5)
    y = synth.lg_observations(A, C, 0.1, 0.5, 20, seed=11)
    g = _gpu_grad(synth.MODEL_LGSSM, th, y, m=4, M=32, dx=dx, dy=dy, mode="adaptive", tau=0.5, seed=2,
                  model_data=md)
    assert _check_against_oracle(synth.MODEL_LGSSM, th, y, m=4, M=32, mode="adaptive", tau=0.5, seed=2, chain=0,
                                 iter=0, dx=dx, dy=dy, model_data=md, g=g)


@pytest.mark.parametrize("launch", ["steps", "split", "cta"])
def test_checkpoint_stride_and_launch_do_not_change_the_result(launch):
    y = synth.ar1_observations(40, seed=2)
    th = np.array(synth.AR1_THETA, float)
    kw = dict(m=16, M=64, mode="adaptive", tau=0.5, seed=8, launch=launch)
    every = _gpu_grad(synth.MODEL_AR1, th, y, ckpt=0, **kw)
    sparse = _gpu_grad(synth.MODEL_AR1, th, y, ckpt=7, **kw)
    np.testing.assert_allclose(sparse["grad"], every["grad"], rtol=1e-12)
    np.testing.assert_allclose(sparse["score"], every["score"], rtol=1e-12)
    assert sparse["log_z"][0] == every["log_z"][0]


def test_fp32_score_estimates_the_kalman_score_lgssm_dx8():
    """The differentiation workload's model (d_x = 8, d_y = 4, Q = 0.1 I, R = 0.5 I) on a
    shorter series and fewer particles: the FP32 Fisher score averaged over runs equals the
    Kalman score within Monte-Carlo error, and the FP32 adjoint is close to the FP64 one."""
    dx, dy, T = 8, 4, 30
    A, C, md = synth.lg_model(dx, dy, seed=4)
    th = synth.lg_theta(A, q=0.1, r=0.5)
    y = synth.lg_observations(A, C, 0.1, 0.5, T, seed=4)
    R = 24
    g = _gpu_grad(synth.MODEL_LGSSM, th, y, m=64, M=128, B=R, dx=dx, dy=dy, mode="adaptive", tau=0.3, seed=1,
                  precision="fp32", model_data=md, ckpt=5)
    assert np.all(np.isfinite(g["score"])) and np.all(np.isfinite(g["grad"]))
    ref = np.zeros(dx + 2)
    for d in range(dx + 2):
        h = 1e-5
        tp, tm = th.copy(), th.copy()
        tp[d] += h
        tm[d] -= h
        ref[d] = (kalman.lg_loglik(tp, md, y, dx, dy) - kalman.lg_loglik(tm, md, y, dx, dy)) / (2 * h)
    mean = g["score"].mean(axis=0)
    se = g["score"].std(axis=0, ddof=1) / np.sqrt(R)
    assert np.all(np.abs(mean - ref) < 4 * se + 0.05 * np.abs(ref) + 0.5), (mean, ref, se)
    g64 = _gpu_grad(synth.MODEL_LGSSM, th, y, m=64, M=128, B=2, dx=dx, dy=dy, mode="adaptive", tau=0.3, seed=1,
                    precision="fp64", model_data=md)
    assert np.all(np.abs(g["grad"][:2] - g64["grad"]) <= 0.05 * np.abs(g64["grad"]) + 0.5)


@pytest.mark.parametrize("model,theta,ymaker,tau", [
    (synth.MODEL_SV, [-1.0, 0.9, 0.35], lambda T: synth.sv_observations(T, 2), 0.5),
    (synth.MODEL_NGM, [10.0, 1.0, 5.0], lambda T: synth.ngm_observations(T, 5), 0.5),
])
def test_nonlinear_models_gradient_and_score_match_oracle(model, theta, ymaker, tau):
    """SV (theta = mu, phi, sigma; the stationary prior depends on all three) and NGM
    (theta = q, r, p0), FP64, against the oracle's references."""
    y = ymaker(25)
    th = np.asarray(theta, float)
    B = 2
    g = _gpu_grad(model, th, y, m=8, M=32, B=B, mode="adaptive", tau=tau, seed=6, chain0=1, iter=2)
    checked = sum(_check_against_oracle(model, th, y, m=8, M=32, mode="adaptive", tau=tau, seed=6, chain=1 + b,
                                        iter=2, g=g, b=b) for b in range(B))
    assert checked >= 1


def test_autograd_log_z_matches_gpu_finite_differences():
    """log_z(...).backward() leaves the adjoint gradient in theta.grad; it equals central
    differences of the GPU filter's own FP64 log Z at the same streams (a perturbation of
    1e-6 changes no ancestor, island choice or s* here), and the oracle's gradient."""
    import torch
    import paper_2312_06484_gb300 as gp
    y = synth.ar1_observations(30, seed=1)
    th0 = np.array([0.85, 1.1, 0.9, 1.3])
    kw = dict(m=8, M=32, T=len(y), B=1, mode="adaptive", tau=0.5, precision="fp64", seed=5)
    f = gp.AIRPF(synth.MODEL_AR1, record=gp.RECORD_GRAD, **kw)
    yy = torch.tensor(y, device="cuda")
    th = torch.tensor(th0, device="cuda", requires_grad=True)
    lz = gp.log_z(f, th, yy, chain0=3, iter=1)
    lz.sum().backward()
    f.sync()
    g = th.grad.cpu().numpy()
    f.close()
    plain = gp.AIRPF(synth.MODEL_AR1, record=0, **kw)

    def logz_at(v):
        out = plain.run(torch.tensor(v[None, :], device="cuda"), yy, chain0=3, iter=1)
        plain.sync()
        return float(out["log_z"][0])

    assert logz_at(th0) == float(lz.detach()[0])
    fd = np.zeros(4)
    for d in range(4):
        h = 1e-6 * max(1.0, abs(th0[d]))
        tp, tm = th0.copy(), th0.copy()
        tp[d] += h
        tm[d] -= h
        fd[d] = (logz_at(tp) - logz_at(tm)) / (2 * h)
    plain.close()
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6)
    r = oracle.airpf(synth.MODEL_AR1, th0, y, m=8, M=32, mode=oracle.MODE_ADAPTIVE, tau=0.5, seed=5, chain=3, iter=1)
    if r["tie"][0] == 0:
        ref = oracle.logz_fixed_gradient(synth.MODEL_AR1, th0, y, r["anc"], r["sstar"], m=8, M=32, seed=5, chain=3,
                                         iter=1)
        np.testing.assert_allclose(g, ref, rtol=1e-6, atol=1e-6 * (1 + np.abs(ref).max()))
