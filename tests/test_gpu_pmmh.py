"""The device PMMH driver (random-walk particle marginal Metropolis-Hastings over AIRPF
likelihood estimates) against the oracle's chain.

In FP64 the GPU chain and the oracle chain draw the same proposals and acceptance
uniforms from the same counter-based streams and run the same filters, so, short of a
resampling or acceptance tie, they take the same accept decisions: the recorded chain
states agree to rounding and the acceptance counts are equal.  Resuming a chain by a
second call continues it exactly.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

AR1_KW = dict(m=16, M=64, mode="adaptive", tau=0.3)
STEP = [0.05, 0.0, 0.0, 0.0]
LO, HI = [-1.0, 0.0, 0.0, 0.0], [1.0, 0.0, 0.0, 0.0]


def _gpu_chain(model, theta0, y, *, B=1, iters, step, lo, hi, m, M, mode, tau, seed, chain0=0,
               launch="auto", splits=None, precision="fp64", state_logz=float("nan")):
    import torch
    import paper_2312_06484_gb300 as gp
    f = gp.AIRPF(model, m=m, M=M, T=len(y), B=B, mode=mode, tau=tau, precision=precision, seed=seed,
                 launch=launch)
    th = torch.tensor(np.tile(np.asarray(theta0, np.float64), (B, 1)), device="cuda")
    lz = torch.full((B,), state_logz, dtype=torch.float64, device="cuda")
    yy = torch.tensor(np.asarray(y, np.float64), device="cuda")
    acc = torch.zeros(B, dtype=torch.int32, device="cuda")
    thetas, logzs = [], []
    it0 = 0
    for n in (splits or [iters]):
        out = f.pmmh(yy, th, lz, step=step, lo=lo, hi=hi, iters=n, chain0=chain0, iter0=it0, n_accept=acc)
        thetas.append(out["theta"])
        logzs.append(out["log_z"])
        it0 += n
    f.sync()
    res = dict(theta=torch.cat(thetas).cpu().numpy(), log_z=torch.cat(logzs).cpu().numpy(),
               n_accept=acc.cpu().numpy(), launch_mode=f.launch_mode, launches=f.launch_count())
    f.close()
    return res


def _oracle_chain(model, theta0, y, *, iters, step, lo, hi, m, M, mode, tau, seed, chain):
    return oracle.pmmh(model, theta0, y, m=m, M=M, step=step, lo=lo, hi=hi, iters=iters,
                       mode={"never": 0, "always": 1, "adaptive": 2}[mode], tau=tau, seed=seed, chain=chain)


def _assert_same_chain(g, b, o, what):
    np.testing.assert_allclose(g["theta"][:, b, :], o["theta"], rtol=1e-12, atol=1e-14, err_msg=what)
    np.testing.assert_allclose(g["log_z"][:, b], o["logz"], rtol=1e-10, atol=1e-12, err_msg=what)
    assert int(g["n_accept"][b]) == o["n_accept"], (what, g["n_accept"][b], o["n_accept"])


@pytest.mark.parametrize("launch", ["steps", "cta"])
def test_pmmh_chain_matches_oracle_ar1(launch):
    y = synth.ar1_observations(100, seed=1)
    theta0 = [0.5, 1.0, 1.0, 1.0]
    g = _gpu_chain(synth.MODEL_AR1, theta0, y, iters=40, step=STEP, lo=LO, hi=HI, seed=3, launch=launch,
                   **AR1_KW)
    o = _oracle_chain(synth.MODEL_AR1, theta0, y, iters=40, step=STEP, lo=LO, hi=HI, seed=3, chain=0,
                      **AR1_KW)
    _assert_same_chain(g, 0, o, f"AR1 PMMH launch={launch}")
    assert 0 < o["n_accept"] < 40


def test_pmmh_batch_of_chains_and_resume():
    """Four chains (chain0 = 5..8) in one batch, run as two calls of 15 iterations: each
    chain equals the oracle's 30-iteration chain of the same index."""
    y = synth.ar1_observations(60, seed=2)
    theta0 = [0.3, 1.0, 1.0, 1.0]
    kw = dict(m=8, M=32, mode="always", tau=0.3, step=STEP, lo=LO, hi=HI, seed=11)
    g = _gpu_chain(synth.MODEL_AR1, theta0, y, B=4, iters=30, chain0=5, splits=[15, 15], launch="steps", **kw)
    for b in range(4):
        o = _oracle_chain(synth.MODEL_AR1, theta0, y, iters=30, chain=5 + b, **kw)
        _assert_same_chain(g, b, o, f"chain {5 + b}")


def test_pmmh_rejects_outside_the_prior_box():
    """Started next to the edge of U(-1, 1) with a wide step, many proposals leave the box;
    they are rejected without a filter pass, exactly as in the oracle."""
    y = synth.ar1_observations(40, seed=4)
    theta0 = [0.97, 1.0, 1.0, 1.0]
    kw = dict(m=4, M=32, mode="adaptive", tau=0.5, step=[0.2, 0, 0, 0], lo=LO, hi=HI, seed=21)
    g = _gpu_chain(synth.MODEL_AR1, theta0, y, iters=40, **kw)
    o = _oracle_chain(synth.MODEL_AR1, theta0, y, iters=40, chain=0, **kw)
    _assert_same_chain(g, 0, o, "edge of the prior box")
    assert np.all(np.abs(g["theta"][:, 0, 0]) <= 1.0)


def test_pmmh_sv_three_parameters():
    """SV with proposals on (mu, phi, sigma) under a box prior; phi's domain |phi| < 1."""
    y = synth.sv_observations(50, seed=1)
    theta0 = list(synth.SV_THETA)
    kw = dict(m=32, M=32, mode="adaptive", tau=0.3, step=[0.05, 0.01, 0.02], lo=[-5.0, -1.0, 0.0],
              hi=[5.0, 1.0, 2.0], seed=7)
    g = _gpu_chain(synth.MODEL_SV, theta0, y, iters=25, launch="steps", **kw)
    o = _oracle_chain(synth.MODEL_SV, theta0, y, iters=25, chain=0, **kw)
    _assert_same_chain(g, 0, o, "SV PMMH")


def test_pmmh_fp32_chain_is_valid():
    """FP32-mixed likelihood estimates: the chain stays in the prior box, its log Z are
    finite and it accepts some but not all proposals."""
    y = synth.ar1_observations(100, seed=1)
    g = _gpu_chain(synth.MODEL_AR1, [0.5, 1, 1, 1], y, iters=60, step=STEP, lo=LO, hi=HI, seed=3,
                   precision="fp32", **AR1_KW)
    assert np.all(np.isfinite(g["log_z"]))
    assert np.all(np.abs(g["theta"][:, 0, 0]) <= 1.0)
    assert 0 < g["n_accept"][0] < 60


def _gpu_langevin(theta0, y, *, iters, splits=None, **kw):
    import torch
    import paper_2312_06484_gb300 as gp
    f = gp.AIRPF(synth.MODEL_AR1, m=kw["m"], M=kw["M"], T=len(y), B=1, mode=kw["mode"], tau=kw["tau"],
                 precision="fp64", seed=kw["seed"], record=gp.RECORD_GRAD)
    th = torch.tensor(np.asarray(theta0, np.float64)[None, :], device="cuda")
    lz = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.zeros_like(th)
    yy = torch.tensor(np.asarray(y, np.float64), device="cuda")
    acc = torch.zeros(1, dtype=torch.int32, device="cuda")
    thetas, logzs, it0 = [], [], 0
    for n in (splits or [iters]):
        out = f.pmmh_langevin(yy, th, lz, g, step=kw["step"], lo=kw["lo"], hi=kw["hi"], iters=n, iter0=it0,
                              n_accept=acc)
        thetas.append(out["theta"])
        logzs.append(out["log_z"])
        it0 += n
    f.sync()
    res = dict(theta=torch.cat(thetas).cpu().numpy()[:, 0, :], log_z=torch.cat(logzs).cpu().numpy()[:, 0],
               n_accept=int(acc.item()))
    f.close()
    return res


LANGEVIN = dict(m=8, M=32, mode="adaptive", tau=0.5, seed=13, step=[0.08, 0.05, 0.0, 0.0],
                lo=[-1.0, 0.1, 0.0, 0.0], hi=[1.0, 3.0, 0.0, 0.0])


def test_langevin_pmmh_chain_matches_oracle():
    """FP64 Langevin chain on AR(1) (a and sigma_v move): the GPU's proposals use the GPU
    score, the oracle's its own; both agree to rounding, so the chains take the same
    decisions."""
    y = synth.ar1_observations(30, seed=1)
    theta0 = [0.5, 1.0, 1.0, 1.0]
    g = _gpu_langevin(theta0, y, iters=10, **LANGEVIN)
    kw = dict(LANGEVIN)
    kw["mode"] = {"never": 0, "always": 1, "adaptive": 2}[kw["mode"]]
    o = oracle.pmmh_langevin(synth.MODEL_AR1, theta0, y, iters=10, chain=0, **kw)
    np.testing.assert_allclose(g["theta"], o["theta"], rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(g["log_z"], o["logz"], rtol=1e-7)
    assert g["n_accept"] == o["n_accept"]
    assert 0 < o["n_accept"] <= 10


def test_langevin_pmmh_resume_continues_the_chain():
    """A chain run as 3 + 5 iterations (the state theta, log Z and gradient carried by the
    caller) takes the same decisions as one call of 8.  The backward pass scatter-adds each
    particle's adjoint into its parent with atomic adds whose order varies from run to run,
    so gradients, hence Langevin proposals, agree to rounding rather than bit for bit."""
    y = synth.ar1_observations(30, seed=1)
    full = _gpu_langevin([0.5, 1.0, 1.0, 1.0], y, iters=8, **LANGEVIN)
    split = _gpu_langevin([0.5, 1.0, 1.0, 1.0], y, iters=8, splits=[3, 5], **LANGEVIN)
    np.testing.assert_allclose(split["theta"], full["theta"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(split["log_z"], full["log_z"], rtol=1e-12)
    assert full["n_accept"] == split["n_accept"]
