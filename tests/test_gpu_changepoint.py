"""The change-point model (Section 4.2: Beta jump kernel, binomial counts) on the GPU.

* FP64 against the oracle element by element (ancestors bit-exact before the first flagged
  tie, s*, ENF, log Z within 1e-10 relative) at the workload's sizes m = 64 x M = 200 and
  M = 500 (neither a power of 2) on a shortened series, in every interaction mode.
* The closed-form ends p = 0 and p = 1 (beta-binomial likelihoods): the mean of Z-hat over
  independent GPU runs matches, as it must for an unbiased estimator.
* FP32 against FP64 on the same streams.
* The PMMH chain on p equals the oracle's chain.
* The gradient record is refused (the jump is discrete).
"""
import numpy as np
import pytest
from scipy import special

import oracle
import synth
from parity_util import compare_filter

pytestmark = pytest.mark.gpu

CP = synth.MODEL_CP
MODES = {"never": oracle.MODE_NEVER, "always": oracle.MODE_ALWAYS, "adaptive": oracle.MODE_ADAPTIVE}


def _run(theta, y, *, m, M, B, mode="adaptive", tau=0.3, seed=0, chain0=0, iter=0, precision="fp64", record=7):
    import torch
    import paper_2312_06484_gb300 as gp
    f = gp.AIRPF(CP, m=m, M=M, T=len(y) // 2, B=B, dy=2, mode=mode, tau=tau, precision=precision, seed=seed,
                 record=record)
    th = torch.tensor(np.asarray(theta, np.float64), device="cuda")
    if th.ndim == 1:
        th = th[None, :].repeat(B, 1)
    out = f.run(th, torch.tensor(np.asarray(y, np.float64), device="cuda"), chain0=chain0, iter=iter,
                lineage=bool(record & 1), enf=bool(record & 2), trace=bool(record & 4))
    f.sync()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    f.close()
    return res


@pytest.mark.parametrize("M,T", [(200, 40), (500, 15)])
@pytest.mark.parametrize("mode", ["adaptive", "always", "never"])
def test_fp64_matches_oracle(M, T, mode):
    y = synth.cp_observations(523, seed=6)[: 2 * T]
    th = np.array([0.1, 2.0, 20.0])
    g = _run(th, y, m=64, M=M, B=2, mode=mode, tau=0.3, seed=3, chain0=1, iter=2)
    for b in range(2):
        o = oracle.airpf(CP, th, y, m=64, M=M, mode=MODES[mode], tau=0.3, dy=2, seed=3, chain=1 + b, iter=2)
        compare_filter(g, b, o, m=64, what=f"changepoint M={M} {mode} b={b}")


def test_boosted_gamma_branch_matches_oracle():
    """alpha < 1 and beta < 1 take the boosted gamma draws."""
    y = synth.cp_observations(30, seed=9, theta=[0.2, 0.6, 0.8])
    th = np.array([0.2, 0.6, 0.8])
    g = _run(th, y, m=16, M=64, B=2, seed=5)
    for b in range(2):
        o = oracle.airpf(CP, th, y, m=16, M=64, mode=oracle.MODE_ADAPTIVE, tau=0.3, dy=2, seed=5, chain=b)
        compare_filter(g, b, o, m=16, what=f"boosted b={b}")


def _lz_exact(y, p, alpha, beta):
    k, n = y[0::2], y[1::2]
    logc = special.gammaln(n + 1) - special.gammaln(k + 1) - special.gammaln(n - k + 1)
    if p == 0.0:
        return logc.sum() + special.betaln(alpha + k.sum(), beta + (n - k).sum()) - special.betaln(alpha, beta)
    return (logc + special.betaln(alpha + k, beta + n - k) - special.betaln(alpha, beta)).sum()


@pytest.mark.parametrize("p", [0.0, 1.0])
def test_unbiased_at_closed_form_ends(p):
    alpha, beta = 2.0, 5.0
    y = synth.cp_observations(6, seed=11, theta=[0.3, alpha, beta], n_lo=5, n_hi=15)
    g = _run([p, alpha, beta], y, m=4, M=32, B=2000, mode="adaptive", tau=0.5, seed=2, record=0)
    ratio = np.exp(g["log_z"] - _lz_exact(y, p, alpha, beta))
    se = ratio.std(ddof=1) / np.sqrt(ratio.size)
    assert abs(ratio.mean() - 1.0) < 4 * se + 1e-3, (ratio.mean(), se)


def test_fp32_matches_fp64_in_distribution():
    """Same streams, FP32-mixed against FP64 at the workload's size (m = 64 x M = 200, the
    full T = 523): the log Z of 64 filters agree on average to well inside their spread."""
    y = synth.cp_observations(523, seed=6)
    th = synth.CP_THETA
    a = _run(th, y, m=64, M=200, B=64, seed=1, precision="fp64", record=0)["log_z"]
    b = _run(th, y, m=64, M=200, B=64, seed=1, precision="fp32", record=0)["log_z"]
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(b))
    d = b - a
    assert abs(d.mean()) < 4 * a.std(ddof=1) / np.sqrt(a.size) + 0.05, (d.mean(), a.std())


def test_pmmh_chain_on_p_matches_oracle():
    import torch
    import paper_2312_06484_gb300 as gp
    y = synth.cp_observations(60, seed=6)
    th0 = np.array([0.05, 2.0, 20.0])
    step, lo, hi = [0.02, 0.0, 0.0], [0.0, 2.0, 20.0], [1.0, 2.0, 20.0]
    f = gp.AIRPF(CP, m=16, M=64, T=60, B=1, dy=2, mode="adaptive", tau=0.3, precision="fp64", seed=4)
    th = torch.tensor(th0[None, :], device="cuda")
    lz = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    acc = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = f.pmmh(torch.tensor(y, device="cuda"), th, lz, step=step, lo=lo, hi=hi, iters=30, chain0=0, iter0=0,
                 n_accept=acc)
    f.sync()
    g_th, g_lz, g_acc = out["theta"].cpu().numpy(), out["log_z"].cpu().numpy(), int(acc.cpu()[0])
    f.close()
    o = oracle.pmmh(CP, th0, y, m=16, M=64, step=step, lo=lo, hi=hi, iters=30, mode=2, tau=0.3, dy=2, seed=4,
                    chain=0)
    np.testing.assert_allclose(g_th[:, 0, :], o["theta"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(g_lz[:, 0], o["logz"], rtol=1e-10, atol=1e-12)
    assert g_acc == o["n_accept"]
    assert 0 < g_acc < 30


def test_gradient_record_is_refused():
    import paper_2312_06484_gb300 as gp
    with pytest.raises(gp.AirpfError, match="UNSUPPORTED"):
        gp.AIRPF(CP, m=4, M=32, T=5, dy=2, record=gp.RECORD_GRAD)
