"""Batched chains of uneven size (one context per (m, M) class, run side by side as a group)
and the tiling autotuner.

* FP64: every chain of a group equals the oracle's run of the same chain index (log Z to
  the parity tolerance, when the oracle flags no tie);
* the group's results equal each member run on its own (the group only orders streams);
* group PMMH equals member-by-member PMMH;
* the autotuner returns a tiling whose pass computes the default tiling's log Z.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _classes(ms, Ms):
    """Chains grouped by (m, M); a class's chains get contiguous chain indices."""
    keys = sorted(set(zip(ms.tolist(), Ms.tolist())))
    members, base = [], 0
    for key in keys:
        idx = [i for i in range(len(ms)) if (ms[i], Ms[i]) == key]
        members.append((key, idx, base))
        base += len(idx)
    return members


def _make_group(members, thetas, T, precision, seed, **kw):
    import torch
    import paper_2312_06484_gb300 as gp
    ctxs, th, c0 = [], [], []
    for (m, M), idx, base in members:
        ctxs.append(gp.AIRPF(synth.MODEL_SV, m=m, M=M, T=T, B=len(idx), mode="adaptive", tau=0.3,
                             precision=precision, seed=seed, stream=torch.cuda.Stream(), **kw))
        th.append(torch.tensor(thetas[idx], device="cuda"))
        c0.append(base)
    return ctxs, th, c0


def test_group_fp64_chains_match_oracle():
    import torch
    import paper_2312_06484_gb300 as gp
    rng = np.random.default_rng(3)
    n, T = 10, 30
    ms = rng.choice([4, 8, 16], n)
    Ms = rng.choice([16, 32], n)
    thetas, _ = synth.batched_sv_thetas(n, seed=7)
    y = synth.sv_observations(T, seed=2)
    members = _classes(ms, Ms)
    ctxs, th, c0 = _make_group(members, thetas, T, "fp64", seed=5)
    grp = gp.Group(ctxs)
    out = grp.run(th, torch.tensor(y, device="cuda"), c0, iter=2)
    grp.sync()
    checked = 0
    for ((m, M), idx, base), lz in zip(members, out):
        lz = lz.cpu().numpy()
        for b, i in enumerate(idx):
            o = oracle.airpf(synth.MODEL_SV, thetas[i], y, m=m, M=M, mode=oracle.MODE_ADAPTIVE, tau=0.3, seed=5,
                             chain=base + b, iter=2)
            if o["tie"][0] == 0:
                assert abs(lz[b] - o["log_z"]) <= 1e-10 * abs(o["log_z"]), (m, M, b, lz[b], o["log_z"])
                checked += 1
    assert checked >= n - 1
    grp.close()


def test_group_equals_members_alone_config3_sizes():
    """The size classes of the batched serving workload (m in {64..4096}, M in {32..1024},
    32 chains, FP32): a group pass equals each member's pass alone, bit for bit."""
    import torch
    import paper_2312_06484_gb300 as gp
    n, T = 32, 12
    ms, Ms = synth.batched_sizes(n, seed=8)
    thetas, _ = synth.batched_sv_thetas(n, seed=7)
    y = torch.tensor(synth.sv_observations(T, seed=2), device="cuda")
    members = _classes(ms, Ms)
    ctxs, th, c0 = _make_group(members, thetas, T, "fp32", seed=9)
    grp = gp.Group(ctxs)
    together = [t.cpu().numpy() for t in grp.run(th, y, c0, iter=4)]
    grp.sync()
    for ctx, t, c, tog in zip(ctxs, th, c0, together):
        alone = ctx.run(t, y, chain0=c, iter=4)["log_z"]
        ctx.sync()
        assert np.array_equal(alone.cpu().numpy(), tog)
        assert np.all(np.isfinite(tog))
    grp.close()


def test_group_pmmh_equals_member_pmmh():
    import torch
    import paper_2312_06484_gb300 as gp
    rng = np.random.default_rng(11)
    n, T, iters = 6, 25, 4
    ms = rng.choice([4, 8], n)
    Ms = rng.choice([16, 32], n)
    thetas, _ = synth.batched_sv_thetas(n, seed=3)
    y = torch.tensor(synth.sv_observations(T, seed=2), device="cuda")
    members = _classes(ms, Ms)
    kw = dict(step=[0.05, 0.01, 0.02], lo=[-5.0, -1.0, 0.0], hi=[5.0, 1.0, 2.0], iters=iters)
    ctxs, th, c0 = _make_group(members, thetas, T, "fp64", seed=2)
    grp = gp.Group(ctxs)
    st_th = [t.clone() for t in th]
    st_lz = [torch.full((t.shape[0],), float("nan"), dtype=torch.float64, device="cuda") for t in th]
    res = grp.pmmh(y, st_th, st_lz, chain0s=c0, record=True, **kw)
    grp.sync()
    for i, ctx in enumerate(ctxs):
        a_th = th[i].clone()
        a_lz = torch.full((th[i].shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        alone = ctx.pmmh(y, a_th, a_lz, chain0=c0[i], **kw)
        ctx.sync()
        assert torch.equal(alone["theta"], res["theta"][i])
        assert torch.equal(alone["log_z"], res["log_z"][i])
        assert torch.equal(alone["n_accept"], res["n_accept"][i])
        assert torch.equal(a_th, st_th[i])
    grp.close()


def test_autotune_picks_a_tiling_that_computes_the_same_pass():
    import torch
    import paper_2312_06484_gb300 as gp
    T = 20
    y = torch.tensor(synth.sv_observations(T, seed=2), device="cuda")
    th = torch.tensor(np.tile(synth.SV_THETA, (2, 1)), device="cuda")
    kw = dict(m=256, M=128, B=2, mode="adaptive", tau=0.3, precision="fp64", seed=3)
    best, ms = gp.autotune(synth.MODEL_SV, th, y, passes=2, **kw)
    assert ms > 0 and best["launch"] in (1, 2, 4) and best["ppt"] in (2, 4)
    ref = gp.AIRPF(synth.MODEL_SV, T=T, **kw)
    tuned = gp.AIRPF(synth.MODEL_SV, T=T, launch=best["launch"], ppt=best["ppt"],
                     islands_per_cta=best["islands_per_cta"], **kw)
    a = ref.run(th, y, iter=6)["log_z"].cpu().numpy()
    b = tuned.run(th, y, iter=6)["log_z"].cpu().numpy()
    np.testing.assert_allclose(b, a, rtol=1e-12)
    ref.close()
    tuned.close()
