"""Element-by-element comparison of the CUDA path with the oracle, under the tie protocol:
ancestors, s* and ENF decisions must agree exactly on every step before the first step the
oracle flags as a tie (a resampling draw, island choice or ENF test within 1e-12 relative of
its threshold); log Z within the FP64 tolerance when the run has no tie."""
import numpy as np

import oracle

LOGZ_RTOL = 1e-10      # FP64 path: relative tolerance on log Z
ENF_RTOL = 1e-10


def run_gpu(model, theta, y, *, m, M, B=1, mode, tau=0.3, dx=1, dy=1, seed=0, chain0=0, iter=0,
            model_data=None, precision="fp64", record=7, launch="auto", tau_int=0.0, radix=2, **tiling):
    """One call of AIRPF.run; tiling: ppt, islands_per_cta."""
    import torch
    import paper_2312_06484_gb300 as gp
    f = gp.AIRPF(model, m=m, M=M, T=len(y) // dy, B=B, dx=dx, dy=dy, mode=mode, tau=tau,
                 precision=precision, seed=seed, record=record, model_data=model_data, launch=launch,
                 tau_int=tau_int, radix=radix, **tiling)
    th = torch.tensor(np.tile(np.asarray(theta, np.float64), (B, 1)), device="cuda")
    if np.ndim(theta) == 2:
        th = torch.tensor(np.asarray(theta, np.float64), device="cuda")
    yy = torch.tensor(np.asarray(y, np.float64), device="cuda")
    out = f.run(th, yy, chain0=chain0, iter=iter, lineage=bool(record & 1), enf=bool(record & 2),
                trace=bool(record & 4))
    f.sync()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["launches"] = f.launch_count()
    res["launch_mode"] = f.launch_mode
    f.close()
    return res


def compare_filter(gpu, b, ora, *, m, what="", min_steps=None):
    """Compare filter b of a GPU batch with one oracle run (dict from oracle.airpf), on every
    step before the oracle's first flagged tie; at least min_steps steps must be compared
    (default: half the run, at least one)."""
    t_tie, kind = ora["tie"]
    T = ora["anc"].shape[0]
    upto = T if t_tie == 0 else t_tie - 1          # steps fully before the first tie
    need = max(1, T // 2) if min_steps is None else min(min_steps, T)
    assert upto >= need, f"{what}: only {upto} of {T} steps before the first tie (kind {kind}); need {need}"
    anc_g = gpu["anc"][b]
    diff = np.nonzero((anc_g[:upto] != ora["anc"][:upto]).any(axis=1))[0]
    assert diff.size == 0, f"{what}: ancestors differ first at step {diff[0] + 1} (tie at {t_tie})"
    assert np.array_equal(gpu["sstar"][b][:upto], ora["sstar"][:upto]), what
    np.testing.assert_allclose(gpu["enf"][b][:upto], ora["enf"][:upto], rtol=ENF_RTOL, atol=1e-13,
                               err_msg=what)
    np.testing.assert_allclose(gpu["trace"][b][:upto], ora["logz_trace"][:upto], rtol=LOGZ_RTOL,
                               atol=1e-12, err_msg=what)
    if t_tie == 0:
        lz_g, lz_o = gpu["log_z"][b], ora["log_z"]
        if np.isfinite(lz_o):
            assert abs(lz_g - lz_o) <= LOGZ_RTOL * abs(lz_o) + 1e-12, (what, lz_g, lz_o)
        else:
            assert lz_g == lz_o, (what, lz_g, lz_o)
    return upto


def compare_first_step(gpu, b, ora, *, M, what=""):
    """Step 1 of filter b draw by draw, for a path whose arithmetic differs from the oracle's
    (FP32-mixed): the oracle (run with tie_masks=True and a wide tie band) marks the draws,
    island walks and ENF tests within the band of a threshold.  Every other particle's
    ancestor, every unmarked island's inherited block, and s* (when no ENF test is marked)
    must equal the oracle's.  Returns the number of particles compared."""
    anc_g, anc_o = gpu["anc"][b][0], ora["anc"][0]
    src_o = anc_o // M
    N = anc_o.size
    if not ora["tie_step"][0]:
        assert gpu["sstar"][b][0] == ora["sstar"][0], (what, gpu["sstar"][b][0], ora["sstar"][0])
        isl_ok = ~ora["tie_src"][0]
        src_g = anc_g // M
        bad = np.nonzero((src_g.reshape(-1, M)[:, 0] != src_o.reshape(-1, M)[:, 0]) & isl_ok)[0]
        assert bad.size == 0, f"{what}: inherited block differs at island {bad[0]}"
        # particle (k, i) holds draw i of island src(k): compare where neither is marked
        i = np.arange(N) % M
        ok = np.repeat(isl_ok, M) & ~ora["tie_draw"][0][src_o * M + i]
        bad = np.nonzero((anc_g != anc_o) & ok)[0]
        assert bad.size == 0, f"{what}: {bad.size} ancestors differ, first at particle {bad[0]}"
        return int(ok.sum())
    return 0
