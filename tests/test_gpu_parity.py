"""FP64 CUDA path vs the oracle, element by element (ancestors bit-exact, log Z within
1e-10 relative, ENF and s* per step), through the C ABI, on seeded inputs:
the AR(1) workload of m=16 x M=64 x T=100 in every interaction mode and batched, ragged
and tiny sizes, every model, m = 1, the degenerate all-zero-weight case, and sampled
filters at the full SV size m=1024 x M=256."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import compare_filter, compare_first_step, run_gpu

pytestmark = pytest.mark.gpu

MODES = {"never": oracle.MODE_NEVER, "always": oracle.MODE_ALWAYS, "adaptive": oracle.MODE_ADAPTIVE}


@pytest.mark.parametrize("launch", ["steps", "cta"])
@pytest.mark.parametrize("mode", ["adaptive", "always", "never"])
def test_ar1_workload_all_modes(gpu_lib, mode, launch):
    y = synth.ar1_observations(100, seed=1)
    B, m, M = 4, 16, 64
    g = run_gpu(synth.MODEL_AR1, synth.AR1_THETA, y, m=m, M=M, B=B, mode=mode, tau=0.3, seed=7,
                chain0=3, iter=2, launch=launch)
    for b in range(B):
        o = oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, m=m, M=M, mode=MODES[mode], tau=0.3,
                         seed=7, chain=3 + b, iter=2)
        compare_filter(g, b, o, m=m, what=f"{mode} {launch} b={b}")
    if launch == "steps":
        # run parameters, prologue, T island steps, the lineage step, and T cascade kernels
        # unless every CTA runs the cascade itself (fused steps)
        assert g["launches"] in (2 * 100 + 3, 100 + 3)
    else:
        assert g["launches"] == 3 and g["launch_mode"] == 2


@pytest.mark.parametrize("model,theta,ymaker,m,M,T,mode,tau", [
    (synth.MODEL_SV, synth.SV_THETA, lambda T: synth.sv_observations(T, 2), 64, 37, 40, "adaptive", 0.8),
    (synth.MODEL_SV, synth.SV_THETA, lambda T: synth.sv_observations(T, 2), 8, 200, 30, "always", 0.3),
    (synth.MODEL_NGM, synth.NGM_THETA, lambda T: synth.ngm_observations(T, 5), 32, 100, 30, "adaptive", 0.5),
    (synth.MODEL_TOY, synth.TOY_THETA, lambda T: synth.toy_observations(T, 3), 4, 2, 25, "always", 0.3),
    (synth.MODEL_AR1, synth.AR1_THETA, lambda T: synth.ar1_observations(T, 1), 1, 129, 20, "adaptive", 0.3),
    (synth.MODEL_AR1, synth.AR1_THETA, lambda T: synth.ar1_observations(T, 1), 2, 1, 20, "always", 0.3),
    (synth.MODEL_SV, synth.SV_THETA, lambda T: synth.sv_observations(T, 2), 4096, 4, 4, "always", 0.3),
    (synth.MODEL_SV, synth.SV_THETA, lambda T: synth.sv_observations(T, 2), 2, 1024, 6, "adaptive", 0.99),
])
def test_models_and_shapes(gpu_lib, model, theta, ymaker, m, M, T, mode, tau):
    y = ymaker(T)
    g = run_gpu(model, theta, y, m=m, M=M, B=2, mode=mode, tau=tau, seed=11, chain0=0, iter=5)
    for b in range(2):
        o = oracle.airpf(model, theta, y, m=m, M=M, mode=MODES[mode], tau=tau, seed=11, chain=b, iter=5)
        compare_filter(g, b, o, m=m, what=f"model {model} m={m} M={M} b={b}")


def test_lgssm(gpu_lib):
    dx, dy = 3, 2
    A, C, md = synth.lg_model(dx, dy, seed=11)
    th = synth.lg_theta(A, q=0.1, r=0.5)
    y = synth.lg_observations(A, C, 0.1, 0.5, 25, seed=11)
    g = run_gpu(synth.MODEL_LGSSM, th, y, m=16, M=32, B=2, dx=dx, dy=dy, model_data=md, mode="adaptive",
                tau=0.6, seed=2)
    for b in range(2):
        o = oracle.airpf(synth.MODEL_LGSSM, th, y, m=16, M=32, dx=dx, dy=dy, model_data=md,
                         mode=oracle.MODE_ADAPTIVE, tau=0.6, seed=2, chain=b)
        compare_filter(g, b, o, m=16, what=f"lgssm b={b}")


def test_m1_equals_oracle_bootstrap_filter(gpu_lib):
    y = synth.sv_observations(50, seed=2)
    g = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, m=1, M=256, B=1, mode="adaptive", seed=4)
    lz, anc, tie = oracle.bpf(synth.MODEL_SV, synth.SV_THETA, y, M=256, seed=4)
    upto = len(y) if tie[0] == 0 else tie[0] - 1
    assert np.array_equal(g["anc"][0][:upto], anc[:upto])
    if tie[0] == 0:
        assert abs(g["log_z"][0] - lz) <= 1e-10 * abs(lz)


def test_dead_filter_is_minus_infinity(gpu_lib):
    y = np.full(6, 1e200)
    g = run_gpu(synth.MODEL_AR1, synth.AR1_THETA, y, m=4, M=8, B=1, mode="adaptive", seed=1)
    o = oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, m=4, M=8, mode=oracle.MODE_ADAPTIVE, seed=1)
    assert g["log_z"][0] == -np.inf and o["log_z"] == -np.inf
    assert np.array_equal(g["anc"][0], o["anc"])


@pytest.mark.parametrize("launch", ["steps", "grid"])
def test_full_size_sv_sampled_filters(gpu_lib, launch):
    """m=1024 x M=256 (the SV workload's size) with T shortened to 6, FP64, every record
    compared: two filters of a batch of 3 in the per-step launch, the single filter of the
    bench configuration in the grid-persistent launch."""
    y = synth.sv_observations(1000, seed=2)[:6]
    B = 3 if launch == "steps" else 1
    g = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, m=1024, M=256, B=B, mode="adaptive", tau=0.3, seed=9,
                launch=launch)
    for b in ((0, 2) if B == 3 else (0,)):
        o = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, m=1024, M=256, mode=oracle.MODE_ADAPTIVE,
                         tau=0.3, seed=9, chain=b)
        compare_filter(g, b, o, m=1024, what=f"full-size {launch} b={b}")


@pytest.mark.parametrize("launch", ["steps", "grid"])
def test_adaptive_ngm_long_run(gpu_lib, launch):
    """Adaptive interaction with frequent partial cascades (nonlinear growth model, tau=0.9),
    m=256 x M=64 x T=60."""
    y = synth.ngm_observations(60, seed=5)
    g = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, m=256, M=64, B=2, mode="adaptive", tau=0.9,
                seed=12, launch=launch)
    for b in range(2):
        o = oracle.airpf(synth.MODEL_NGM, synth.NGM_THETA, y, m=256, M=64, mode=oracle.MODE_ADAPTIVE,
                         tau=0.9, seed=12, chain=b)
        compare_filter(g, b, o, m=256, what=f"ngm {launch} b={b}")


def test_grid_barrier_timeout_is_reported_and_context_survives(gpu_lib):
    """A grid-persistent pass whose barrier never completes (one CTA leaves early) ends after
    the bounded wait with AIRPF_ERR_TIMEOUT; the next pass on the same context is correct."""
    import torch
    import paper_2312_06484_gb300 as gp
    y = synth.sv_observations(8, seed=2)
    f = gp.AIRPF(synth.MODEL_SV, m=1024, M=256, T=len(y), B=1, mode="adaptive", tau=0.3, seed=9,
                 launch="grid")
    th = torch.tensor(synth.SV_THETA[None, :], device="cuda")
    yy = torch.tensor(y, device="cuda")
    f.inject(1)
    f.run(th, yy)
    with pytest.raises(gp.AirpfError, match="TIMEOUT"):
        f.sync()
    out = f.run(th, yy)
    f.sync()
    o = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, m=1024, M=256, mode=oracle.MODE_ADAPTIVE, tau=0.3,
                     seed=9, record=False)
    if o["tie"][0] == 0:
        assert abs(float(out["log_z"][0]) - o["log_z"]) <= 1e-10 * abs(o["log_z"])
    f.close()


@pytest.mark.parametrize("mode", ["adaptive", "always"])
def test_split_steps_match_oracle(gpu_lib, mode):
    """Split steps (island-step kernel + one-CTA cascade kernel that leaves the block-sum tree
    in global memory; each CTA walks its own islands) against the oracle."""
    y = synth.ngm_observations(40, seed=5)
    m, M = 64, 32
    g = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, m=m, M=M, B=2, mode=mode, tau=0.5, seed=4, chain0=1,
                iter=3, launch="split")
    assert g["launch_mode"] == 4
    for b in range(2):
        o = oracle.airpf(synth.MODEL_NGM, synth.NGM_THETA, y, m=m, M=M, mode=MODES[mode], tau=0.5, seed=4,
                         chain=1 + b, iter=3)
        compare_filter(g, b, o, m=m, what=f"split {mode} b={b}")


def test_ngm_m65536_full_size_fp64():
    """The large nonlinear-growth workload at full size (m = 65536 islands x M = 256,
    N = 16.8M) on a short series, FP64, against the oracle: ancestors, s*, ENF and log Z."""
    y = synth.ngm_observations(3, seed=5)
    m, M = 65536, 256
    g = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, m=m, M=M, B=1, mode="adaptive", tau=0.3, seed=1)
    assert g["launch_mode"] == 4            # AUTO splits the step when a filter spans > 512 CTAs
    o = oracle.airpf(synth.MODEL_NGM, synth.NGM_THETA, y, m=m, M=M, mode=oracle.MODE_ADAPTIVE, tau=0.3, seed=1)
    upto = compare_filter(g, 0, o, m=m, what="NGM m=65536")
    assert upto >= 1
    # the pass that records nothing runs the lean split kernel with M = 256 fixed at
    # compile time (the bench's kernel): the same log Z, bit for bit
    lean = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, m=m, M=M, B=1, mode="adaptive", tau=0.3, seed=1, record=0)
    assert lean["launch_mode"] == 4
    np.testing.assert_array_equal(lean["log_z"], g["log_z"])


@pytest.mark.parametrize("launch,B", [("steps", 1), ("steps", 3), ("split", 1)])
def test_lean_passes_match_oracle(gpu_lib, launch, B):
    """Passes that record nothing run the lean instantiations: fused steps with up to 128
    registers a thread where the grid is one wave at that occupancy (B = 1 at m=1024 x
    M=256), with 64 otherwise (B = 3), and split steps.  FP64 log Z against the oracle, and
    equal, bit for bit, to the recording pass's; FP32 log Z independent of the batch size
    (filter b draws the same numbers whichever instantiation runs it)."""
    y = synth.sv_observations(1000, seed=2)[:6]
    kw = dict(m=1024, M=256, mode="adaptive", tau=0.3, seed=9, launch=launch)
    lean = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, B=B, record=0, **kw)
    rec = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, B=B, record=7, **kw)
    np.testing.assert_array_equal(lean["log_z"], rec["log_z"])
    for b in range(B):
        o = oracle.airpf(synth.MODEL_SV, synth.SV_THETA, y, m=1024, M=256, mode=oracle.MODE_ADAPTIVE, tau=0.3,
                         seed=9, chain=b, record=False)
        if o["tie"][0] == 0:
            assert abs(float(lean["log_z"][b]) - o["log_z"]) <= 1e-10 * abs(o["log_z"]), (b, lean["log_z"][b])
    f32_one = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, B=1, record=0, precision="fp32", **kw)
    f32_many = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, B=3, record=0, precision="fp32", **kw)
    assert f32_one["log_z"][0] == f32_many["log_z"][0]
    # FP32 too: the lean kernels (M = 256 fixed at compile time) give the recording kernel's bits
    f32_rec = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, B=3, record=7, precision="fp32", **kw)
    np.testing.assert_array_equal(f32_many["log_z"], f32_rec["log_z"])


@pytest.mark.parametrize("M,launch,ppt", [(M, l, 0) for M in (128, 512, 1024) for l in ("steps", "split")] +
                         [(M, l, 8) for M in (256, 512, 1024) for l in ("steps", "split")])
def test_fixed_size_fp32_kernels_match_recording_kernel(gpu_lib, M, launch, ppt):
    """FP32 islands of 128, 512 and 1024 particles (and 256 to 1024 at eight particles a
    thread) run lean kernels with the island size fixed at compile time (fused steps with 64
    registers, split steps): the same log Z, bit for bit, as the recording kernel, whose island
    size is read at run time; at eight particles a thread also the log Z of four."""
    y = synth.ngm_observations(8, seed=5)
    m = 64
    ctas = m * max(32, M // 4) // 256          # CTAs a filter (256-thread CTAs)
    B = 2 if launch == "split" else -(-320 // ctas)   # enough CTAs that the fused grid is not one wave
    kw = dict(m=m, M=M, B=B, mode="adaptive", tau=0.5, seed=3, launch=launch, precision="fp32")
    if ppt:
        kw["ppt"] = ppt
    lean = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, record=0, **kw)
    rec = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, record=7, **kw)
    np.testing.assert_array_equal(lean["log_z"], rec["log_z"])
    assert np.all(np.isfinite(lean["log_z"]))
    if ppt:
        kw["ppt"] = 4
        four = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, record=0, **kw)
        np.testing.assert_allclose(lean["log_z"], four["log_z"], rtol=1e-12)


@pytest.mark.parametrize("model", [synth.MODEL_NGM, synth.MODEL_SV])
def test_split_fp32_islands_of_256_take_one_warp(gpu_lib, model):
    """FP32 split steps of the SV and NGM filters with islands of 256 particles run one warp an
    island (eight particles a thread, four islands a CTA: the same CTAs and records as four
    particles a thread).  The lean kernel (M = 256 fixed at compile time) gives the recording
    kernel's bits; the log Z is the one of four particles a thread; the draws of step 1 agree
    with the oracle's draw by draw; FP64 and fused steps keep four particles a thread."""
    import torch
    import paper_2312_06484_gb300 as gp
    theta = synth.NGM_THETA if model == synth.MODEL_NGM else synth.SV_THETA
    y = synth.ngm_observations(8, seed=5) if model == synth.MODEL_NGM else synth.sv_observations(8, 2)
    m, M = 4096, 256                                 # 1024 CTAs a filter: AUTO splits the step
    tilings = {}
    for prec, launch in (("fp32", "auto"), ("fp64", "auto"), ("fp32", "steps")):
        f = gp.AIRPF(model, m=m, M=M, T=len(y), B=1, mode="adaptive", tau=0.5, precision=prec, seed=3,
                     launch=launch)
        tilings[prec, launch] = (f.launch_mode, f.tiling)
        f.close()
    assert tilings["fp32", "auto"] == (4, {"threads_per_island": 32, "particles_per_thread": 8, "islands_per_cta": 4})
    assert tilings["fp64", "auto"][1]["particles_per_thread"] == 4
    assert tilings["fp32", "steps"][1]["particles_per_thread"] == 4
    kw = dict(m=m, M=M, B=2, mode="adaptive", tau=0.5, seed=3, precision="fp32")
    lean = run_gpu(model, theta, y, record=0, **kw)
    rec = run_gpu(model, theta, y, record=7, **kw)
    assert lean["launch_mode"] == 4 and rec["launch_mode"] == 4
    np.testing.assert_array_equal(lean["log_z"], rec["log_z"])
    four = run_gpu(model, theta, y, record=0, ppt=4, **kw)
    np.testing.assert_allclose(lean["log_z"], four["log_z"], rtol=1e-12)
    assert np.all(np.isfinite(lean["log_z"]))
    g1 = run_gpu(model, theta, y[:1], m=m, M=M, B=2, mode="adaptive", tau=0.5, seed=3, precision="fp32")
    for b in range(2):
        o = oracle.airpf(model, theta, y[:1], m=m, M=M, mode=oracle.MODE_ADAPTIVE, tau=0.5, seed=3, chain=b,
                         tie_rel=1e-5, tie_masks=True)
        n = compare_first_step(g1, b, o, M=M, what=f"one warp an island, b={b}")
        assert n >= 0.95 * m * M, (n, m * M)


@pytest.mark.parametrize("tau_int,radix", [(0.5, 2), (0.0, 4), (0.5, 4)])
def test_eight_particles_a_thread_with_internal_resampling_and_radix(gpu_lib, tau_int, radix):
    """Adaptive internal resampling (carried log-weights) and radix-4 interactions on the FP32
    split steps that take eight particles a thread (NGM, islands of 256): the same log Z as
    four particles a thread, and the lean kernel's equal to the recording kernel's."""
    y = synth.ngm_observations(10, seed=5)
    kw = dict(m=4096, M=256, B=2, mode="adaptive", tau=0.5, seed=5, precision="fp32", tau_int=tau_int,
              radix=radix)
    eight = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, record=0, **kw)
    rec = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, record=7, **kw)
    four = run_gpu(synth.MODEL_NGM, synth.NGM_THETA, y, record=0, ppt=4, **kw)
    assert eight["launch_mode"] == 4
    np.testing.assert_array_equal(eight["log_z"], rec["log_z"])
    np.testing.assert_allclose(eight["log_z"], four["log_z"], rtol=1e-12)
    assert np.all(np.isfinite(eight["log_z"]))


@pytest.mark.parametrize("launch", ["cta", "grid", "steps", "split"])
@pytest.mark.parametrize("M", [256, 200])
def test_eight_particles_a_thread_in_every_launch_form(gpu_lib, launch, M):
    """Eight particles a thread (which the batch autotuner may pick for FP32 SV filters) in
    every launch form, with islands of 256 (one warp) and of 200 (a ragged island: the last
    lanes idle, the CDF rows swizzled): the log Z of four particles a thread."""
    y = synth.sv_observations(12, seed=2)
    kw = dict(m=8, M=M, B=3, mode="adaptive", tau=0.8, seed=13, precision="fp32", launch=launch)
    eight = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, record=0, ppt=8, **kw)
    four = run_gpu(synth.MODEL_SV, synth.SV_THETA, y, record=0, ppt=4, **kw)
    np.testing.assert_allclose(eight["log_z"], four["log_z"], rtol=1e-12)
    assert np.all(np.isfinite(eight["log_z"]))
