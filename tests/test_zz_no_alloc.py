"""airpf_run_static (a pass with no context and no device allocation, on the library's
static scratch) against the context entry point airpf_create + airpf_run.

Both run the same kernels with the same random streams, so log Z agrees to the FP64
parity tolerance (in practice bit for bit).  Two calls in a row check that a pass leaves
nothing in the scratch that the next one depends on.  Collected last, and independent of
every other test file, so it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _context_logz(model, theta, y, *, B, chain0, iter, model_data=None, **kw):
    import torch
    import paper_2312_06484_gb300 as gp
    f = gp.AIRPF(model, T=len(y) // kw.get("dy", 1), B=B, model_data=model_data, **kw)
    out = f.run(torch.tensor(theta, device="cuda"), torch.tensor(y, device="cuda"), chain0=chain0, iter=iter)
    f.sync()
    lz = out["log_z"].cpu().numpy()
    f.close()
    return lz


def _static_logz(model, theta, y, *, B, chain0, iter, model_data=None, **kw):
    import torch
    import paper_2312_06484_gb300 as gp
    lz = torch.full((B,), np.nan, dtype=torch.float64, device="cuda")
    md = torch.tensor(np.asarray(model_data, np.float64).ravel(), device="cuda") if model_data is not None else None
    gp.run_static(model, torch.tensor(theta, device="cuda"), torch.tensor(y, device="cuda"), lz, B=B,
                  chain0=chain0, iter=iter, model_data=md, **kw)
    torch.cuda.synchronize()
    return lz.cpu().numpy()


CASES = [
    # (name, model, theta of one filter, y, B, kwargs)
    ("ar1 m16 M64 fp64 (one CTA per filter)", synth.MODEL_AR1, synth.AR1_THETA, synth.ar1_observations(100, seed=1),
     2, dict(m=16, M=64, mode="adaptive", tau=0.3, precision="fp64", seed=5)),
    ("sv m1024 M256 fp32 (per-step launches)", synth.MODEL_SV, synth.SV_THETA, synth.sv_observations(60, seed=2),
     1, dict(m=1024, M=256, mode="adaptive", tau=0.3, precision="fp32", seed=9)),
    ("ngm m64 M37 fp64 always (ragged M)", synth.MODEL_NGM, synth.NGM_THETA, synth.ngm_observations(30, seed=5),
     3, dict(m=64, M=37, mode="always", tau=0.3, precision="fp64", seed=2, launch="steps")),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_static_matches_context_two_calls_in_a_row(case):
    _, model, th1, y, B, kw = case
    theta = np.tile(np.asarray(th1, np.float64), (B, 1))
    y = np.asarray(y, np.float64)
    for chain0, it in ((0, 3), (7, 4)):
        ref = _context_logz(model, theta, y, B=B, chain0=chain0, iter=it, **kw)
        got = _static_logz(model, theta, y, B=B, chain0=chain0, iter=it, **kw)
        assert np.all(np.isfinite(ref))
        np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0, err_msg=f"chain0={chain0} iter={it}")


def test_static_lgssm_model_data_on_device():
    A, C, md = synth.lg_model(dx=2, dy=2, seed=4)
    theta = synth.lg_theta(A, q=0.1, r=0.5)
    y = synth.lg_observations(A, C, 0.1, 0.5, 40, seed=4)
    kw = dict(m=8, M=64, dx=2, dy=2, mode="adaptive", tau=0.3, precision="fp64", seed=1)
    theta = np.asarray(theta, np.float64)[None, :]
    ref = _context_logz(synth.MODEL_LGSSM, theta, y, B=1, chain0=0, iter=1, model_data=md, **kw)
    got = _static_logz(synth.MODEL_LGSSM, theta, y, B=1, chain0=0, iter=1, model_data=md, **kw)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


def test_static_rejects_configurations_beyond_the_scratch():
    import torch
    import paper_2312_06484_gb300 as gp
    from paper_2312_06484_gb300 import _binding
    lib = _binding.load()
    # 4 filters of 4096 x 1024 FP64 particles need 256 MiB of particle stores alone
    cfg = _binding.AirpfConfig(model=synth.MODEL_SV, dx=1, dy=1, m=4096, M=1024, T=10, B=4, mode=2, tau=0.3,
                               precision=0, record=0, seed=0, launch=0, reserved=0)
    th = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    y = torch.zeros(10, dtype=torch.float64, device="cuda")
    lz = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.airpf_run_static(ctypes.byref(cfg), th.data_ptr(), y.data_ptr(), None, 0, 0, lz.data_ptr(), None)
    assert st == 3                                   # AIRPF_ERR_WORKSPACE
    msg = lib.airpf_last_error(None).decode()
    assert "static scratch" in msg and str(32 << 20) in msg
    # recording outputs needs a context
    cfg.m, cfg.M, cfg.B, cfg.record = 16, 64, 1, 1
    assert lib.airpf_run_static(ctypes.byref(cfg), th.data_ptr(), y.data_ptr(), None, 0, 0, lz.data_ptr(),
                                None) == 1          # AIRPF_ERR_ARG
    with pytest.raises(gp.AirpfError):
        gp.run_static(synth.MODEL_SV, th[:1], y, lz[:1], m=16, M=64, launch="grid")
