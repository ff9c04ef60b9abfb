"""Kernel timing of a context created with RECORD_TIMING (CUDA event-record nodes in the
pass's graph): the pass computes the same log Z as without the events, and the summed
island-step and cascade kernel durations are positive and fit inside the pass."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_timing_graph_same_result_and_positive_times():
    import torch
    import paper_2312_06484_gb300 as gp
    y = torch.tensor(synth.sv_observations(80, seed=2), device="cuda")
    th = torch.tensor(synth.SV_THETA[None, :], device="cuda")
    kw = dict(m=256, M=128, T=80, B=1, mode="adaptive", tau=0.3, precision="fp32", seed=4, launch="steps")
    plain = gp.AIRPF(synth.MODEL_SV, **kw)
    timed = gp.AIRPF(synth.MODEL_SV, record=gp.RECORD_TIMING, **kw)
    a = plain.run(th, y, iter=5)["log_z"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b = timed.run(th, y, iter=5)["log_z"]
    e1.record()
    isl, cas = timed.kernel_times()
    torch.cuda.synchronize()
    assert a.item() == b.item()
    assert isl > 0 and cas >= 0
    assert isl + cas <= e0.elapsed_time(e1) * 1.01
    with pytest.raises(gp.AirpfError):
        plain.kernel_times()
    with pytest.raises(gp.AirpfError):
        gp.AIRPF(synth.MODEL_SV, record=gp.RECORD_TIMING, **dict(kw, launch="cta", m=4))
    plain.close()
    timed.close()
