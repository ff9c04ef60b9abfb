"""The sharded pass on one GPU: the islands of one filter split over 2 or 4 contexts (the
ranks), each running the island launches of its own CTA range through the stepwise C ABI,
with the records and rows exchanged by copies between the contexts' workspaces.  log Z
equals the single-context airpf_run's bit for bit (FP64 and FP32-mixed, split and fused
steps, rows moved only when needed or every step) and the oracle's within the FP64
tolerance."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2312_06484_gb300 import sharded
from parity_util import LOGZ_RTOL

pytestmark = pytest.mark.gpu

CASES = [  # model, theta, observations, m, M, launch, mode
    (synth.MODEL_NGM, synth.NGM_THETA, synth.ngm_observations(24, seed=5), 2048, 32, "split", "adaptive"),
    (synth.MODEL_NGM, synth.NGM_THETA, synth.ngm_observations(16, seed=5), 1024, 64, "split", "always"),
    (synth.MODEL_SV, synth.SV_THETA, synth.sv_observations(20, seed=2), 256, 64, "steps", "adaptive"),
    # M = 256: the lean kernels with the island size fixed at compile time
    (synth.MODEL_NGM, synth.NGM_THETA, synth.ngm_observations(12, seed=5), 2048, 256, "split", "adaptive"),
    (synth.MODEL_SV, synth.SV_THETA, synth.sv_observations(12, seed=2), 512, 256, "steps", "always"),
]


def _ctx(model, m, M, T, launch, mode, precision):
    import paper_2312_06484_gb300 as gp
    return gp.AIRPF(model, m=m, M=M, T=T, B=1, mode=mode, tau=0.5, precision=precision, seed=11, launch=launch)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sharded_equals_one_context(case, precision):
    model, theta, y, m, M, launch, mode = CASES[case]
    T = len(y)
    th = torch.tensor(np.asarray(theta, np.float64)[None, :], device="cuda")
    yy = torch.tensor(y, device="cuda")
    one = _ctx(model, m, M, T, launch, mode, precision)
    ref = one.run(th, yy, chain0=3, iter=5)["log_z"].cpu().numpy()[0]
    assert one.launch_mode == {"split": 4, "steps": 1}[launch]
    lz1, _ = sharded.run_pass([(one, 0)], th, yy, world=1, exchange=sharded.LocalExchange(), chain0=3, iter=5)
    assert lz1.cpu().numpy()[0] == ref                      # the stepwise pass on one context
    one.close()
    for world in (2, 4):
        shards = [(_ctx(model, m, M, T, launch, mode, precision), r) for r in range(world)]
        for rows in ("needed", "always"):
            lz, moved = sharded.run_pass(shards, th, yy, world=world, exchange=sharded.LocalExchange(),
                                         chain0=3, iter=5, rows=rows)
            torch.cuda.synchronize()
            assert lz.cpu().numpy()[0] == ref, (world, rows, lz, ref)
            if launch == "steps" or rows == "always" or mode == "always":
                assert moved == T - 1
        for f, _ in shards:
            f.close()
    if precision == "fp64":
        o = oracle.airpf(model, theta, y, m=m, M=M, mode={"adaptive": 2, "always": 1}[mode], tau=0.5, seed=11,
                         chain=3, iter=5)
        if o["tie"][0] == 0:
            assert abs(ref - o["log_z"]) <= LOGZ_RTOL * abs(o["log_z"]) + 1e-12, (ref, o["log_z"])


def test_rows_stay_local_on_quiet_steps():
    """Adaptive NGM on 2 ranks: on most steps no interaction crosses the ranks, and the rows
    move only on the others."""
    model, theta, y, m, M, launch, mode = CASES[0]
    T = len(y)
    th = torch.tensor(np.asarray(theta, np.float64)[None, :], device="cuda")
    yy = torch.tensor(y, device="cuda")
    shards = [(_ctx(model, m, M, T, launch, mode, "fp32"), r) for r in range(2)]
    _, moved = sharded.run_pass(shards, th, yy, world=2, exchange=sharded.LocalExchange())
    assert moved < (T - 1) // 2
    for f, _ in shards:
        f.close()


def test_unsupported_configurations_are_refused():
    import paper_2312_06484_gb300 as gp
    y = torch.tensor(synth.sv_observations(4, seed=2), device="cuda")
    th = torch.tensor(np.asarray(synth.SV_THETA, np.float64)[None, :], device="cuda")
    for kw in (dict(B=2), dict(record=gp.RECORD_ENF), dict(launch="grid")):
        args = dict(m=64, M=32, T=4, mode="adaptive", precision="fp64", seed=1, launch="steps")
        args.update(kw)
        f = gp.AIRPF(synth.MODEL_SV, **args)
        with pytest.raises(gp.AirpfError, match="UNSUPPORTED"):
            f.step_begin(th if args.get("B", 1) == 1 else th.repeat(2, 1), y)
        f.close()
    f = gp.AIRPF(synth.MODEL_SV, m=256, M=32, T=4, precision="fp64", launch="steps")
    f.step_begin(th, y)
    with pytest.raises(gp.AirpfError, match="ARG"):
        f.step_islands(1, 1, 2)                     # a range not aligned to its size
    with pytest.raises(gp.AirpfError, match="UNSUPPORTED"):
        f.step_levels()                             # fused steps: no separate cascade
    f.close()
