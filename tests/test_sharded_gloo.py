"""The sharded pass (one filter's islands split over ranks) on CPU.

* The driver and its exchanges with a stand-in filter of the same region layout, whose every
  value carries the step that wrote it: an island that reads a parent row or a cascade that
  reads a record not written at the step before fails.  Two gloo ranks as separate
  processes, and 2 or 4 shards in one process, reach the single-shard result exactly.
* The locality the driver relies on, pinned on the oracle: with s* - 1 binary stages
  interacting (stage s pairs islands 2^(s-1) apart, eq. (3)), island k's source block lies in
  k's aligned block of 2^(s*-1) islands, so a rank of m/G contiguous islands needs another
  rank's rows only when s* - 1 > log2(m/G)."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2312_06484_gb300 import sharded

import oracle
import synth


class StandIn:
    """A CPU stand-in for a stepwise AIRPF context: m islands of M particles, G islands a CTA,
    dx rows; record regions [P], [P 2G], [P 8] and rows [N] per dimension, double-buffered by
    step parity, each laid out by CTA.  A value written at step t is 1000 t + (a fraction)."""

    def __init__(self, m, G, M, T, dx, fused):
        self.m, self.G, self.M, self.T, self.dx = m, G, M, T, dx
        self.ctas, self.N, self.S = m // G, m * M, int(math.log2(m))
        self.launch_mode = 1 if fused else 4
        P = self.ctas
        self.rec = [[torch.full((n,), -1.0, dtype=torch.float64) for n in (P, 2 * G * P, 8 * P)] for _ in range(2)]
        self.X = [[torch.full((self.N,), -1.0, dtype=torch.float64) for _ in range(dx)] for _ in range(2)]

    def step_begin(self, theta, y, chain0=0, iter=0):
        self.src = torch.arange(self.m)
        self.logz = 0.0
        self.history = []
        self.y = torch.as_tensor(y, dtype=torch.float64)

    def step_regions(self, t):
        return self.rec[t & 1] + self.X[t & 1]

    def step_islands(self, t, c0, n):
        M, G = self.M, self.G
        par = t & 1
        i = torch.arange(M, dtype=torch.float64)
        for j in range(c0, c0 + n):
            means = []
            for k in range(j * G, (j + 1) * G):
                fr = []
                for d in range(self.dx):
                    if t == 1:
                        f = ((k * M + i) * 0.6180339887 + 0.1 * d) % 1.0
                    else:
                        pv = self.X[par ^ 1][d][int(self.src[k]) * M:(int(self.src[k]) + 1) * M]
                        assert torch.all(torch.floor(pv / 1000) == t - 1), f"stale parent row at step {t}"
                        f = (pv - 1000 * (t - 1)) * 0.7 + 0.1 * (k + 1) / self.m + 0.05 * d + 0.013 * i / M \
                            + 0.01 * float(self.y[t - 1])
                        f = f % 1.0
                    self.X[par][d][k * M:(k + 1) * M] = 1000 * t + f
                    fr.append(f)
                means.append(float(torch.stack(fr).mean()))
            self.rec[par][0][j] = 1000 * t + (sum(means) / G) % 1.0
            self.rec[par][1][j * 2 * G:j * 2 * G + G] = 1000 * t + torch.tensor(means)
            self.rec[par][1][j * 2 * G + G:(j + 1) * 2 * G] = 1000 * t
            self.rec[par][2][j * 8:(j + 1) * 8] = 1000 * t + torch.tensor(means[:1] * 8) * 0.5

    def step_cascade(self, t):
        par = t & 1
        for r in self.rec[par]:
            assert torch.all(torch.floor(r / 1000) == t), f"stale record at step {t}"
        tot = float((self.rec[par][0] - 1000 * t).sum() + (self.rec[par][2] - 1000 * t).sum())
        self.levels = int(tot * 997) % (self.S + 1)
        self.history.append(self.levels)
        k = torch.arange(self.m)
        low = (1 << self.levels) - 1
        self.src = (k & ~low) | ((k * 5 + t) & low)
        self.logz += math.log1p(tot)

    def step_levels(self):
        assert self.launch_mode == 4
        return self.levels

    def step_end(self):
        return torch.tensor([self.logz], dtype=torch.float64)


CFG = dict(m=64, G=4, M=8, T=14, dx=2)


def _run(world, fused, rows="needed", exchange=None):
    shards = [(StandIn(fused=fused, **CFG), r) for r in range(world)]
    y = np.linspace(-1.0, 1.0, CFG["T"])
    lz, moved = sharded.run_pass(shards, None, y, world=world, exchange=exchange or sharded.LocalExchange(),
                                 rows=rows)
    return float(lz[0]), moved, shards


def test_ranges_and_levels():
    assert sharded.cta_range(16, 3, 4) == (12, 4)
    assert sharded.local_levels(1024, 4) == 8
    for bad in [(16, 0, 3), (16, 2, 2 ** 5), (6, 0, 4)]:
        with pytest.raises(ValueError):
            sharded.cta_range(*bad)
    reg = torch.arange(12)
    assert sharded.part(reg, 2, 4).tolist() == [6, 7, 8]


@pytest.mark.parametrize("fused", [False, True])
def test_local_shards_match_one_shard(fused):
    ref, moved1, one = _run(1, fused)
    levels = one[0][0].history[:-1]                 # the steps before the last
    for world in (2, 4):
        lz, moved, shards = _run(world, fused)
        need = sum(lv > sharded.local_levels(CFG["m"], world) for lv in levels)
        assert lz == ref and moved == (CFG["T"] - 1 if fused else need)
        if not fused:                   # rows move only on steps that interact across ranks
            assert 0 < need < CFG["T"] - 1
        for f, r in shards:             # each shard's own part of the last step's rows
            for d in range(CFG["dx"]):
                assert torch.equal(sharded.part(f.X[CFG["T"] & 1][d], r, world),
                                   sharded.part(one[0][0].X[CFG["T"] & 1][d], r, world))
    lz, moved, _ = _run(2, fused, rows="always")
    assert lz == ref and moved == CFG["T"] - 1


def test_a_missing_row_exchange_is_caught():
    """Row exchanges dropped: the first step that reads another rank's parent row fails."""
    class RecordsOnly(sharded.LocalExchange):
        def __call__(self, regions_by_shard, ranks, world):
            if len(regions_by_shard[0]) == sharded.N_RECORD_REGIONS:
                super().__call__(regions_by_shard, ranks, world)

    with pytest.raises(AssertionError, match="stale parent row"):
        _run(2, False, exchange=RecordsOnly())


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, fused):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    f = StandIn(fused=fused, **CFG)
    y = np.linspace(-1.0, 1.0, CFG["T"])
    lz, moved = sharded.run_pass([(f, rank)], None, y, world=world, exchange=sharded.DistExchange())
    rows = torch.cat([sharded.part(x, rank, world) for x in f.X[CFG["T"] & 1]]).numpy()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([[float(lz[0]), moved], rows]))
    dist.destroy_process_group()


@pytest.mark.parametrize("fused", [False, True])
def test_two_gloo_ranks_match_one_shard(tmp_path, fused):
    pytest.importorskip("torch.distributed")
    ref, moved1, one = _run(1, fused)
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path), fused), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        want = torch.cat([sharded.part(x, r, 2) for x in one[0][0].X[CFG["T"] & 1]]).numpy()
        got = np.load(tmp_path / f"rank{r}.npy")
        need = sum(lv > sharded.local_levels(CFG["m"], 2) for lv in one[0][0].history[:-1])
        assert got[0] == ref and got[1] == (CFG["T"] - 1 if fused else need)
        np.testing.assert_array_equal(got[2:], want)


@pytest.mark.parametrize("mode,tau", [(oracle.MODE_ADAPTIVE, 0.5), (oracle.MODE_ALWAYS, 0.3)])
def test_oracle_sources_stay_in_the_interacting_block(mode, tau):
    """Oracle: island k's source block lies in k's aligned block of 2^(s*-1) islands, and a
    rank of m/G islands needs no other rank's rows when s* - 1 <= log2(m/G)."""
    m, M, T = 64, 16, 40
    y = synth.ngm_observations(T, seed=5)
    o = oracle.airpf(synth.MODEL_NGM, synth.NGM_THETA, y, m=m, M=M, mode=mode, tau=tau, seed=4, chain=1)
    k = np.arange(m)
    seen = set()
    for t in range(T):
        lv = int(o["sstar"][t]) - 1
        src = o["src"][t]
        assert np.all(src >> lv == k >> lv), t
        seen.add(lv)
        for world in (2, 4, 8):
            if lv <= sharded.local_levels(m, world):
                assert np.all(src // (m // world) == k // (m // world)), (t, world)
    assert mode == oracle.MODE_ALWAYS and seen == {int(math.log2(m))} or len(seen) > 1
