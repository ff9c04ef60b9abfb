"""The N > 1 path on CPU: two gloo ranks as separate processes.  Ranks own disjoint chain
ranges, the job time is the slowest rank's, and the replicas' oracle runs (one chain each)
are independent estimates of the same likelihood."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_2312_06484_gb300 import replicas
    import oracle
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, _ = replicas.world()
    c0 = replicas.chain_base(r, chains_per_rank=3)
    fake_seconds = 1.0 + r                       # rank 1 is the slow one
    slowest = replicas.max_over_ranks(fake_seconds)
    rate = replicas.job_rate(100.0, slowest, ws)
    y = synth.ar1_observations(30, seed=1)
    lz = [oracle.airpf(synth.MODEL_AR1, synth.AR1_THETA, y, m=4, M=16, seed=3, chain=c0 + j)["log_z"]
          for j in range(3)]
    dist.barrier()
    np.save(os.path.join(out_dir, f"rank{r}.npy"), np.array([ws, c0, slowest, rate] + lz))
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    pytest.importorskip("torch.distributed")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert r0[0] == r1[0] == 2
    assert (r0[1], r1[1]) == (0, 3)                       # disjoint chain ranges
    assert r0[2] == r1[2] == 2.0                          # slowest rank's time on every rank
    assert r0[3] == r1[3] == 100.0                        # 2 x 100 units / 2 s
    lz = np.concatenate([r0[4:], r1[4:]])
    assert np.all(np.isfinite(lz)) and len(set(lz.tolist())) == 6   # six distinct chains
