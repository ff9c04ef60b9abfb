"""One filter's islands split over several processes, one GPU each.

Algorithm 1 couples the m islands of a filter only through the interaction stages: the
weighting, internal resampling and mutation of an island touch its own particles, and
stage s pairs islands 2^(s-1) apart (butterfly matrices, eq. (3)).  With G = 2^g processes,
process j owns the contiguous islands [j m/G, (j+1) m/G) -- a contiguous range of the
filter's CTAs -- and a pass runs step by step through the stepwise C ABI:

  * airpf_step_islands(t, own CTA range) -- the island work of step t;
  * an all-gather of the step's CTA records (exponent, block-sum subtree and sums of
    squares of each CTA: a few doubles a CTA), after which every process holds all of them;
  * airpf_step_cascade(t) -- every process runs the same cascade over the same records and
    so reaches the same s*, island choices and log Z;
  * an all-gather of the step's particle rows, needed only when an island's chosen source
    block lies on another process: the stages s <= log2(m/G) stay inside a process, so with
    split steps the rows move only on steps whose interacting stages reach the top g
    (airpf_step_levels after the cascade).  Fused steps (small filters) run a step's cascade
    inside the next island launch and exchange the rows every step.

Every process holds the whole filter's buffers; the exchange writes the other processes'
parts of them.  ``run_pass`` drives the shards one process holds: one shard per process
with ``DistExchange`` (torch.distributed all-gathers), or every shard of the filter in one
process with ``LocalExchange`` (copies between the shards' workspaces; used to check the
sharded pass on one GPU).
"""
from __future__ import annotations

N_RECORD_REGIONS = 3          # CTA exponents, block-sum subtrees, sums of squares


def cta_range(ctas: int, rank: int, world: int):
    """(first CTA, CTA count) of a rank: world equal, contiguous, aligned ranges."""
    if world < 1 or world & (world - 1) or ctas % world or not 0 <= rank < world:
        raise ValueError(f"world = {world} must be a power of 2 dividing the {ctas} CTAs, 0 <= rank < world")
    n = ctas // world
    return rank * n, n


def local_levels(m: int, world: int) -> int:
    """Binary interaction levels that stay inside one rank's m/world islands."""
    if m % world:
        raise ValueError("world must divide m")
    return (m // world).bit_length() - 1


def part(region, rank: int, world: int):
    """Rank's part of a region (every region is laid out by CTA, in order)."""
    n = region.numel() // world
    return region[rank * n:(rank + 1) * n]


class LocalExchange:
    """All shards of the filter in this process: rank j's part of every region is copied
    into the other shards' regions (on the current stream)."""

    def __call__(self, regions_by_shard, ranks, world):
        assert sorted(ranks) == list(range(world)), "a local exchange needs every rank's shard"
        for r in range(len(regions_by_shard[0])):
            for i, j in enumerate(ranks):
                src = part(regions_by_shard[i][r], j, world)
                for i2 in range(len(ranks)):
                    if i2 != i:
                        part(regions_by_shard[i2][r], j, world).copy_(src)


class DistExchange:
    """One shard per process: an all-gather of each region over the default process group
    (in place: the rank's part is the input)."""

    def __init__(self, group=None):
        self.group = group

    def __call__(self, regions_by_shard, ranks, world):
        import torch.distributed as dist
        assert len(ranks) == 1
        rank = ranks[0]
        for reg in regions_by_shard[0]:
            dist.all_gather_into_tensor(reg, part(reg, rank, world).clone(), group=self.group)


def run_pass(shards, theta, y, *, world: int, exchange, chain0: int = 0, iter: int = 0,
             rows: str = "needed"):
    """One stepwise pass of one filter split over ``world`` ranks.

    shards: list of (AIRPF context, rank) held by this process; every context has the same
    configuration (B = 1, record = 0, per-step launches) and runs on the current stream.
    exchange: LocalExchange or DistExchange.  rows: "needed" moves the particle rows only
    when the step's interactions cross ranks (split steps), "always" every step.
    Returns (log Z [1] CUDA tensor of the first shard, steps whose rows were exchanged)."""
    f0 = shards[0][0]
    ranges = [cta_range(f0.ctas, rank, world) for _, rank in shards]
    ranks = [rank for _, rank in shards]
    fused = f0.launch_mode == 1
    local = local_levels(f0.m, world)
    for f, _ in shards:
        f.step_begin(theta, y, chain0=chain0, iter=iter)
    moved = 0
    T = f0.T
    for t in range(1, T + 1):
        for (f, _), (c0, n) in zip(shards, ranges):
            f.step_islands(t, c0, n)
        regs = [f.step_regions(t) for f, _ in shards]
        exchange([r[:N_RECORD_REGIONS] for r in regs], ranks, world)
        if fused or rows == "always":
            if t < T:
                exchange([r[N_RECORD_REGIONS:] for r in regs], ranks, world)
                moved += 1
            for f, _ in shards:
                f.step_cascade(t)
        else:
            for f, _ in shards:
                f.step_cascade(t)
            if t < T and f0.step_levels() > local:
                exchange([r[N_RECORD_REGIONS:] for r in regs], ranks, world)
                moved += 1
    return f0.step_end(), moved
