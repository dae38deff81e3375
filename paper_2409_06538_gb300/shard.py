"""Multi-GPU layout of TNMC: disorder realizations are independent units, so ranks take
disjoint slices of the seed list and share nothing while they run (no data-path
collective).  The only exchange is one gather of the per-realization thermal means at the
end, to form the disorder averages [.] of Sec. III.C over all ranks."""
import numpy as np

from .tnmc import disorder_average


def shard_seeds(seeds, rank, world):
    """Contiguous, balanced slice of `seeds` for `rank` of `world` (sizes differ by <= 1)."""
    seeds = np.asarray(seeds)
    n = len(seeds)
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return seeds[start:start + base + (1 if rank < extra else 0)]


def gather_disorder_average(per_realization, L, beta, group=None):
    """All-gather the per-realization observable dicts of every rank (torch.distributed,
    any backend) and return the disorder average over all realizations on every rank
    (tnmc_disorder_average, for lattice side L at inverse temperature beta)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, list(per_realization), group=group)
    merged = [o for part in parts for o in part]
    return disorder_average(merged, L, beta), len(merged)
