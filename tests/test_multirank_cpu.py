"""The multi-rank path on CPU (gloo, world size 2): realizations are sharded with no
data-path exchange, and the one gather at the end -- through the library's host-side
tnmc_disorder_average -- reproduces the single-process disorder averages exactly, on
per-realization thermal means that the oracle's own TNMC run produced."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


_OBS_CACHE = {}


def _realization_obs(seed):
    """Thermal means of one seeded realization (L = 4, chi = 2, p = 0.109) from the oracle."""
    if seed not in _OBS_CACHE:
        from tests.test_disorder_host import oracle_realizations
        _OBS_CACHE[seed] = oracle_realizations(4, 0.109, 2, [int(seed)], 12, 2)[0]
    return _OBS_CACHE[seed]


def _worker(rank, world, port, seeds, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_2409_06538_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.shard_seeds(seeds, rank, world)
    avg, n = shard.gather_disorder_average([_realization_obs(s) for s in mine], 4, 0.9)
    if rank == 0:
        np.save(out_path, np.array([avg["E"][0], avg["E"][1], avg["m2"][0], avg["U_m"], avg["Q_q"],
                                    avg["acceptance"], n, avg["chi_q"], avg["chi_edge"]], dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_are_disjoint_and_cover():
    from paper_2409_06538_gb300 import shard
    seeds = np.arange(13)
    for world in (1, 2, 3, 5):
        parts = [shard.shard_seeds(seeds, r, world) for r in range(world)]
        assert np.array_equal(np.concatenate(parts), seeds)
        assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


def test_gloo_two_ranks_reproduce_single_process(tmp_path):
    import torch.multiprocessing as mp
    from paper_2409_06538_gb300 import build, disorder_average
    build()
    seeds = np.arange(100, 113)
    out = str(tmp_path / "avg.npy")
    mp.spawn(_worker, args=(2, _free_port(), seeds, out), nprocs=2, join=True)
    got = np.load(out)
    ref = disorder_average([_realization_obs(s) for s in seeds], 4, 0.9)
    want = np.array([ref["E"][0], ref["E"][1], ref["m2"][0], ref["U_m"], ref["Q_q"], ref["acceptance"], len(seeds),
                     ref["chi_q"], ref["chi_edge"]])
    assert np.allclose(got, want, rtol=0, atol=1e-12)
