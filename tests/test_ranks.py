"""Multi-rank bookkeeping of a multi-GPU run, exercised with two gloo ranks on
the CPU: system sharding covers every system once, the whole-job rate is the
sum of units over the slowest rank's time, and the replica seeds differ."""
import os
import socket

import numpy as np
import pytest

from paper_1005_5384_gb300 import ranks


def test_shard_systems_covers_each_system_once():
    rng = np.random.default_rng(1)
    for world in (1, 2, 3, 8):
        sizes = rng.integers(1, 1000, size=37)
        got = [ranks.shard_systems(sizes, r, world) for r in range(world)]
        flat = [i for lo, hi in got for i in range(lo, hi)]
        assert flat == list(range(37))
        loads = [int(sizes[lo:hi].sum()) for lo, hi in got]
        assert max(loads) <= sizes.sum() / world + sizes.max()
    assert ranks.shard_systems([], 0, 2) == (0, 0)
    with pytest.raises(ValueError):
        ranks.shard_systems([1, 2], 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = 1.0 + rank          # rank 1 is the slow one
        units = 1000 * (rank + 1)
        rate = ranks.job_rate(dist, units, seconds)
        mx = ranks.max_over_ranks(dist, seconds)
        dist.barrier()
        q.put((rank, rate, mx, ranks.rank_seed(5, rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_job_rate():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, mx, seed in out:
        assert mx == 2.0
        assert rate == pytest.approx(3000 / 2.0)
    assert out[0][3] != out[1][3]
