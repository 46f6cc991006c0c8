"""Multi-rank host logic on CPU with the gloo backend (world size 2 and 3):
contiguous sharding covers every point once, partial sums reduce to the
single-process total, and the timing maximum is taken over ranks."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_19456_b300 import distributed as qd


def test_shard_covers_every_point_once():
    for n in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            spans = [qd.shard(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        qd.shard(10, 2, 2)


def _worker(rank, world, port, values, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = qd.shard(len(values), world, rank)
        local = values[a:b]
        mean = qd.mc_mean(float(np.sum(local)), len(local))
        tmax = qd.max_over_ranks(float(rank + 1) * 0.5)
        results[rank] = (mean, tmax)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_reductions(world):
    values = np.random.default_rng(0).random(1001)
    port = 29500 + world + (os.getpid() % 500)
    with mp.get_context("spawn").Manager() as m:
        results = m.dict()
        mp.spawn(_worker, args=(world, port, values, results), nprocs=world, join=True)
        got = dict(results)
    for r in range(world):
        mean, tmax = got[r]
        assert abs(mean - values.mean()) < 1e-12
        assert tmax == 0.5 * world


def test_single_process_reductions_are_identity():
    assert qd.max_over_ranks(3.5) == 3.5
    assert qd.mc_mean(10.0, 4) == 2.5
