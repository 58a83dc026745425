"""Host logic of the multi-GPU path on CPU: world-size-2 gloo process group.

Each rank takes a disjoint channel block; the blocks tile the band; the
timing reduction is the maximum over ranks; the gathered blocks reassemble the
full channel axis in order.  The per-rank payload stands in for the
visibilities a GPU would compute (no GPU here).
"""
import os
import socket

import numpy as np
import pytest

from paper_2506_02130_gb300 import shard


@pytest.mark.parametrize("n_freq,world", [(64, 2), (7, 3), (1, 1), (5, 8)])
def test_channel_blocks_tile_the_band(n_freq, world):
    seen = []
    for r in range(world):
        lo, hi = shard.channel_block(n_freq, r, world)
        assert 0 <= lo <= hi <= n_freq
        seen.extend(range(lo, hi))
    assert seen == list(range(n_freq))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_freq, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard.channel_block(n_freq, rank, world)
    block = np.arange(lo, hi, dtype=np.float64)[:, None] * np.ones((1, 3))
    t = shard.max_over_ranks(1.5 + rank, dist)
    full = shard.gather_blocks(block, n_freq, dist)
    if rank == 0:
        q.put((t, full))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_partition_time_and_gather():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world, n_freq = 2, 11
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_freq, q)) for r in range(world)]
    for p in procs:
        p.start()
    t, full = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 2.5
    np.testing.assert_array_equal(full[:, 0], np.arange(n_freq))


def test_sub_problem_restricts_channels():
    from paper_2506_02130_gb300 import workloads as W
    prob = W.config_hex127(seed=3, n_chan=10, n_time=1, n_point=50, nside=0, radius=1)
    sub, (lo, hi) = shard.sub_problem(prob, 1, 3)
    assert (lo, hi) == (4, 7)
    np.testing.assert_array_equal(sub.freqs_hz, prob.freqs_hz[4:7])
    np.testing.assert_array_equal(sub.sky.flux, prob.sky.flux[:, :, 4:7])
    assert prob.sky.flux.shape[2] == 10
