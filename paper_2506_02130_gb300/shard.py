"""Multi-GPU sharding of a simulation: independent (time, channel) slices.

Slices share nothing but the read-only array and sky, so N GPUs each take a
disjoint block of channels and simulate it with their own plan; no collective
touches the data path.  This is the paper's own multi-node scheme (frequency
blocks as independent jobs, Section 5.4) with one process per GPU.  The only
communication is on the host: the ranks' wall-clock maximum for timing and an
optional gather of the visibility blocks.
"""
from __future__ import annotations

import numpy as np


def channel_block(n_freq: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) channel range of `rank`: contiguous, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_freq, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def sub_problem(prob, rank: int, world: int):
    """The workload restricted to this rank's channel block (a shallow copy)."""
    import copy
    lo, hi = channel_block(len(prob.freqs_hz), rank, world)
    p = copy.copy(prob)
    p.sky = copy.copy(prob.sky)
    p.freqs_hz = np.asarray(prob.freqs_hz)[lo:hi]
    p.sky.flux = prob.sky.flux[:, :, lo:hi]
    return p, (lo, hi)


def max_over_ranks(value: float, dist=None) -> float:
    """Maximum of a per-rank scalar (seconds) over the process group, on the host."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_blocks(block: np.ndarray, n_freq: int, dist=None) -> np.ndarray | None:
    """Assemble [n_freq, ...] on rank 0 from every rank's channel block (host gather)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return block
    world, rank = dist.get_world_size(), dist.get_rank()
    parts = [None] * world
    dist.gather_object(block, parts if rank == 0 else None, dst=0)
    if rank != 0:
        return None
    out = np.concatenate(parts, axis=0)
    assert out.shape[0] == n_freq
    return out
