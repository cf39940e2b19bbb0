"""Sharding a visibility cube over ranks (one process per GPU).

The path partitions with no exchange on the data: every rank takes whole
frequency slabs [f0, f1) of the cube (so the autocorrelations its rounding
needs are its own, Sec. 3.1's noise being per frequency and time) and
compresses them into its own framed stream.  Putting the streams one after
another needs one number per rank: the exclusive scan of the stream lengths,
which is the only collective here (one int64 per rank).  Host logic only.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def freq_shards(n_freq: int, world: int):
    """[(f0, f1)] per rank: contiguous, covering [0, n_freq), sizes differing
    by at most one."""
    if world < 1:
        raise ValueError("world must be >= 1")
    q, r = divmod(n_freq, world)
    out, f = [], 0
    for k in range(world):
        n = q + (1 if k < r else 0)
        out.append((f, f + n))
        f += n
    return out


def concat_offsets(local_nbytes: int, group=None) -> tuple[int, int, list[int]]:
    """(this rank's byte offset in the concatenation, total bytes, every
    rank's length): an exclusive scan of the ranks' stream lengths by one
    all_gather of an int64 each."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    mine = torch.tensor([int(local_nbytes)], dtype=torch.int64, device=dev)
    allv = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(allv, mine, group=group)
    lens = [int(v.item()) for v in allv]
    return sum(lens[:rank]), sum(lens), lens


def shard_index(lens, shards) -> list[dict]:
    """A table of contents for the concatenated streams: per rank its
    frequency range, byte offset and length."""
    out, o = [], 0
    for (f0, f1), n in zip(shards, lens):
        out.append({"freq": (f0, f1), "offset": o, "nbytes": n})
        o += n
    return out
