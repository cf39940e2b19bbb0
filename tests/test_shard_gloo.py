"""Sharding host logic on two gloo ranks (CPU, no GPU): frequency slabs per
rank, the exclusive scan of stream lengths, and the concatenation decoding
back to the whole rounded cube.  The shard streams are made by the oracle
(the GPU path is exercised by the GPU tests; here only the host logic)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1503_00638_gb300 import shard, synth

CFG = synth.VisConfig(7, 6, 16, 2 ** 12, 0.05, seed=3)
B = 512


def test_freq_shards():
    for n, w in ((7, 2), (1024, 8), (3, 3), (5, 1), (2, 4)):
        s = shard.freq_shards(n, w)
        assert len(s) == w and s[0][0] == 0 and s[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(s, s[1:]))
        sizes = [b - a for a, b in s]
        assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    f0, f1 = shard.freq_shards(CFG.n_freq, world)[rank]
    vis = synth.visibilities(CFG, f0, f1)
    rounded = oracle.reduce_precision_c64(vis, CFG.n_samp, CFG.f)
    stream = oracle.compress(rounded.view(np.float32).reshape(-1), B)
    off, total, lens = shard.concat_offsets(len(stream))
    # every rank writes its stream at its offset of one shared file
    path = os.path.join(out_dir, "cube.bin")
    if rank == 0:
        with open(path, "wb") as fh:
            fh.truncate(total)
    dist.barrier()
    with open(path, "r+b") as fh:
        fh.seek(off)
        fh.write(stream)
    dist.barrier()
    if rank == 0:
        np.save(os.path.join(out_dir, "lens.npy"), np.array(lens))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_ranks_concatenate(tmp_path, world, orc):
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    lens = np.load(tmp_path / "lens.npy").tolist()
    data = (tmp_path / "cube.bin").read_bytes()
    assert len(data) == sum(lens)
    shards = shard.freq_shards(CFG.n_freq, world)
    whole = orc.reduce_precision_c64(synth.visibilities(CFG), CFG.n_samp, CFG.f)
    for ent in shard.shard_index(lens, shards):
        f0, f1 = ent["freq"]
        s = data[ent["offset"]:ent["offset"] + ent["nbytes"]]
        want = whole[f0:f1].view(np.float32).reshape(-1)
        rc, back = orc.decompress(s, want.size, np.float32, B)
        assert rc == 0 and np.array_equal(back.view(np.uint32), want.view(np.uint32))
