"""GPU tests of the batched codec (one persistent launch over many chunks):

* every chunk's stream is byte-identical to the single-chunk bsgpu_compress()
  stream of the same chunk (so it is also oracle-decodable: checked too);
* the batch decompressor restores every chunk, with the block index and by
  walking each chunk's block chain, with lengths from the host or the device;
* a corrupt chunk is reported in its own status word and leaves the others
  intact; results do not depend on the launch shape; a captured CUDA graph
  replays to the same bytes and reads the inputs at replay time;
* 2-byte elements through the in-place transposes, single-chunk path.
"""
import numpy as np
import pytest
import torch

from paper_1503_00638_gb300 import synth

pytestmark = pytest.mark.gpu

DT = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}


@pytest.fixture(scope="module")
def bs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00638_gb300 import build
    build.build()
    from paper_1503_00638_gb300 import bsgpu
    return bsgpu


@pytest.fixture(scope="module")
def eng_mod(bs):
    from paper_1503_00638_gb300 import engine
    return engine


def mixed_batch(seed=0, n_chunks=40, max_elems=300_000):
    """(host arrays, elem sizes, block sizes): every element size, empty and
    tiny chunks, ragged lengths, several block sizes up to 8 KiB, random-walk
    and rounded-visibility contents."""
    rng = np.random.default_rng(seed)
    fixed = [(0, 4, 0), (1, 1, 0), (7, 8, 0), (8, 2, 8), (9, 4, 8), (4099, 2, 0),
             (2048 * 3, 4, 2048), (4096 * 2 + 17, 2, 4096), (1024 * 5 + 3, 8, 1024),
             (333, 1, 24), (65536 + 5, 1, 8192)]
    arrays, es_l, bl = [], [], []
    for k, (n, es, B) in enumerate(fixed):
        arrays.append(synth.random_walk(n, DT[es], seed=100 + k))
        es_l.append(es)
        bl.append(B)
    vis = synth.visibilities(synth.CONFIG_SMALL).view(np.uint32).reshape(-1)
    while len(arrays) < n_chunks:
        es = int(rng.choice([1, 2, 4, 8]))
        n = int(np.exp(rng.uniform(np.log(8), np.log(max_elems))))
        choices = [b for b in (0, 8, 64, 256, 512, 1024, 2048, 4096) if b * es <= 8192]
        B = int(rng.choice(choices))
        if es == 4 and rng.random() < 0.5:
            a = vis[:n].copy() if n <= vis.size else np.resize(vis, n)
        else:
            a = synth.random_walk(n, DT[es], seed=int(rng.integers(1 << 30)))
        arrays.append(a)
        es_l.append(es)
        bl.append(B)
    return arrays, es_l, bl


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).copy()).cuda()


@pytest.mark.parametrize("level", [0, 1])
def test_batch_equals_single_chunk_streams(bs, orc, eng_mod, level):
    arrays, es_l, bl = mixed_batch(seed=level)
    xs = [to_dev(a) for a in arrays]
    e = eng_mod.BatchCodec(xs, es_l, bl, level=level)
    e.compress()
    e.decompress()
    sc, sd = e.statuses()
    assert sc == [0] * e.n and sd == [0] * e.n
    for i, (a, x, es, B) in enumerate(zip(arrays, xs, es_l, bl)):
        got = e.stream(i)
        single = bs.compress(x, B, elem_size=es, level=level)
        assert single.nbytes == got.numel(), i
        assert torch.equal(single.buf[:single.nbytes], got), i
        assert torch.equal(e.output(i), x), i
        if i % 4 == 0:
            rc, back = orc.decompress(got.cpu().numpy().tobytes(), a.size, a.dtype, B)
            assert rc == 0 and np.array_equal(back, a), i


def test_batch_decompress_without_index_and_host_lengths(bs, eng_mod):
    arrays, es_l, bl = mixed_batch(seed=5, n_chunks=24, max_elems=50_000)
    xs = [to_dev(a) for a in arrays]
    e = eng_mod.BatchCodec(xs, es_l, bl, with_offsets=False)
    e.compress()
    # host-side lengths in the table instead of the device array
    lens = e.out_bytes.cpu().tolist()
    base = e.stream_arena.data_ptr()
    dbase = e.dec_arena.data_ptr()
    e.dec_arena.zero_()
    ch = [bs.Chunk(base + so, dbase + do, n, ln, 0, es, B)
          for so, do, n, ln, es, B in zip(e.stream_off, e.dec_off, e.n_elem, lens, es_l, bl)]
    table, n_items, ws = bs.batch_plan(bs.OP_DECOMPRESS, ch)
    status = torch.zeros(e.n, dtype=torch.int32, device="cuda")
    wsd = bs.new_workspace(ws)
    bs.decompress_batch(table.cuda(), e.n, n_items, None, None, status, wsd)
    assert status.cpu().tolist() == [0] * e.n
    for i, x in enumerate(xs):
        assert torch.equal(e.output(i), x), i


def test_corrupt_chunk_is_isolated(bs, eng_mod):
    arrays, es_l, bl = mixed_batch(seed=7, n_chunks=16, max_elems=40_000)
    xs = [to_dev(a) for a in arrays]
    e = eng_mod.BatchCodec(xs, es_l, bl)
    e.compress()
    torch.cuda.synchronize()
    victims = [i for i in range(e.n) if e.n_elem[i] >= 4096][:2]
    for v in victims:
        o = e.stream_off[v]
        e.stream_arena[o + 12 + 4 + 5] ^= 0xFF      # inside block 0's LZ4 data
    hdr = [i for i in range(e.n) if i not in victims and e.n_elem[i] > 0][0]
    e.stream_arena[e.stream_off[hdr] + 3] ^= 1      # header byte
    e.decompress()
    _, sd = e.statuses()
    for i in range(e.n):
        if i in victims or i == hdr:
            assert sd[i] in (0, bs.ERR_CORRUPT)
            if i == hdr:
                assert sd[i] == bs.ERR_CORRUPT
        else:
            assert sd[i] == 0, i
            assert torch.equal(e.output(i), xs[i]), i


def test_launch_shape_does_not_change_streams(bs, eng_mod):
    arrays, es_l, bl = mixed_batch(seed=9, n_chunks=30, max_elems=100_000)
    xs = [to_dev(a) for a in arrays]
    e = eng_mod.BatchCodec(xs, es_l, bl)
    ref = None
    for w, k in ((1, 0), (1, 1), (1, 3), (1, 16), (2, 0), (2, 3), (4, 0), (4, 1)):
        e.ctas_c = e.ctas_d = k
        e.warps_c = e.warps_d = w
        e.stream_arena.zero_()
        e.dec_arena.zero_()
        e.compress()
        e.decompress()
        snap = [e.stream(i).clone() for i in range(e.n)]
        assert all(torch.equal(e.output(i), xs[i]) for i in range(e.n))
        if ref is None:
            ref = snap
        else:
            assert all(torch.equal(a, b) for a, b in zip(ref, snap))
    c, d = e.autotune(shapes=((1, 0), (1, 4), (2, 8), (4, 0)), reps=1)
    assert (c.warps_per_cta, c.ctas_per_sm) in ((1, 0), (1, 4), (2, 8), (4, 0))
    assert (d.warps_per_cta, d.ctas_per_sm) in ((1, 0), (1, 4), (2, 8), (4, 0))
    assert set(c.table) == {"1x0", "1x4", "2x8", "4x0"}
    with pytest.raises(bs.BsgpuError):
        bs.compress_batch(e.table_c, e.n, e.n_items, e.out_bytes, e.offsets, e.status_c, e.ws_c,
                          warps_per_cta=3)


def test_tuner_picks_block_size_and_shapes(bs, eng_mod, orc):
    """The batch autotuner over block size x warps per CTA x CTAs per SM:
    every candidate is timed and listed, the chosen codec runs with the
    chosen shapes, and its streams decode with the oracle."""
    arrays, es_l, _ = mixed_batch(seed=13, n_chunks=24, max_elems=120_000)
    xs = [to_dev(a) for a in arrays]
    best, table, e = eng_mod.tune(xs, es_l, (2048, 8192), shapes=((1, 0), (2, 0), (4, 2)), reps=1)
    assert best in (2048, 8192) and set(table) == {2048, 8192}
    for rec in table.values():
        assert set(rec["compress"]["candidates_ms"]) == {"1x0", "2x0", "4x2"}
        assert rec["round_trip_ms"] > 0 and rec["compressed_bytes"] > 0
    assert (e.warps_c, e.ctas_c) == (table[best]["compress"]["warps_per_cta"],
                                     table[best]["compress"]["ctas_per_sm"])
    e.compress()
    e.decompress()
    assert all(torch.equal(e.output(i), xs[i]) for i in range(e.n))
    for i in range(0, e.n, 5):
        rc, back = orc.decompress(e.stream(i).cpu().numpy().tobytes(), arrays[i].size,
                                  arrays[i].dtype, best // es_l[i])
        assert rc == 0 and np.array_equal(back, arrays[i])


def test_graph_replay(bs, eng_mod):
    arrays, es_l, bl = mixed_batch(seed=11, n_chunks=20, max_elems=80_000)
    xs = [to_dev(a) for a in arrays]
    e = eng_mod.BatchCodec(xs, es_l, bl)
    g = e.capture()
    for rep in range(2):
        # new contents, same shapes: the graph reads the inputs at replay time
        for i, x in enumerate(xs):
            x.copy_(to_dev(synth.random_walk(x.numel() // es_l[i], DT[es_l[i]], seed=rep * 100 + i)))
        e.stream_arena.zero_()
        g.replay()
        torch.cuda.synchronize()
        for i, x in enumerate(xs):
            single = bs.compress(x, bl[i], elem_size=es_l[i])
            assert torch.equal(single.buf[:single.nbytes], e.stream(i)), (rep, i)
            assert torch.equal(e.output(i), x), (rep, i)


def test_many_chunks_one_launch(bs, eng_mod):
    # 1000 chunks of 1..40 blocks: look-back within every chunk at once
    rng = np.random.default_rng(3)
    es_l = [int(rng.choice([2, 4, 8])) for _ in range(1000)]
    xs, arrays = [], []
    for i, es in enumerate(es_l):
        n = int(rng.integers(1, 41)) * (8192 // es) - int(rng.integers(0, 20))
        a = synth.random_walk(max(n, 1), DT[es], seed=i)
        arrays.append(a)
        xs.append(to_dev(a))
    bl = [8192 // es for es in es_l]
    e = eng_mod.BatchCodec(xs, es_l, bl)
    e.compress()
    e.decompress()
    sc, sd = e.statuses()
    assert sc == [0] * e.n and sd == [0] * e.n
    for i in range(0, e.n, 37):
        single = bs.compress(xs[i], bl[i], elem_size=es_l[i])
        assert torch.equal(single.buf[:single.nbytes], e.stream(i)), i
    assert all(torch.equal(e.output(i), xs[i]) for i in range(e.n))


@pytest.mark.parametrize("B", [64, 128, 1536, 2048, 4096, 0])
def test_two_byte_elements_single_path(bs, orc, B):
    a = synth.random_walk(4096 * 9 + 77, np.uint16, seed=B)
    x = to_dev(a)
    rows = bs.bitshuffle(x.view(torch.int16), B)
    assert np.array_equal(rows.cpu().numpy().view(np.uint16), orc.bitshuffle(a, B))
    for level in (0, 1):
        c = bs.compress(x, B, elem_size=2, level=level)
        assert bs.status(c.ws) == 0
        rc, back = orc.decompress(c.stream_bytes().cpu().numpy().tobytes(), a.size, np.uint16, B)
        assert rc == 0 and np.array_equal(back, a)
        out = bs.decompress(c.buf, c.nbytes, a.size, 2, B, offsets=c.offsets)
        assert torch.equal(out, x)
