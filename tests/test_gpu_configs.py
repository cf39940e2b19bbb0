"""GPU parity at the stated sizes of the codec-only and batched workloads.

* Bitshuffle + LZ4 only (Sec. 4.2, Sec. 6 steps 4-5): uint8 / uint16 / int32
  / float64 random walks of 1 GB and 4 GB with blocks of 1024, 2048, 4096
  and 8192 elements.  The oracle bit-transposes sampled blocks (the first,
  one in the middle, the last full one, the shortened last block and the
  verbatim tail of reading R9) and decodes sampled blocks of the GPU stream;
  both GPU round trips (un-Bitshuffle, decompress) return the input exactly.
* The batched workload (Sec. 4.2.1: blocks are independent units of work):
  a few hundred chunks of the batch generator (sizes log-uniform on 64 KiB ..
  64 MiB, element sizes 2 / 4 / 8, half rounded visibility cubes, half
  random walks) in one persistent launch each way.  The GPU rounding of the
  visibility chunks equals the oracle's (Sec. 3.2); the oracle decodes one
  chunk of every (element size, kind) pair; every chunk round-trips exactly.
"""
import numpy as np
import pytest
import torch

from paper_1503_00638_gb300 import synth

pytestmark = pytest.mark.gpu

DT = {1: np.uint8, 2: np.uint16, 4: np.int32, 8: np.float64}


@pytest.fixture(scope="module")
def bs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00638_gb300 import build
    build.build()
    from paper_1503_00638_gb300 import bsgpu
    return bsgpu


def _elems(t: torch.Tensor, es: int, a: int, b: int) -> np.ndarray:
    """Elements [a, b) of the byte tensor t as a host array."""
    return t[a * es:b * es].cpu().numpy().view(DT[es])


def _same(x: np.ndarray, y: np.ndarray) -> bool:
    """Bitwise equality (float64 walks hold no NaN, but transposed bits do)."""
    return np.array_equal(x.view(np.uint8), y.view(np.uint8))


@pytest.mark.parametrize("size", [10 ** 9, 4 * 10 ** 9], ids=["1GB", "4GB"])
@pytest.mark.parametrize("es", [1, 2, 4, 8])
def test_codec_only_at_size(bs, orc, es, size):
    n = size // es + 13                         # a ragged last block and a verbatim tail
    x = synth.random_walk_device(n, es, seed=es * 7 + size % 97, floating=(es == 8))
    stream = torch.cuda.current_stream().cuda_stream
    for B in (1024, 2048, 4096, 8192):
        nfull = n // B
        last = (n % B) - (n % B) % 8            # the shortened last block (R9)
        # Bitshuffle: sampled blocks and the tail against the oracle
        sh = torch.empty_like(x)
        bs._check(bs._lib.bsgpu_bitshuffle(x.data_ptr(), sh.data_ptr(), n, es, B, stream),
                  "bitshuffle")
        for b in sorted({0, 1, nfull // 2, nfull - 1}):
            want = orc.bitshuffle(_elems(x, es, b * B, (b + 1) * B), B)
            assert _same(_elems(sh, es, b * B, (b + 1) * B), want), (B, b)
        want = orc.bitshuffle(_elems(x, es, nfull * B, n), B)   # short block + verbatim tail
        assert _same(_elems(sh, es, nfull * B, n), want), (B, "tail")
        back = torch.empty_like(x)
        bs._check(bs._lib.bsgpu_bitunshuffle(sh.data_ptr(), back.data_ptr(), n, es, B, stream),
                  "bitunshuffle")
        assert torch.equal(back, x), B
        del sh, back
        # LZ4: the GPU stream round-trips; the oracle decodes sampled blocks
        c = bs.compress(x, B, elem_size=es)
        assert bs.status(c.ws) == 0
        out = bs.decompress(c.buf, c.nbytes, n, es, B, offsets=c.offsets)
        assert torch.equal(out, x), B
        del out
        nblk = bs.num_blocks(n, es, B)
        assert nblk == nfull + (1 if last else 0)
        offs = c.offsets[:nblk].cpu().numpy()
        for b in sorted({0, nfull // 3, nblk - 1}):
            o = int(offs[b])
            clen = int.from_bytes(c.buf[o:o + 4].cpu().numpy().tobytes(), "big")
            blk = c.buf[o + 4:o + 4 + clen].cpu().numpy().tobytes()
            Bb = B if b < nfull else last
            rc, rows = orc.lz4_decompress_block(blk, Bb * es)
            assert rc == 0, (B, b)
            plain = orc.bitunshuffle(np.frombuffer(rows, dtype=DT[es]).copy(), Bb)
            assert _same(plain, _elems(x, es, b * B, b * B + Bb)), (B, b)
        # the verbatim tail closes the stream
        tb = (n % 8) * es
        assert torch.equal(c.buf[c.nbytes - tb:c.nbytes], x[n * es - tb:])
        del c
        torch.cuda.empty_cache()


def test_batch_workload_against_oracle(bs, orc):
    from paper_1503_00638_gb300 import engine
    specs = synth.batch_specs(300, seed=1)
    xs, raw = [], {}
    per_freq = synth.n_products(16) * 64 * 8
    # the smallest visibility chunk of each element size keeps its raw cube
    keep = {}
    for k, (nb, es, kind) in enumerate(specs):
        if kind == "vis" and (es not in keep or nb < specs[keep[es]][0]):
            keep[es] = k
    for k, (nb, es, kind) in enumerate(specs):
        if kind == "vis":
            F = -(-nb // per_freq)
            cfg = synth.VisConfig(F, 16, 64, 2 ** 16, 0.01, seed=1000 + k)
            cube = synth.visibilities_torch(cfg)
            r = bs.reduce_precision_c64(cube, cfg.n_samp, cfg.f)
            xs.append(r.view(torch.uint8).reshape(-1)[:nb].clone())
            if k in keep.values():
                raw[k] = (cube.cpu().numpy(), cfg)
            del cube, r
        else:
            xs.append(synth.random_walk_torch(nb // es, es, seed=2000 + k))
    # the GPU rounding of the visibility chunks against the oracle's
    for k, (cube, cfg) in raw.items():
        want = orc.reduce_precision_c64(cube, cfg.n_samp, cfg.f).view(np.uint8).reshape(-1)
        assert np.array_equal(xs[k].cpu().numpy(), want[:specs[k][0]]), k
    es_l = [es for _, es, _ in specs]
    e = engine.BatchCodec(xs, es_l, [8192 // es for es in es_l])
    e.compress()
    e.decompress()
    sc, sd = e.statuses()
    assert sc == [0] * e.n and sd == [0] * e.n
    for i in range(e.n):
        assert torch.equal(e.output(i), xs[i]), i
    # the oracle decodes the smallest chunk of every (element size, kind) pair
    pick = {}
    for k, (nb, es, kind) in enumerate(specs):
        if (es, kind) not in pick or nb < specs[pick[(es, kind)]][0]:
            pick[(es, kind)] = k
    assert len(pick) == 6
    udt = {2: np.uint16, 4: np.uint32, 8: np.uint64}
    for (es, kind), k in pick.items():
        a = xs[k].cpu().numpy().view(udt[es])
        rc, back = orc.decompress(e.stream(k).cpu().numpy().tobytes(), a.size, a.dtype, 8192 // es)
        assert rc == 0 and np.array_equal(back, a), (es, kind)
