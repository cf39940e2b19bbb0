"""Pins for the oracle's Bitshuffle (Sec. 4.2, Sec. 6 step 4).

The bit matrix of a block (elements x bits) is transposed; bits are numbered
LSB-first within little-endian bytes as in the caption of Fig. f:bits.  The
oracle is checked against numpy's unpackbits/packbits written as "arrange the
bits in a matrix, transpose" (an independent formulation), the textbook 8x8
bit-matrix transpose, single-bit probes, popcount, zero blocks and the
involution with bitunshuffle, including ragged tails (reading R9).
"""
import numpy as np
import pytest

DTYPES = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}


def np_bitshuffle(a, B):
    """Sec. 6 step 4 with numpy: per block, an (elements x 8*es) bit matrix
    (bit column r = 8 * byte + bit, LSB first) transposed and repacked."""
    es = a.itemsize
    n = a.size
    raw = a.view(np.uint8).reshape(n, es)
    bits = np.unpackbits(raw, axis=1, bitorder="little")          # (n, 8 es)
    out = bytearray()
    done = 0
    while done < n:
        Bb = B if n - done >= B else (n - done) - (n - done) % 8
        if Bb == 0:
            break
        m = bits[done:done + Bb].T                                  # (8 es, Bb)
        out += np.packbits(m, axis=1, bitorder="little").tobytes()
        done += Bb
    out += raw[done:].tobytes()
    return np.frombuffer(bytes(out), dtype=a.dtype)


def _rand(n, es, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=n * es, dtype=np.uint8).view(DTYPES[es])


@pytest.mark.parametrize("es", [1, 2, 4, 8])
@pytest.mark.parametrize("B", [8, 16, 64, 1024, 2048])
@pytest.mark.parametrize("n", [0, 5, 8, 9, 15, 16, 100, 2048, 2049, 2055, 2056, 5000])
def test_matches_numpy_formulation(orc, es, B, n):
    a = _rand(n, es, seed=n * 31 + es * 7 + B)
    got = orc.bitshuffle(a, B)
    assert np.array_equal(got.view(np.uint8), np_bitshuffle(a, B).view(np.uint8))
    assert np.array_equal(orc.bitunshuffle(got, B).view(np.uint8), a.view(np.uint8))


def test_textbook_8x8(orc):
    """es = 1, B = 8: the 8x8 bit-matrix transpose, out byte r bit e = in byte e bit r."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        a = rng.integers(0, 256, size=8, dtype=np.uint8)
        out = orc.bitshuffle(a, 8)
        for r in range(8):
            for e in range(8):
                assert (out[r] >> e) & 1 == (a[e] >> r) & 1


@pytest.mark.parametrize("es,B", [(1, 16), (2, 24), (4, 32), (8, 8)])
def test_single_bit_probes(orc, es, B):
    for e in range(B):
        for r in range(8 * es):
            a = np.zeros(B * es, dtype=np.uint8)
            a[e * es + r // 8] = 1 << (r % 8)
            out = orc.bitshuffle(a.view(DTYPES[es]), B).view(np.uint8)
            nz = np.flatnonzero(out)
            assert nz.tolist() == [r * (B // 8) + e // 8]
            assert out[nz[0]] == 1 << (e % 8)


def test_popcount_and_zero(orc):
    a = _rand(4096 + 13, 4, 9)
    out = orc.bitshuffle(a, 1024)
    pc = lambda x: int(np.unpackbits(x.view(np.uint8)).sum())
    for b in range(4):
        assert pc(a[b * 1024:(b + 1) * 1024]) == pc(out[b * 1024:(b + 1) * 1024])
    z = np.zeros(4096, dtype=np.uint16)
    assert not orc.bitshuffle(z, 512).any()


def test_default_block_is_4096_bytes(orc):
    # Sec. 4.2.1: the default block size is 4096 bytes
    for es in (1, 2, 4, 8):
        a = _rand(3 * 4096 // es + 40, es, es)
        assert np.array_equal(orc.bitshuffle(a, 0), orc.bitshuffle(a, 4096 // es))


def test_twos_complement_rows_repeat(orc):
    """Sec. 4.2: for small signed values crossing zero, the most significant
    bit rows are identical to one another."""
    rng = np.random.default_rng(2)
    a = rng.integers(-50, 50, size=1024).astype(np.int32)
    out = orc.bitshuffle(a, 1024).view(np.uint8).reshape(32, 128)
    for r in range(8, 32):
        assert np.array_equal(out[r], out[31])


def test_each_column_is_one_integration(orc):
    """Caption of Fig. f:bits: after the transpose of 16-bit (re, im) data laid
    out in rows of 96 bits, each column holds a single integration.  A block of
    B = 96 16-bit elements (48 integrations of re, im) transposes to 16 rows of
    96 bits; element e lands in bit column e of every row."""
    a = np.arange(96, dtype=np.uint16) * 37
    out = orc.bitshuffle(a, 96).view(np.uint8)
    rows = np.unpackbits(out.reshape(16, 12), axis=1, bitorder="little")     # (16, 96)
    for e in range(96):
        col = rows[:, e]
        assert int(sum(int(b) << r for r, b in enumerate(col))) == int(a[e])


def test_bad_arguments(orc):
    with pytest.raises(ValueError):
        orc.bitshuffle(np.zeros(16, dtype=np.uint32), 12)
    with pytest.raises(ValueError):
        orc.bitshuffle(np.zeros(16, dtype=np.uint32), 4)
