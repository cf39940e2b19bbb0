"""Pins for the oracle's LZ4 block codec and framing (Sec. 4.1, Sec. 4.2.1).

Sec. 4.1 describes the LZ77 class that LZ4 belongs to: literals plus
(length, offset) back-references, run-length encoding when the length exceeds
the offset.  The byte layout checked here is the public LZ4 block format
(token nibbles = literal length and match length - 4, 255-continued length
bytes, 2-byte little-endian offsets, a literals-only last sequence, the last
5 bytes literals, the last match starting at least 12 bytes before the end).
Streams below are built by hand from that definition, with their expected
outputs written out; the system liblz4 (when present) cross-checks both ways.
"""
import ctypes
import ctypes.util
import itertools

import numpy as np
import pytest


def tok(ll, ml):
    """Token byte and the length-extension bytes for a literal length ll and
    a match length ml (None for the last, literals-only sequence)."""
    ext = b""
    hi = min(ll, 15)
    if ll >= 15:
        v = ll - 15
        ext += b"\xff" * (v // 255) + bytes([v % 255])
    if ml is None:
        return bytes([hi << 4]), ext, b""
    m = ml - 4
    lo = min(m, 15)
    mext = b""
    if m >= 15:
        v = m - 15
        mext = b"\xff" * (v // 255) + bytes([v % 255])
    return bytes([(hi << 4) | lo]), ext, mext


# hand-built streams and their decoded blocks
HAND = []
# literal-only block
HAND.append(("literals-only", b"\x30abc", b"abc"))
# 'a', match offset 1 length 20 (run-length), last literals "bcdef"
HAND.append(("rle-offset-1", b"\x1fa\x01\x00\x01" + b"\x50bcdef", b"a" * 21 + b"bcdef"))
# "xyz", overlapping match offset 3 length 10, last literals "12345"
HAND.append(("overlap-offset-3", b"\x36xyz\x03\x00" + b"\x5012345", b"xyzxyzxyzxyzx" + b"12345"))
# final literal runs across the 15 / 255 extension boundaries
for ll, head in [(14, b"\xe0"), (15, b"\xf0\x00"), (269, b"\xf0\xfe"), (270, b"\xf0\xff\x00"),
                 (271, b"\xf0\xff\x01")]:
    lits = bytes((7 * k + 3) % 251 for k in range(ll))
    HAND.append((f"literals-{ll}", head + lits, lits))
# match lengths across the boundaries: 'q' + run of length ml + "vwxyz"
for ml, head, ext in [(18, b"\x1e", b""), (19, b"\x1f", b"\x00"), (273, b"\x1f", b"\xfe"),
                      (274, b"\x1f", b"\xff\x00")]:
    HAND.append((f"match-{ml}", head + b"q\x01\x00" + ext + b"\x50vwxyz", b"q" * (1 + ml) + b"vwxyz"))


@pytest.mark.parametrize("name,stream,plain", HAND, ids=[h[0] for h in HAND])
def test_hand_built_streams_decode(orc, name, stream, plain):
    rc, out = orc.lz4_decompress_block(stream, len(plain))
    assert rc == 0 and out == plain


def test_tok_helper_matches_hand_bytes():
    # the helper used for generated streams agrees with the hand-written bytes
    assert b"".join(tok(1, 20)) == b"\x1f\x01"
    assert b"".join(tok(270, None)) == b"\xf0\xff\x00"
    assert b"".join(tok(1, 274)) == b"\x1f\xff\x00"


@pytest.mark.parametrize("name,stream,plain", HAND, ids=[h[0] for h in HAND])
def test_hand_built_round_trip(orc, name, stream, plain):
    c = orc.lz4_compress_block(plain)
    rc, out = orc.lz4_decompress_block(c, len(plain))
    assert rc == 0 and out == plain


def test_strict_decoder_rejects(orc):
    good = b"\x1fa\x01\x00\x01" + b"\x50bcdef"
    n = 26
    assert orc.lz4_decompress_block(good, n)[0] == 0
    assert orc.lz4_decompress_block(b"\x1fa\x00\x00\x01\x50bcdef", n)[0] == -3      # offset 0
    assert orc.lz4_decompress_block(b"\x1fa\x02\x00\x01\x50bcdef", n)[0] == -4      # before start
    assert orc.lz4_decompress_block(good, n - 1)[0] != 0                           # overrun
    assert orc.lz4_decompress_block(good, n + 1)[0] == -6                          # too short
    for cut in range(len(good)):
        assert orc.lz4_decompress_block(good[:cut], n)[0] != 0                     # truncated
    # a match reaching into the last 5 bytes breaks the end-of-block rule
    assert orc.lz4_decompress_block(b"\x1fa\x01\x00\x01\x40bcde", 25)[0] == -7
    assert orc.lz4_decompress_block(b"\x30abc", 4)[0] == -6
    assert orc.lz4_decompress_block(b"\x30abc", 2)[0] == -2


def test_brute_force_round_trip(orc):
    for L in range(0, 15):
        for s in itertools.product(b"\x00\x01", repeat=L):
            s = bytes(s)
            c = orc.lz4_compress_block(s)
            rc, out = orc.lz4_decompress_block(c, L)
            assert rc == 0 and out == s
    rng = np.random.default_rng(0)
    for _ in range(3000):
        L = int(rng.integers(0, 65))
        alpha = int(rng.integers(1, 5))
        s = rng.integers(0, alpha, size=L, dtype=np.uint8).tobytes()
        c = orc.lz4_compress_block(s)
        assert len(c) <= orc.lz4_bound(L)
        rc, out = orc.lz4_decompress_block(c, L)
        assert rc == 0 and out == s


def test_structured_round_trip_and_zero_block(orc):
    rng = np.random.default_rng(1)
    for L in (13, 100, 4096, 8192, 65536):
        for kind in ("zero", "period", "rand", "mixed"):
            if kind == "zero":
                s = bytes(L)
            elif kind == "period":
                s = (bytes(rng.integers(0, 256, 7, dtype=np.uint8)) * (L // 7 + 1))[:L]
            elif kind == "rand":
                s = rng.integers(0, 256, L, dtype=np.uint8).tobytes()
            else:
                s = b"".join(bytes([k % 3]) * int(rng.integers(1, 40)) + rng.integers(0, 256, 5, dtype=np.uint8).tobytes()
                             for k in range(L // 20 + 1))[:L]
            c = orc.lz4_compress_block(s)
            rc, out = orc.lz4_decompress_block(c, L)
            assert rc == 0 and out == s
            if kind == "zero" and L >= 4096:
                assert len(c) < 0.01 * L


def _liblz4():
    name = ctypes.util.find_library("lz4")
    if not name:
        return None
    try:
        L = ctypes.CDLL(name)
        L.LZ4_decompress_safe.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int]
        L.LZ4_compress_default.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int]
        return L
    except OSError:
        return None


def test_third_party_liblz4_cross_check(orc):
    L = _liblz4()
    if L is None:
        pytest.skip("no system liblz4")
    rng = np.random.default_rng(2)
    cases = [bytes(8192), rng.integers(0, 256, 8192, dtype=np.uint8).tobytes()]
    cases += [h[2] for h in HAND]
    cases += [rng.integers(0, 3, int(rng.integers(1, 3000)), dtype=np.uint8).tobytes() for _ in range(50)]
    for s in cases:
        c = orc.lz4_compress_block(s)
        buf = ctypes.create_string_buffer(len(s) + 16)
        n = L.LZ4_decompress_safe(c, buf, len(c), len(s))
        assert n == len(s) and buf.raw[:n] == s
        cap = len(s) + len(s) // 255 + 16
        cbuf = ctypes.create_string_buffer(cap)
        m = L.LZ4_compress_default(s, cbuf, len(s), cap)
        assert m > 0
        rc, out = orc.lz4_decompress_block(cbuf.raw[:m], len(s))
        assert rc == 0 and out == s


# -- framing (reading R11) ---------------------------------------------------

@pytest.mark.parametrize("es,dt", [(1, np.uint8), (2, np.uint16), (4, np.uint32), (8, np.uint64)])
@pytest.mark.parametrize("n", [0, 3, 8, 9, 1000, 4096, 4101, 10000])
def test_framing_round_trip(orc, es, dt, n):
    from paper_1503_00638_gb300 import synth
    a = synth.random_walk(n, dt, seed=n + es)
    B = 512
    s, sizes = orc.compress(a, B, return_block_sizes=True)
    hdr = np.frombuffer(s[:12], dtype=np.uint8)
    assert int.from_bytes(s[:8], "big") == n * es
    assert int.from_bytes(s[8:12], "big") == B * es
    # walk the block headers
    pos, k = 12, 0
    done = 0
    while done < n:
        Bb = B if n - done >= B else (n - done) - (n - done) % 8
        if Bb == 0:
            break
        c = int.from_bytes(s[pos:pos + 4], "big")
        assert c == sizes[k]
        pos += 4 + c
        done += Bb
        k += 1
    assert pos + (n - done) * es == len(s)
    assert s[pos:] == a[done:].tobytes()
    rc, back = orc.decompress(s, n, dt, B)
    assert rc == 0 and np.array_equal(back, a)
    assert len(s) <= orc.compress_bound(n, es, B)
    # corrupt streams fail cleanly
    if len(s) > 12:
        assert orc.decompress(s[:-1], n, dt, B)[0] != 0
        assert orc.decompress(s + b"\x00", n, dt, B)[0] == -13
    assert orc.decompress(s, n + 1, dt, B)[0] == -11
