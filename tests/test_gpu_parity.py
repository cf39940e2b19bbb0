"""GPU parity: every step of the path through the C-ABI against the CPU oracle.

* precision reduction: bit-exact float32 results (the granularity is decided
  in float32 on both sides by the same formula, reading R1);
* Bitshuffle / un-Bitshuffle: bit-exact bytes;
* LZ4 + framing: LZ4 output is not unique, so the GPU stream must decode with
  the oracle's strict decoder to exactly the input, the GPU decoder must read
  the oracle's streams, and the GPU encoder must be deterministic;
* the fused visibility path: GPU stream -> oracle decoder equals the oracle's
  rounded cube, bit for bit.
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


def to_dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).copy()).cuda()


def host_bytes(t: torch.Tensor) -> np.ndarray:
    return t.view(torch.uint8).cpu().numpy()


# ---------------------------------------------------------------- rounding --

VIS_CASES = [
    ("small", synth.CONFIG_SMALL),
    ("one-input", synth.VisConfig(3, 1, 5, 2 ** 10, 0.05, seed=2)),
    ("T1", synth.VisConfig(4, 7, 1, 2 ** 12, 0.01, seed=3)),
    ("T3", synth.VisConfig(5, 9, 3, 2 ** 14, 0.1, seed=4)),
    ("T40", synth.VisConfig(2, 12, 40, 2 ** 16, 1e-3, seed=5)),
    ("chime-slab", synth.VisConfig(4, 128, 16, 2 ** 17, 0.01, seed=6, drift=True)),
]


@pytest.mark.parametrize("name,cfg", VIS_CASES, ids=[c[0] for c in VIS_CASES])
@pytest.mark.parametrize("f", [None, 0.0, 1e-5, 0.1])
def test_reduce_precision_bit_exact(bs, orc, name, cfg, f):
    f = cfg.f if f is None else f
    vis = synth.visibilities(cfg)
    want = orc.reduce_precision_c64(vis, cfg.n_samp, f)
    d = torch.from_numpy(vis.copy()).cuda()
    got = bs.reduce_precision_c64(d, cfg.n_samp, f)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy().view(np.uint32), want.view(np.uint32))


def test_reduce_precision_special_values(bs, orc):
    cfg = synth.VisConfig(2, 4, 64, 2 ** 12, 0.05, seed=9)
    vis = synth.visibilities(cfg)
    flat = vis.view(np.float32).reshape(-1)
    rng = np.random.default_rng(0)
    idx = rng.choice(flat.size, 200, replace=False)
    specials = np.array([np.nan, np.inf, -np.inf, 0.0, -0.0, 1e-42, -1e-42, 3.4e38, -3.4e38,
                         1e-30], dtype=np.float32)
    flat[idx] = np.resize(specials, idx.size)
    # a zero and a negative auto (no usable q: values pass through, reading R2)
    vis[0, 0, 3] = 0.0
    vis[1, synth.auto_product_index(2, 4), 7] = -50.0
    want = orc.reduce_precision_c64(vis, cfg.n_samp, cfg.f)
    got = bs.reduce_precision_c64(torch.from_numpy(vis.copy()).cuda(), cfg.n_samp, cfg.f)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), want.view(np.uint32))


# ------------------------------------------------------------- bitshuffle --

SHUF = [(es, B, n) for es in (1, 2, 4, 8) for B in (8, 24, 512, 2048)
        for n in (0, 5, 8, 9, 2047, 4096 + 13, 20000)]
SHUF += [(4, 2048, 2048 * 300 + 77), (8, 1024, 1024 * 200 + 9), (2, 4096, 4096 * 64 + 15),
         (1, 8192, 8192 * 40 + 3), (4, 0, 50000), (8, 8192, 8192 * 7), (4, 16384, 16384 * 5 + 8),
         # blocks over 16 KiB go by 1024-element tiles: full blocks, a shortened
         # last block, a verbatim tail
         (4, 8192, 8192 * 40 + 19), (4, 8192, 8192 * 3), (8, 4096, 4096 * 30 + 5),
         (8, 8192, 8192 * 9 + 1029), (4, 5120, 5120 * 11 + 8), (8, 3072, 3072 * 7 + 100)]


@pytest.mark.parametrize("es,B,n", SHUF)
def test_bitshuffle_bit_exact(bs, orc, es, B, n):
    a = synth.random_walk(n, {1: np.uint8, 2: np.uint16, 4: np.int32, 8: np.float64}[es], seed=n + B)
    want = orc.bitshuffle(a, B)
    d = to_dev(a)
    if n == 0:
        return
    out = torch.empty_like(d)
    bs._check(bs._lib.bsgpu_bitshuffle(d.data_ptr(), out.data_ptr(), n, es, B,
                                       torch.cuda.current_stream().cuda_stream), "shuffle")
    assert np.array_equal(host_bytes(out), want.view(np.uint8))
    back = torch.empty_like(d)
    bs._check(bs._lib.bsgpu_bitunshuffle(out.data_ptr(), back.data_ptr(), n, es, B,
                                         torch.cuda.current_stream().cuda_stream), "unshuffle")
    assert np.array_equal(host_bytes(back), a.view(np.uint8))


def test_bitshuffle_large_sampled(bs, orc):
    """64 MiB of int32 random walk in 2048-element blocks: sampled blocks and
    the tail against the oracle; the full round trip exactly."""
    n = (64 << 20) // 4 + 1029
    a = synth.random_walk(n, np.int32, seed=11)
    d = to_dev(a)
    out = bs.bitshuffle(d.view(torch.int32), 2048)
    h = out.view(torch.uint8).cpu().numpy()
    for b in (0, 1, 4095, 8191, n // 2048 - 1):
        want = orc.bitshuffle(a[b * 2048:(b + 1) * 2048], 2048)
        assert np.array_equal(h[b * 8192:(b + 1) * 8192], want.view(np.uint8))
    tail0 = (n // 2048) * 2048
    want = orc.bitshuffle(a[tail0:], 2048)
    assert np.array_equal(h[tail0 * 4:], want.view(np.uint8))
    back = bs.bitunshuffle(out, 2048)
    assert torch.equal(back, d.view(torch.int32))


# ------------------------------------------------------------ LZ4 framing --

CODEC = [(es, B, n, kind) for es in (1, 2, 4, 8) for B in (8, 64, 1024)
         for n in (0, 3, 8, 13, 1000, 9000) for kind in ("walk",)]
CODEC += [(4, 2048, 2048 * 64 + 5, k) for k in ("walk", "zero", "rand", "const")]
CODEC += [(8, 8192, 8192 * 9 + 17, "walk"), (2, 4096, 4096 * 33, "walk"), (1, 16384, 16384 * 3 + 9, "walk"),
          (4, 0, 70001, "walk"), (4, 16384, 16384 * 4, "rand"), (8, 1024, 1024 * 257, "zero")]


def make(n, es, kind, seed):
    dt = {1: np.uint8, 2: np.uint16, 4: np.int32, 8: np.float64}[es]
    if kind == "walk":
        return synth.random_walk(n, dt, seed=seed)
    if kind == "zero":
        return np.zeros(n, dtype=dt)
    if kind == "const":
        return np.full(n, 7, dtype=dt)
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=n * es, dtype=np.uint8).view(dt)


CODEC_L = [(es, B, n, kind, 0) for (es, B, n, kind) in CODEC]
CODEC_L += [(es, B, n, kind, 1) for (es, B, n, kind) in CODEC[::3]]


@pytest.mark.parametrize("es,B,n,kind,level", CODEC_L)
def test_compress_decodes_with_oracle(bs, orc, es, B, n, kind, level):
    a = make(n, es, kind, seed=n * 3 + es)
    d = to_dev(a)
    c = bs.compress(d, B, elem_size=es, level=level)
    nbytes = c.nbytes
    assert bs.status(c.ws) == 0
    assert nbytes <= bs.compress_bound(n, es, B)
    s = c.buf[:nbytes].cpu().numpy().tobytes()
    rc, back = orc.decompress(s, n, a.dtype, B)
    assert rc == 0 and np.array_equal(back.view(np.uint8), a.view(np.uint8))
    # block offsets point at each block's length field
    if n >= 8:
        offs = c.offsets.cpu().numpy()
        pos = 12
        for b in range(bs.num_blocks(n, es, B)):
            assert offs[b] == pos
            pos += 4 + int.from_bytes(s[pos:pos + 4], "big")
    # deterministic: a second run writes the same bytes
    c2 = bs.compress(d, B, elem_size=es, level=level)
    assert c2.nbytes == nbytes and torch.equal(c2.buf[:nbytes], c.buf[:nbytes])
    # ... also into an output that does not start on a 16-byte boundary
    raw = torch.zeros(c.buf.numel() + 16, dtype=torch.uint8, device="cuda")
    c3 = bs.compress(d, B, elem_size=es, level=level, out=raw[5:5 + c.buf.numel()])
    assert c3.nbytes == nbytes and torch.equal(raw[5:5 + nbytes], c.buf[:nbytes])
    # GPU decoder, with and without the index, from an aligned and a
    # misaligned copy of the stream
    mis = torch.zeros(nbytes + 16, dtype=torch.uint8, device="cuda")
    mis[3:3 + nbytes] = c.buf[:nbytes]
    for src in (c.buf, mis[3:3 + nbytes]):
        for offs in (c.offsets if n >= 8 else None, None):
            out = bs.decompress(src, nbytes, n, es, B, offsets=offs)
            assert np.array_equal(host_bytes(out), a.view(np.uint8))
    # GPU decoder on the oracle's stream
    o = orc.compress(a, B)
    od = torch.from_numpy(np.frombuffer(o, dtype=np.uint8).copy()).cuda()
    ws = bs.new_workspace(bs.workspace_size(bs.OP_DECOMPRESS, n, es, B))
    out = bs.decompress(od, len(o), n, es, B, ws=ws)
    assert bs.status(ws) == 0
    assert np.array_equal(host_bytes(out), a.view(np.uint8))


def _structured_rows(rng, nwords, rowwords, kind):
    """One block's bit-rows as 32-bit words, built so that the level-0 parse
    sees many short matches: runs of equal words ("runs"), words copied from
    the bit-row above ("rows") or both with long zero stretches ("mixed").
    "runs" places a 4-word run every 40 words (about 50 candidate runs, so
    more than 32 sequences); "dense" every 12 (more than 127 candidate runs)."""
    w = rng.integers(0, 2 ** 32, size=nwords, dtype=np.uint64).astype(np.uint32)
    step = {"runs": 40, "dense": 12, "rows": 30, "mixed": 23}[kind]
    for i in range(step, nwords - 8, step):
        if kind in ("runs", "dense") or (kind == "mixed" and (i // step) % 3 == 0):
            w[i:i + 4] = w[i - 1]
        elif i >= rowwords:
            w[i:i + 5] = w[i - rowwords:i - rowwords + 5]
    if kind == "mixed":
        z0 = int(rng.integers(0, nwords // 2))
        w[z0:z0 + int(rng.integers(70, 300))] = 0
    return w


@pytest.mark.parametrize("es", [2, 4, 8])
def test_fast_encoder_structured_blocks(bs, orc, es):
    """Blocks whose bit-rows hold many short matches (more than 32 sequences,
    and more than 127 candidate runs, which take the encoder's walk instead
    of its parse graph) round-trip through the oracle's decoder."""
    B = 8192 // es
    rng = np.random.default_rng(20 + es)
    kinds = ["runs", "dense", "rows", "mixed"] * 3
    rows = np.concatenate([_structured_rows(rng, 2048, B // 32, k) for k in kinds])
    dt = {2: np.uint16, 4: np.int32, 8: np.float64}[es]
    a = orc.bitunshuffle(rows.view(dt), B)
    assert np.array_equal(orc.bitshuffle(a, B).view(np.uint32), rows)
    tail = np.arange(5, dtype=np.uint8).view(np.uint8)
    full = np.concatenate([a.view(np.uint8), np.resize(tail, 5 * es)]).view(dt)
    n = full.size
    c = bs.compress(to_dev(full), B, elem_size=es, level=0)
    assert bs.status(c.ws) == 0
    s = c.buf[:c.nbytes].cpu().numpy().tobytes()
    rc, back = orc.decompress(s, n, dt, B)
    assert rc == 0 and np.array_equal(back.view(np.uint8), full.view(np.uint8))
    out = bs.decompress(c.buf, c.nbytes, n, es, B, offsets=c.offsets)
    assert np.array_equal(host_bytes(out), full.view(np.uint8))
    # the matches were found: the stream is well below the input
    assert c.nbytes < 0.97 * full.nbytes


def test_ratio_close_to_oracle(bs, orc):
    """Compression ratio of the GPU encoder beside the oracle's greedy one on a
    rounded visibility cube (reported; the GPU must stay within 10 %)."""
    cfg = synth.CONFIG_SMALL
    vis = synth.visibilities(cfg)
    r = orc.reduce_precision_c64(vis, cfg.n_samp, cfg.f)
    d = torch.from_numpy(r.view(np.float32).reshape(-1).copy()).cuda()
    c = bs.compress(d, 2048)
    o = orc.compress(r.view(np.float32).reshape(-1), 2048)
    g_ratio, o_ratio = c.nbytes / r.nbytes, len(o) / r.nbytes
    print(f"ratio gpu {g_ratio:.4f} oracle {o_ratio:.4f}")
    assert g_ratio < 1.10 * o_ratio


# -------------------------------------------------------- fused vis path --

@pytest.mark.parametrize("name,cfg", VIS_CASES, ids=[c[0] for c in VIS_CASES])
@pytest.mark.parametrize("B,level", [(2048, 0), (1024, 0), (0, 0), (2048, 1)])
def test_compress_vis_matches_oracle(bs, orc, name, cfg, B, level):
    vis = synth.visibilities(cfg)
    rounded = orc.reduce_precision_c64(vis, cfg.n_samp, cfg.f)
    flat = rounded.view(np.float32).reshape(-1)
    d = torch.from_numpy(vis.copy()).cuda()
    c = bs.compress_vis(d, cfg.n_samp, cfg.f, B, level=level)
    assert bs.status(c.ws) == 0
    s = c.buf[:c.nbytes].cpu().numpy().tobytes()
    rc, back = orc.decompress(s, flat.size, np.float32, B)
    assert rc == 0 and np.array_equal(back.view(np.uint32), flat.view(np.uint32))
    out = bs.decompress(c.buf, c.nbytes, flat.size, 4, B, offsets=c.offsets)
    assert np.array_equal(host_bytes(out), flat.view(np.uint8))
    # the fused stream equals compress() of the GPU-rounded cube
    rd = bs.reduce_precision_c64(d, cfg.n_samp, cfg.f)
    c2 = bs.compress(rd.view(torch.float32).reshape(-1), B, level=level)
    assert c2.nbytes == c.nbytes and torch.equal(c2.buf[:c.nbytes], c.buf[:c.nbytes])


# ------------------------------------------------------------- corruption --

@pytest.mark.parametrize("es,B", [(4, 1024), (1, 2048), (2, 8192), (4, 8192)])
def test_corrupt_streams_report_status(bs, orc, es, B):
    """Corrupt streams give CORRUPT and never a fault, in the 8 KiB in-place
    decoder (4-byte elements) and in the in-place decoder for other shapes
    (1-byte elements, 16 and 32 KiB blocks)."""
    dt = {1: np.uint8, 2: np.uint16, 4: np.int32}[es]
    a = synth.random_walk(B * 5 + 3, dt, seed=1)
    d = to_dev(a)
    c = bs.compress(d, B, elem_size=es)
    n, nbytes = a.size, c.nbytes
    good = c.buf[:nbytes].clone()
    ws = bs.new_workspace(bs.workspace_size(bs.OP_DECOMPRESS, n, es, B))
    cases = []
    t = good.clone(); t[3] ^= 1; cases.append((t, nbytes, "header"))
    cases.append((good.clone(), nbytes - 1, "truncated"))
    cases.append((torch.cat([good, torch.zeros(16, dtype=torch.uint8, device="cuda")]),
                  nbytes + 1, "trailing"))
    t = good.clone(); t[12] = 0xFF; cases.append((t, nbytes, "length field"))
    for buf, L, what in cases:
        for offs in (None, c.offsets):
            bs.decompress(buf, L, n, es, B, offsets=offs, ws=ws)
            assert bs.status(ws) == bs.ERR_CORRUPT, what
    # random byte flips: never a fault; status is OK or CORRUPT
    rng = np.random.default_rng(3)
    for _ in range(40):
        t = good.clone()
        k = int(rng.integers(12, nbytes))
        t[k] ^= int(rng.integers(1, 256))
        bs.decompress(t, nbytes, n, es, B, offsets=c.offsets, ws=ws)
        assert bs.status(ws) in (0, bs.ERR_CORRUPT)
    # the good stream still decodes with the same workspace
    out = bs.decompress(good, nbytes, n, es, B, offsets=c.offsets, ws=ws)
    assert bs.status(ws) == 0 and np.array_equal(host_bytes(out), a.view(np.uint8))


def test_argument_errors(bs):
    d = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(bs.BsgpuError):
        bs.compress(d, 12)
    with pytest.raises(bs.BsgpuError):
        bs.compress(d, 0, elem_size=3)
    small = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(bs.BsgpuError) as e:
        bs.compress(d, 0, out=small)
    assert e.value.code == bs.ERR_SPACE


# ------------------------------------------------ full CHIME-shaped size --

def _substream(buf: np.ndarray, offs: np.ndarray, b0: int, b1: int, block_bytes: int) -> bytes:
    """The framed stream (reading R11) of blocks b0 .. b1-1 of a stream whose
    block index is `offs`: a header for their bytes, then their length fields
    and LZ4 blocks as they stand."""
    head = ((b1 - b0) * block_bytes).to_bytes(8, "big") + block_bytes.to_bytes(4, "big")
    end = int(offs[b1]) if b1 < offs.size else None
    return head + buf[int(offs[b0]):end].tobytes()


@pytest.mark.parametrize("f", [1e-3, 0.01, 0.1])
def test_chime_full_size_all_slabs(bs, orc, f):
    """1024 freq x 8256 products x 16 time (1.08 GB) in the launch the benchmark
    times, against the oracle over the whole cube: every frequency slab is
    rounded independently (Sec. 3.1: the noise of a sample depends on its own
    frequency's autos), so the host cores take one slab each.  For every slab
    the GPU round trip equals the oracle's rounding bit for bit, and the
    slab's 129 blocks of the GPU stream, framed on their own, decode with the
    oracle's strict decoder to the same bytes.  The compression ratios of the
    GPU encoder and of the oracle's greedy encoder are printed side by side."""
    import concurrent.futures as cf
    import os
    cfg = synth.VisConfig(1024, 128, 16, 2 ** 17, f, seed=0, drift=True)
    vis = _chime_cube(cfg)
    d = torch.from_numpy(vis).cuda()
    n_fl = vis.size * 2
    c = bs.compress_vis(d, cfg.n_samp, f, 2048)
    assert bs.status(c.ws) == 0
    out = bs.decompress(c.buf, c.nbytes, n_fl, 4, 2048, offsets=c.offsets)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    buf = c.buf[:c.nbytes].cpu().numpy()
    offs = c.offsets.cpu().numpy()
    slab = 8256 * 16 * 8
    per = slab // 8192                       # 129 blocks of 8 KiB per slab

    def check(fr):
        want = orc.reduce_precision_c64(vis[fr:fr + 1], cfg.n_samp, f)
        wb = want.view(np.uint8).reshape(-1)
        ok = np.array_equal(got[fr * slab:(fr + 1) * slab], wb)
        rc, back = orc.decompress(_substream(buf, offs, fr * per, (fr + 1) * per, 8192),
                                  slab // 4, np.float32, 2048)
        ok = ok and rc == 0 and np.array_equal(back.view(np.uint8), wb)
        return ok, orc.compress(want.view(np.float32).reshape(-1), 2048)[12:]

    with cf.ThreadPoolExecutor(max_workers=max(1, len(os.sched_getaffinity(0)))) as ex:
        res = list(ex.map(check, range(1024)))
    bad = [fr for fr, (ok, _) in enumerate(res) if not ok]
    assert not bad, f"slabs differing from the oracle: {bad[:10]}"
    orc_bytes = 12 + sum(len(b) for _, b in res)
    # both whole-cube streams decode on the GPU without their block index
    # (recovered on the device from the chain of length fields)
    whole = vis.nbytes.to_bytes(8, "big") + (8192).to_bytes(4, "big") + b"".join(b for _, b in res)
    od = torch.frombuffer(bytearray(whole), dtype=torch.uint8).cuda()
    for st in (c.buf[:c.nbytes], od):
        ws = bs.new_workspace(bs.workspace_size(bs.OP_DECOMPRESS, n_fl, 4, 2048))
        o2 = bs.decompress(st, st.numel(), n_fl, 4, 2048, offsets=None, ws=ws)
        assert bs.status(ws) == 0 and np.array_equal(o2.cpu().numpy(), got)
    print(f"f={f}: ratio gpu {c.nbytes / vis.nbytes:.4f} oracle {orc_bytes / vis.nbytes:.4f}")
    assert c.nbytes < 1.15 * orc_bytes


_CUBE = {}


def _chime_cube(cfg):
    key = (cfg.seed,)
    if key not in _CUBE:
        _CUBE.clear()
        _CUBE[key] = synth.visibilities(cfg)
    return _CUBE[key]
