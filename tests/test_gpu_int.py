"""GPU parity of the integer path and the compensated f (Sec. 3.2) through the
C-ABI, against the oracle:

* bsgpu_reduce_precision_ex: bit-exact int32 / float32 results, with and
  without the compensated f;
* bsgpu_compress_vis_ex: the GPU stream, read by the oracle's strict decoder,
  equals the oracle's rounded cube byte for byte, for 4-byte components and
  8-byte (re, im) elements, through the fast kernel (full blocks of at most
  8 KiB) and the general one (other block sizes, a shortened last block, the
  verbatim tail).
"""
import numpy as np
import pytest
import torch

from paper_1503_00638_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00638_gb300 import build
    build.build()
    from paper_1503_00638_gb300 import bsgpu
    return bsgpu


# (name, cube config, int scale): scales put the noise granularity at a few
# to a few hundred counts; 2^22 brings the autos near the int32 limit
INT_CASES = [
    ("small", synth.CONFIG_SMALL, 4096.0),
    ("one-input", synth.VisConfig(3, 1, 5, 2 ** 10, 0.05, seed=2), 300.0),
    ("T1", synth.VisConfig(4, 7, 1, 2 ** 12, 0.01, seed=3), 5e4),
    ("T3", synth.VisConfig(5, 9, 3, 2 ** 14, 0.1, seed=4), 2.0 ** 20),
    ("T40", synth.VisConfig(2, 12, 40, 2 ** 16, 1e-3, seed=5), 1e3),
    ("chime-slab", synth.VisConfig(4, 128, 16, 2 ** 17, 0.01, seed=6, drift=True), 2.0 ** 22),
]


def cube(cfg, dtype, scale):
    if dtype == "i32":
        return synth.visibilities_int(cfg, scale)
    return synth.visibilities(cfg)


def as_u32(a):
    return np.ascontiguousarray(a).view(np.uint32).reshape(-1)


@pytest.mark.parametrize("name,cfg,scale", INT_CASES, ids=[c[0] for c in INT_CASES])
@pytest.mark.parametrize("dtype", ["i32", "f32"])
@pytest.mark.parametrize("compensate", [False, True])
def test_reduce_precision_ex_bit_exact(bs, orc, name, cfg, scale, dtype, compensate):
    vis = cube(cfg, dtype, scale)
    want = orc.reduce_precision(vis, cfg.n_samp, cfg.f, compensate)
    got = bs.reduce_precision(torch.from_numpy(vis.copy()).cuda(), cfg.n_samp, cfg.f,
                              compensate).cpu().numpy()
    assert np.array_equal(as_u32(got), as_u32(want))
    if dtype == "i32" and cfg.n_inputs > 1 and scale >= 4096:
        assert not np.array_equal(as_u32(got), as_u32(vis))  # rounding took place


def test_reduce_precision_ex_defaults_equal_c64(bs):
    cfg = synth.VisConfig(3, 10, 32, 2 ** 14, 0.05, seed=9)
    d = torch.from_numpy(synth.visibilities(cfg)).cuda()
    a = bs.reduce_precision_c64(d, cfg.n_samp, cfg.f)
    b = bs.reduce_precision(d, cfg.n_samp, cfg.f)
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_compensation_lowers_granularity(bs, orc):
    # strongly correlated inputs (rho near 1) leave little room: compensated
    # rounding is never coarser than plain rounding, and finer somewhere
    cfg = synth.VisConfig(2, 6, 16, 2 ** 12, 0.1, seed=11, rho=0.95)
    vis = synth.visibilities_int(cfg, 2.0 ** 16)
    d = torch.from_numpy(vis.copy()).cuda()
    plain = bs.reduce_precision(d, cfg.n_samp, cfg.f).cpu().numpy().astype(np.int64)
    comp = bs.reduce_precision(d, cfg.n_samp, cfg.f, True).cpu().numpy().astype(np.int64)
    x = vis.astype(np.int64)
    e_plain, e_comp = np.abs(plain - x), np.abs(comp - x)
    assert e_comp.sum() < e_plain.sum()


# (cube, dtype, scale, elem_size, block_elems, level, compensate)
STREAM_CASES = [
    ("small", "i32", 4096.0, 4, 2048, 0, False),   # fast kernel, 4-byte components
    ("small", "i32", 4096.0, 4, 2048, 0, True),
    ("small", "i32", 4096.0, 8, 1024, 0, False),   # fast kernel, 8-byte samples
    ("small", "f32", 0.0, 8, 1024, 0, True),
    ("small", "f32", 0.0, 8, 0, 1, False),         # default block, hash matches
    ("small", "i32", 4096.0, 4, 0, 1, True),
    ("T3", "i32", 2.0 ** 20, 4, 2048, 0, True),    # n_time % 16 != 0: general kernel
    ("T3", "i32", 2.0 ** 20, 8, 1024, 0, False),   # odd n_time, fast 8-byte kernel
    ("T40", "f32", 0.0, 8, 96, 0, True),           # general kernel, many small blocks
    ("T40", "i32", 1e3, 4, 520, 1, False),
    ("one-input", "i32", 300.0, 8, 8, 0, True),    # 15 samples: blocks of 8 + tail
    ("T1", "f32", 0.0, 8, 2048, 0, False),         # 28 samples: one short block + tail
    ("chime-slab", "i32", 2.0 ** 22, 4, 2048, 0, True),
    ("chime-slab", "i32", 2.0 ** 22, 8, 1024, 0, True),
]
CFG = {c[0]: c[1] for c in INT_CASES}


@pytest.mark.parametrize("case", STREAM_CASES, ids=lambda c: "-".join(map(str, c)))
def test_compress_vis_ex_matches_oracle(bs, orc, case):
    name, dtype, scale, es, B, level, comp = case
    cfg = CFG[name]
    vis = cube(cfg, dtype, scale)
    rounded = orc.reduce_precision(vis, cfg.n_samp, cfg.f, comp)
    flat = np.ascontiguousarray(rounded).view(np.uint32 if es == 4 else np.uint64).reshape(-1)
    d = torch.from_numpy(vis.copy()).cuda()
    c = bs.compress_vis_ex(d, cfg.n_samp, cfg.f, comp, es, B, level=level)
    assert bs.status(c.ws) == 0
    s = c.buf[:c.nbytes].cpu().numpy().tobytes()
    rc, back = orc.decompress(s, flat.size, flat.dtype, B)
    assert rc == 0 and np.array_equal(back, flat)
    out = bs.decompress(c.buf, c.nbytes, flat.size, es, B, offsets=c.offsets)
    assert np.array_equal(out.cpu().numpy(), flat.view(np.uint8))
    # the fused stream equals compress() of the GPU-rounded cube
    rd = bs.reduce_precision(d, cfg.n_samp, cfg.f, comp)
    c2 = bs.compress(rd.view(torch.uint8).reshape(-1), B, elem_size=es, level=level)
    assert c2.nbytes == c.nbytes and torch.equal(c2.buf[:c.nbytes], c.buf[:c.nbytes])


def test_compress_vis_ex_defaults_equal_compress_vis(bs):
    cfg = synth.CONFIG_SMALL
    d = torch.from_numpy(synth.visibilities(cfg)).cuda()
    a = bs.compress_vis(d, cfg.n_samp, cfg.f, 2048)
    b = bs.compress_vis_ex(d, cfg.n_samp, cfg.f, False, 4, 2048)
    assert a.nbytes == b.nbytes and torch.equal(a.buf[:a.nbytes], b.buf[:b.nbytes])


def test_ex_argument_errors(bs):
    import ctypes
    lib = ctypes.CDLL(bs.library_path())
    lib.bsgpu_reduce_precision_ex.argtypes = bs._SIGS["bsgpu_reduce_precision_ex"][0]
    lib.bsgpu_compress_vis_ex.argtypes = bs._SIGS["bsgpu_compress_vis_ex"][0]
    d = torch.zeros((2, 3, 16, 2), dtype=torch.int32, device="cuda")
    o = torch.empty_like(d)
    ws = bs.new_workspace(1 << 20)
    p, q, w = d.data_ptr(), o.data_ptr(), ws.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    rp = lib.bsgpu_reduce_precision_ex
    assert rp(p, q, 2, 2, 2, 16, 1e3, 0.1, 0, w, ws.numel(), s) == bs.ERR_ARG      # dtype
    assert rp(p, q, 1, 2, 2, 16, 1e3, 0.1, 8, w, ws.numel(), s) == bs.ERR_ARG      # flags
    assert rp(p, q, 1, 2, 2, 16, 1e3, 0.1, 1, w, 64, s) == bs.ERR_SPACE            # workspace
    cap = 1 << 16
    buf = torch.empty(cap, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    cv = lib.bsgpu_compress_vis_ex
    for es in (1, 2, 16):
        assert cv(p, 1, 2, 2, 16, 1e3, 0.1, 0, es, 0, 0, buf.data_ptr(), cap, nb.data_ptr(),
                  None, w, ws.numel(), s) == bs.ERR_ARG
    assert bs.vis_workspace_size_ex(bs.OP_COMPRESS_VIS, 2, 2, 16, 2) == 0
    assert (bs.vis_workspace_size_ex(bs.OP_REDUCE_PRECISION, 2, 2, 16, flags=1)
            > bs.vis_workspace_size_ex(bs.OP_REDUCE_PRECISION, 2, 2, 16))
    torch.cuda.synchronize()
