"""GPU parity of the post-acquisition reorder (Sec. 2), alone and fused into
the rounding and the compression: bit-exact against the oracle, and the
fused stream equals the stream of the already-reordered cube."""
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


@pytest.mark.parametrize("shape", [(1, 5), (3, 7), (16, 1000), (40, 33), (64, 4096), (1000, 31),
                                   (2, 1)])
@pytest.mark.parametrize("dt", [np.uint8, np.uint16, np.float32, np.complex64])
def test_reorder_alone(bs, orc, shape, dt):
    rng = np.random.default_rng(shape[0] * 7 + shape[1])
    a = rng.integers(0, 1 << 15, size=shape).astype(dt)
    got = bs.reorder_time(torch.from_numpy(a.copy()).cuda()).cpu().numpy()
    assert np.array_equal(got, orc.reorder_time(a))


def test_reorder_empty_and_errors(bs):
    x = torch.zeros((0, 5), dtype=torch.float32, device="cuda")
    assert bs._lib.bsgpu_reorder_time(x.data_ptr(), x.data_ptr(), 0, 5, 4, None) == 0
    y = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert bs._lib.bsgpu_reorder_time(y.data_ptr(), y.data_ptr() + 8, 2, 4, 3, None) == bs.ERR_ARG
    assert bs._lib.bsgpu_reorder_time(y.data_ptr() + 2, y.data_ptr() + 32, 2, 2, 4,
                                      None) == bs.ERR_ALIGN


CASES = [
    ("small", synth.CONFIG_SMALL, 4096.0),
    ("T3", synth.VisConfig(5, 9, 3, 2 ** 14, 0.1, seed=4), 2.0 ** 20),
    ("T40", synth.VisConfig(2, 12, 40, 2 ** 16, 1e-3, seed=5), 1e3),
    ("one-input", synth.VisConfig(3, 1, 5, 2 ** 10, 0.05, seed=2), 300.0),
    ("chime-slab", synth.VisConfig(4, 128, 16, 2 ** 17, 0.01, seed=6, drift=True), 2.0 ** 22),
    # series of 32 and 48 samples: a block holds whole series, or starts and
    # ends inside one (1024 / 48 is not whole), and the cube ends in a short block
    ("T32", synth.VisConfig(3, 10, 32, 2 ** 15, 0.02, seed=7), 2.0 ** 16),
    ("T48", synth.VisConfig(2, 16, 48, 2 ** 16, 0.01, seed=8, drift=True), 2.0 ** 20),
    # an odd time axis with several full blocks (samples gathered and rounded
    # one by one in the fast kernel)
    ("T7", synth.VisConfig(4, 20, 7, 2 ** 14, 0.03, seed=9), 2.0 ** 18),
]


def tslow_of(v):
    return np.ascontiguousarray(np.moveaxis(v, 2, 0))   # [F][P][T](...) -> [T][F][P](...)


@pytest.mark.parametrize("name,cfg,scale", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dtype", ["f32", "i32"])
@pytest.mark.parametrize("compensate", [False, True])
def test_fused_reorder_rounding(bs, orc, name, cfg, scale, dtype, compensate):
    v = synth.visibilities_int(cfg, scale) if dtype == "i32" else synth.visibilities(cfg)
    want = orc.reduce_precision(v, cfg.n_samp, cfg.f, compensate)
    ts = tslow_of(v)
    got = bs.reduce_precision(torch.from_numpy(ts).cuda(), cfg.n_samp, cfg.f, compensate,
                              time_slowest=True).cpu().numpy()
    assert got.shape == want.shape
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("name,dtype,es,B,level,comp", [
    ("small", "f32", 4, 2048, 0, False),
    ("small", "i32", 8, 1024, 0, True),
    ("T3", "i32", 4, 520, 1, False),
    ("T40", "f32", 8, 96, 0, True),
    ("one-input", "i32", 8, 8, 0, False),
    ("chime-slab", "f32", 4, 2048, 0, True),
    ("chime-slab", "i32", 4, 0, 1, False),
    ("small", "f32", 8, 1024, 1, False),
    ("T32", "f32", 4, 2048, 0, False),
    ("T32", "i32", 8, 1024, 1, False),
    ("T48", "f32", 4, 2048, 1, True),
    ("T48", "f32", 8, 1024, 0, False),
    ("T48", "i32", 4, 2048, 0, True),
    ("T48", "f32", 4, 512, 0, False),
    ("T40", "f32", 4, 2048, 0, False),
    ("T40", "i32", 8, 1024, 0, True),
    ("T40", "i32", 4, 1024, 1, True),
    ("T7", "f32", 4, 2048, 0, True),
    ("T7", "i32", 8, 1024, 1, False),
])
def test_fused_reorder_compression(bs, orc, name, dtype, es, B, level, comp):
    cfg, scale = {c[0]: (c[1], c[2]) for c in CASES}[name]
    v = synth.visibilities_int(cfg, scale) if dtype == "i32" else synth.visibilities(cfg)
    rounded = orc.reduce_precision(v, cfg.n_samp, cfg.f, comp)
    flat = np.ascontiguousarray(rounded).view(np.uint32 if es == 4 else np.uint64).reshape(-1)
    dv = torch.from_numpy(tslow_of(v)).cuda()
    c = bs.compress_vis_ex(dv, cfg.n_samp, cfg.f, comp, es, B, level=level, time_slowest=True)
    assert bs.status(c.ws) == 0
    s = c.buf[:c.nbytes].cpu().numpy().tobytes()
    rc, back = orc.decompress(s, flat.size, flat.dtype, B)
    assert rc == 0 and np.array_equal(back, flat)
    # the same bytes as compressing the reordered cube
    ref = bs.compress_vis_ex(torch.from_numpy(v.copy()).cuda(), cfg.n_samp, cfg.f, comp, es, B,
                             level=level)
    assert ref.nbytes == c.nbytes and torch.equal(ref.buf[:ref.nbytes], c.buf[:c.nbytes])
