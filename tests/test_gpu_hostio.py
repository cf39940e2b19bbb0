"""GPU test of the host-buffer codec: slabs of a host cube are compressed into
independent framed streams and decompressed back, pipelined over streams; the
round trip returns the oracle's rounded cube and every slab stream decodes
with the oracle's decoder."""
import numpy as np
import pytest
import torch

from paper_1503_00638_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00638_gb300 import build
    build.build()
    from paper_1503_00638_gb300 import bsgpu, hostio
    return bsgpu, hostio


@pytest.mark.parametrize("slab,depth,lag", [(4, 3, 1), (5, 2, 2), (16, 1, 1), (3, 4, 1)])
def test_round_trip_through_host(mods, orc, slab, depth, lag):
    bs, hostio = mods
    cfg = synth.CONFIG_SMALL
    v = synth.visibilities(cfg)
    want = orc.reduce_precision_c64(v, cfg.n_samp, cfg.f)
    h_vis = torch.from_numpy(v.copy()).pin_memory()
    h_out = torch.empty_like(h_vis).pin_memory()
    codec = hostio.HostVisCodec(cfg.n_freq, cfg.n_inputs, cfg.n_time, cfg.n_samp, cfg.f,
                                block_elems=2048, slab_freq=slab, depth=depth)
    chunks = codec.round_trip(h_vis, h_out, lag=lag)
    assert all(c == (0, 0) for c in codec.statuses())
    assert np.array_equal(h_out.numpy().view(np.uint32), want.view(np.uint32))
    for c in chunks:
        f0, f1 = c.freq
        flat = want[f0:f1].view(np.float32).reshape(-1)
        rc, back = orc.decompress(c.stream.numpy().tobytes(), flat.size, np.float32, 2048)
        assert rc == 0 and np.array_equal(back.view(np.uint32), flat.view(np.uint32))
    h2d, d2h = codec.bytes_moved(chunks)
    assert h2d > v.nbytes and d2h > v.nbytes


@pytest.mark.parametrize("cfg", [synth.VisConfig(6, 16, 40, 2 ** 16, 0.01, seed=3),
                                 synth.VisConfig(5, 12, 7, 2 ** 14, 0.03, seed=4)],
                         ids=["T40", "T7"])
def test_round_trip_with_other_time_axes(mods, orc, cfg):
    # time axes that are not a multiple of 16: slabs go through the fast
    # kernel's per-sample rounding; the result is still the oracle's cube
    bs, hostio = mods
    v = synth.visibilities(cfg)
    want = orc.reduce_precision_c64(v, cfg.n_samp, cfg.f)
    h_vis = torch.from_numpy(v.copy()).pin_memory()
    h_out = torch.empty_like(h_vis).pin_memory()
    codec = hostio.HostVisCodec(cfg.n_freq, cfg.n_inputs, cfg.n_time, cfg.n_samp, cfg.f,
                                block_elems=2048, slab_freq=2, depth=2)
    chunks = codec.round_trip(h_vis, h_out, lag=1)
    assert all(c == (0, 0) for c in codec.statuses())
    assert np.array_equal(h_out.numpy().view(np.uint32), want.view(np.uint32))
    for c in chunks:
        f0, f1 = c.freq
        flat = want[f0:f1].view(np.float32).reshape(-1)
        rc, back = orc.decompress(c.stream.numpy().tobytes(), flat.size, np.float32, 2048)
        assert rc == 0 and np.array_equal(back.view(np.uint32), flat.view(np.uint32))


@pytest.mark.parametrize("group_bytes,lag", [(1 << 20, 1), (3 << 20, 2), (64 << 20, 1)])
def test_batch_round_trip_through_host(mods, orc, group_bytes, lag):
    """Chunks of 1-, 2-, 4- and 8-byte elements in pinned host memory go
    through the pipelined batch codec in groups: every output equals its
    input, and every stream read back from host memory decodes with the
    oracle's decoder."""
    bs, hostio = mods
    rng = np.random.default_rng(7)
    arrays, es_l, bl = [], [], []
    for k in range(23):
        es = (1, 2, 4, 8)[k % 4]
        n = int(rng.integers(1000, 300_000)) // es
        dt = {1: np.uint8, 2: np.uint16, 4: np.int32, 8: np.float64}[es]
        arrays.append(synth.random_walk(n, dt, seed=k))
        es_l.append(es)
        bl.append(8192 // es)
    h_in = [torch.from_numpy(a.view(np.uint8).copy()).pin_memory() for a in arrays]
    h_out = [torch.empty_like(h).pin_memory() for h in h_in]
    hb = hostio.HostBatchCodec([h.numel() for h in h_in], es_l, bl, group_bytes=group_bytes)
    assert len(hb.groups) > (1 if group_bytes < (8 << 20) else 0)
    hb.round_trip(h_in, h_out, lag=lag)
    for sc, sd in hb.statuses():
        assert sc == [0] * len(sc) and sd == [0] * len(sd)
    for i in range(len(h_in)):
        assert torch.equal(h_out[i], h_in[i]), i
    for g, (g0, g1) in enumerate(hb.groups):
        for k in range(g1 - g0):
            i = g0 + k
            s = hb.h_streams[g][k][:hb.lens[g][k]].numpy().tobytes()
            rc, back = orc.decompress(s, arrays[i].size, arrays[i].dtype, bl[i])
            assert rc == 0 and np.array_equal(back.view(np.uint8), arrays[i].view(np.uint8))
    h2d, d2h = hb.bytes_moved()
    assert h2d > sum(h.numel() for h in h_in) and d2h > sum(h.numel() for h in h_in)
