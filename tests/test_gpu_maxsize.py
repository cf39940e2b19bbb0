"""The largest cube the visibility entry points take: complex indices are
32-bit, so a cube must hold fewer than 2^32 complex samples.  256 freq x
8256 products (128 inputs) x 2032 time is 4,294,705,152 samples (34.4 GB),
just below the limit: the fused compress (Sec. 6 steps 1-5) and the
decompress run at that size, the last frequency slab (the highest indices)
round-trips to the oracle's rounding bit for bit, and the last blocks of the
stream decode with the oracle's block decoder.  One sample more per time
step is refused with BSGPU_ERR_ARG before anything is launched."""
import numpy as np
import pytest
import torch

from paper_1503_00638_gb300 import synth

pytestmark = pytest.mark.gpu

F, N_IN, T = 256, 128, 2032
P = N_IN * (N_IN + 1) // 2
SLAB = 8   # frequencies generated at a time


@pytest.fixture(scope="module")
def bs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if torch.cuda.get_device_properties(0).total_memory < 160 * 2 ** 30:
        pytest.skip("needs about 110 GB of device memory")
    from paper_1503_00638_gb300 import build
    build.build()
    from paper_1503_00638_gb300 import bsgpu
    return bsgpu


def test_cube_just_below_the_index_limit(bs, orc):
    assert F * P * T < 2 ** 32 < F * P * (T + 16)
    f, N = 0.01, 2.0 ** 17
    d = torch.empty((F, P, T), dtype=torch.complex64, device="cuda")
    for f0 in range(0, F, SLAB):
        cfg = synth.VisConfig(SLAB, N_IN, T, N, f, seed=1000 + f0, drift=True)
        d[f0:f0 + SLAB] = synth.visibilities_torch(cfg)
        torch.cuda.empty_cache()
    n_fl = F * P * T * 2
    c = bs.compress_vis(d, N, f, 2048)
    assert bs.status(c.ws) == 0
    out = bs.decompress(c.buf, c.nbytes, n_fl, 4, 2048, offsets=c.offsets)
    torch.cuda.synchronize()
    # the last frequency slab against the oracle
    last = d[F - 1:F].cpu().numpy()
    want = orc.reduce_precision_c64(last, N, f).view(np.uint8).reshape(-1)
    slab_bytes = P * T * 8
    got = out[(F - 1) * slab_bytes:].cpu().numpy()
    assert np.array_equal(got, want)
    # the stream's last blocks through the oracle's block decoder
    nb = n_fl // 2048
    assert c.offsets.numel() >= nb
    offs = c.offsets[nb - 3:nb].cpu().numpy()
    tail = want[-3 * 8192:]
    for k, b in enumerate(range(nb - 3, nb)):
        o = int(offs[k])
        clen = int.from_bytes(c.buf[o:o + 4].cpu().numpy().tobytes(), "big")
        blk = c.buf[o + 4:o + 4 + clen].cpu().numpy().tobytes()
        rc, shuf = orc.lz4_decompress_block(blk, 8192)
        assert rc == 0
        plain = orc.bitunshuffle(np.frombuffer(shuf, dtype=np.uint32).copy(), 2048)
        assert np.array_equal(plain.view(np.uint8), tail[k * 8192:(k + 1) * 8192])
    assert c.nbytes == int(offs[-1]) + 4 + clen
    del d, out, c
    torch.cuda.empty_cache()


def test_one_more_time_step_is_refused(bs):
    # the size check comes before the workspace and the launch, so a small
    # buffer standing in for the cube is never touched
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = bs._lib.bsgpu_compress_vis_ex(x.data_ptr(), bs.VIS_F32, F, N_IN, T + 16, 2.0 ** 17, 0.01,
                                       0, 4, 2048, 0, x.data_ptr(), x.numel(), nb.data_ptr(),
                                       None, x.data_ptr(), x.numel(), None)
    assert rc == bs.ERR_ARG
