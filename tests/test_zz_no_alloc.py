"""bsgpu_compress_noalloc, the compress entry point for callers that cannot
allocate device memory (filter callbacks handed only their buffers, real-time
loops that may not call cudaMalloc after start-up, pool-owned devices): it
keeps its scratch in a fixed array inside the library instead of a
caller-provided workspace.  Its output must equal bsgpu_compress's, byte for
byte (the encoder is deterministic), on consecutive calls that reuse the
array.  This file is collected last."""

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


def _call_noalloc(bs, d, n, es, B, level):
    cap = bs.compress_bound(n, es, B)
    out = torch.full((cap,), 0xAB, dtype=torch.uint8, device="cuda")
    nbytes = torch.zeros(1, dtype=torch.int64, device="cuda")
    offs = torch.zeros(max(bs.num_blocks(n, es, B), 1), dtype=torch.int64, device="cuda")
    rc = bs._lib.bsgpu_compress_noalloc(d.data_ptr(), n, es, B, level, out.data_ptr(), cap,
                                        nbytes.data_ptr(), offs.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    return out, int(nbytes.item()), offs


@pytest.mark.parametrize("level", [0, 1])
def test_noalloc_matches_compress_on_consecutive_calls(bs, orc, level):
    cfg = synth.CONFIG_SMALL
    rounded = orc.reduce_precision_c64(synth.visibilities(cfg), cfg.n_samp, cfg.f)
    inputs = [(rounded.view(np.float32).reshape(-1), 4, 2048),
              (synth.random_walk(3000 * 8 + 5, np.float64, seed=3), 8, 1024),
              (synth.random_walk(5, np.int32, seed=4), 4, 2048)]      # no block: verbatim
    for a, es, B in inputs:                 # two calls in a row sharing the scratch
        d = torch.from_numpy(a.view(np.uint8).copy()).cuda()
        n = a.size
        ref = bs.compress(d, B, elem_size=es, level=level)
        out, nbytes, offs = _call_noalloc(bs, d, n, es, B, level)
        assert nbytes == ref.nbytes > 12
        assert torch.equal(out[:nbytes], ref.buf[:nbytes])
        nblk = bs.num_blocks(n, es, B)
        assert torch.equal(offs[:nblk], ref.offsets[:nblk])
        rc, back = orc.decompress(out[:nbytes].cpu().numpy().tobytes(), n, a.dtype, B)
        assert rc == 0 and np.array_equal(back.view(np.uint8), a.view(np.uint8))


def test_noalloc_rejects_inputs_beyond_its_scratch(bs):
    n = 131072 * 2048 + 2048          # one block more than the fixed scratch holds
    d = torch.empty(64, dtype=torch.uint8, device="cuda")   # never read: rejected first
    nbytes = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = bs._lib.bsgpu_compress_noalloc(d.data_ptr(), n, 4, 2048, 0, d.data_ptr(),
                                        bs.compress_bound(n, 4, 2048), nbytes.data_ptr(), None,
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == bs.ERR_SPACE


def test_noalloc_reports_a_device_side_failure_as_zero_length(bs, tmp_path):
    """A bounded wait that runs out inside the kernel must show as a zero
    stream length (the call itself returns 0: the failure happens on the
    device, after the call has returned).  A test build of the library makes
    the look-back see predecessors that never publish (a flag nothing sets),
    so block 1 waits out its bounded spin; nothing faults or hangs.  The
    regular library, called afterwards in the same process, still works."""
    import ctypes
    from paper_1503_00638_gb300 import build
    path = build.build(force=True, extra_flags=("-DBSG_TEST_LOOKBACK_STALL",),
                       lib=str(tmp_path / "libbsgpu_stall.so"))
    lib = ctypes.CDLL(path)
    fn = lib.bsgpu_compress_noalloc
    v, z = ctypes.c_void_p, ctypes.c_size_t
    fn.argtypes = [v, z, z, z, ctypes.c_int, v, z, v, v, v]
    fn.restype = ctypes.c_int
    n, es, B = 2 * 2048, 4, 2048                    # two blocks: block 1 looks back
    a = synth.random_walk(n, np.int32, seed=5)
    d = torch.from_numpy(a.view(np.uint8).copy()).cuda()
    cap = bs.compress_bound(n, es, B)
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    nbytes = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
    rc = fn(d.data_ptr(), n, es, B, 0, out.data_ptr(), cap, nbytes.data_ptr(), None,
            torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(nbytes.item()) == 0
    # the context is still usable: the regular entry point gives a full stream
    ref = bs.compress(d, B, elem_size=es, level=0)
    good, nb2, _ = _call_noalloc(bs, d, n, es, B, 0)
    assert nb2 == ref.nbytes > 12 and torch.equal(good[:nb2], ref.buf[:nb2])
