"""The batch planner (bsgpu_batch_plan) is host code: its table image, item
counts and argument checks are tested here without a GPU (the pointers are
never dereferenced)."""
import ctypes

import numpy as np
import pytest

bs = pytest.importorskip("paper_1503_00638_gb300.bsgpu")

REC = np.dtype([("in", "<u8"), ("out", "<u8"), ("n_elem", "<u8"), ("in_bytes", "<u8"),
                ("out_cap", "<u8"), ("item0", "<u8"), ("es", "<u4"), ("B", "<u4"),
                ("nb", "<u4"), ("last_B", "<u4"), ("tail", "<u4"), ("pad", "<u4"),
                ("offs", "<u8")])
BASE = 1 << 40  # fake, 16-byte aligned device addresses


def chunk(n, es, B=0, cap=None, k=0, in_bytes=0):
    cap = bs.compress_bound(n, es, B) if cap is None else cap
    return bs.Chunk(BASE + (k << 28), BASE + (k << 28) + (1 << 27), n, in_bytes, cap, es, B)


def blocks(n, es, B):
    B = B or 4096 // es
    full, rem = divmod(n, B)
    last = rem - rem % 8
    return full + (1 if last else 0), (last or B), rem % 8, B


def test_table_layout_and_items():
    specs = [(0, 4, 0), (5, 8, 0), (8, 1, 8), (4099, 2, 0), (100000, 4, 2048), (1000, 8, 1024),
             (77, 1, 24)]
    ch = [chunk(n, es, B, k=i) for i, (n, es, B) in enumerate(specs)]
    ch[3].block_offsets = BASE + (1 << 30)
    table, n_items, ws = bs.batch_plan(bs.OP_COMPRESS, ch)
    n = len(specs)
    assert bs.batch_table_bytes(n) == (80 * n + 8 * (n + 1) + 15) // 16 * 16
    rec = np.frombuffer(table.numpy().tobytes()[:80 * n], dtype=REC)
    starts = np.frombuffer(table.numpy().tobytes()[80 * n:80 * n + 8 * (n + 1)], dtype="<u8")
    item = 0
    for i, (nel, es, B) in enumerate(specs):
        nb, last_B, tail, Bf = blocks(nel, es, B)
        r = rec[i]
        assert (r["n_elem"], r["es"], r["B"], r["nb"], r["last_B"], r["tail"]) == \
            (nel, es, Bf, nb, last_B, tail)
        assert r["in"] == ch[i].in_ptr and r["out"] == ch[i].out_ptr
        assert r["offs"] == (ch[i].block_offsets or 0)
        assert r["item0"] == item == starts[i]
        item += max(nb, 1)
    assert starts[n] == item == n_items
    # status word + counter, look-back state per item, two staging slots per warp
    assert ws >= 256 + 8 * n_items + 2 * 8304 * 2560


def test_decompress_plan_workspace():
    ch = [chunk(100000, 4, 0, in_bytes=5000), chunk(3, 2, 0, in_bytes=18, k=1)]
    _, n_items, ws = bs.batch_plan(bs.OP_DECOMPRESS, ch)
    assert n_items == blocks(100000, 4, 0)[0] + 1 == 99 and ws >= 256 + 8 * n_items


def _plan_rc(op, chunks, table_bytes=None):
    n = len(chunks)
    arr = (bs.Chunk * n)(*chunks)
    tb = bs.batch_table_bytes(n) if table_bytes is None else table_bytes
    buf = (ctypes.c_uint8 * max(tb, 1))()
    ni, ws = ctypes.c_uint64(0), ctypes.c_size_t(0)
    return bs._lib.bsgpu_batch_plan(op, ctypes.cast(arr, ctypes.c_void_p), n,
                                    ctypes.cast(buf, ctypes.c_void_p), tb,
                                    ctypes.byref(ni), ctypes.byref(ws))


def test_plan_argument_errors():
    ok = chunk(1000, 4)
    assert _plan_rc(bs.OP_COMPRESS, [ok]) == bs.OK
    assert _plan_rc(7, [ok]) == bs.ERR_ARG
    assert _plan_rc(bs.OP_COMPRESS, [chunk(1000, 3)]) == bs.ERR_ARG             # element size
    assert _plan_rc(bs.OP_COMPRESS, [chunk(1000, 4, 12)]) == bs.ERR_ARG         # not a multiple of 8
    assert _plan_rc(bs.OP_COMPRESS, [chunk(1000, 4, 2056)]) == bs.ERR_ARG       # > 8192 bytes
    assert _plan_rc(bs.OP_COMPRESS, [chunk(1000, 8, 1024)]) == bs.OK            # = 8192 bytes
    assert _plan_rc(bs.OP_COMPRESS, [chunk(1000, 4, cap=100)]) == bs.ERR_SPACE  # out_cap
    assert _plan_rc(bs.OP_COMPRESS, [ok], table_bytes=50) == bs.ERR_SPACE
    bad = chunk(1000, 4)
    bad.in_ptr = BASE + 8
    assert _plan_rc(bs.OP_COMPRESS, [bad]) == bs.ERR_ALIGN
    mis = chunk(1000, 4)
    mis.block_offsets = BASE + 4
    assert _plan_rc(bs.OP_COMPRESS, [mis]) == bs.ERR_ALIGN                     # index alignment
    nul = chunk(1000, 4)
    nul.out_ptr = None
    assert _plan_rc(bs.OP_COMPRESS, [nul]) == bs.ERR_ARG
    # an empty chunk needs no input pointer
    empty = chunk(0, 4)
    empty.in_ptr = None
    assert _plan_rc(bs.OP_COMPRESS, [empty]) == bs.OK
