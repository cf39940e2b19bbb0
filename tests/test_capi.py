"""The C-ABI library loads, exports every entry point include/*.h declares, and
answers the host-only queries (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1503_00638_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(bsgpu_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_bounds_match_oracle(lib, orc):
    lib.bsgpu_compress_bound.restype = ctypes.c_size_t
    lib.bsgpu_compress_bound.argtypes = [ctypes.c_size_t] * 3
    lib.bsgpu_num_blocks.restype = ctypes.c_size_t
    lib.bsgpu_num_blocks.argtypes = [ctypes.c_size_t] * 3
    for n in (0, 1, 7, 8, 9, 100, 4096, 4103, 10 ** 6 + 3):
        for es in (1, 2, 4, 8):
            for B in (0, 8, 512, 2048):
                assert lib.bsgpu_compress_bound(n, es, B) == orc.compress_bound(n, es, B)
                Bb = B or 4096 // es
                want = n // Bb + (1 if n % Bb >= 8 else 0)
                assert lib.bsgpu_num_blocks(n, es, B) == want


def test_argument_errors_on_host(lib):
    f = lib.bsgpu_bitshuffle
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                  ctypes.c_size_t, ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(None, None, 64, 3, 0, None) == -1          # element size
    assert f(None, None, 64, 4, 12, None) == -1         # block not a multiple of 8
    assert f(None, None, 64, 8, 16384, None) == -1      # block over 64 KiB
    assert f(None, None, 64, 4, 0, None) == -1          # null pointers
    assert f(17, 32, 64, 4, 0, None) == -6          # misaligned (checked before any launch)
    lib.bsgpu_compress_bound.restype = ctypes.c_size_t
    lib.bsgpu_compress_bound.argtypes = [ctypes.c_size_t] * 3
    assert lib.bsgpu_compress_bound(10, 3, 0) == 0
    w = lib.bsgpu_vis_workspace_size
    w.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_size_t]
    w.restype = ctypes.c_size_t
    assert w(3, 16, 16, 64, 2048) > 0
    assert w(3, 0, 16, 64, 2048) == 0
    assert w(3, 1 << 20, 1024, 64, 2048) == 0            # complex index over 32 bits


def test_binding_module_imports():
    from paper_1503_00638_gb300 import bsgpu
    assert bsgpu.version().startswith("bsgpu")
    assert bsgpu.num_blocks(270532608, 4, 2048) == 132096
