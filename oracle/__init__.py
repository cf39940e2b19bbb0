"""Plain CPU oracle for the compression scheme of arXiv:1503.00638.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs are the only callers.
The product path (``paper_1503_00638_gb300``) never imports this package and
shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, one element or bit at a time);
this module compiles it with gcc and wraps it with ctypes and numpy.  Each
function names the passage of the paper it follows:

* ``rad_simple_var``       -- Sec. 3.1, Eq. rad_simple (diagonal), Eq. noise
* ``rad_full_cov``         -- Sec. 3.1, Eq. rad_full1-3
* ``q32``                  -- Sec. 3.2, Eq. trunc_error as q = 12 f s^2 (reading R1)
* ``granularity_exponent`` -- Sec. 3.2, Eq. trunc_error: largest 2^k < sqrt(q)
* ``round_pow2``           -- Sec. 3.2: round to a multiple of 2^k, ties to even
* ``reduce_precision_c64`` -- Sec. 6 steps 1-3 on a visibility cube
* ``bitshuffle`` / ``bitunshuffle`` -- Sec. 4.2, Sec. 6 step 4 (bit transpose per block)
* ``lz4_compress_block`` / ``lz4_decompress_block`` -- Sec. 4.1 / Sec. 6 step 5
* ``compress`` / ``decompress`` -- Sec. 4.2.1 blocking with the framing of reading R11

Parity is pinned by ``tests/test_oracle_*.py`` against closed forms, brute
force, Python's exact rational arithmetic, numpy's bit routines, hand-built
LZ4 streams written out from the LZ4 block format (``tests/test_oracle_lz4.py``)
and (where present) the system liblz4.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/lib/liboracle.so (gcc -O2 -ffp-contract=off)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
             "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            c_sz, c_vp, c_d, c_f, c_i, c_l = (ctypes.c_size_t, ctypes.c_void_p, ctypes.c_double,
                                              ctypes.c_float, ctypes.c_int, ctypes.c_long)
            L.orc_rad_simple_var.argtypes = [c_i, c_i, c_i, c_d, c_d, c_d]
            L.orc_rad_simple_var.restype = c_d
            L.orc_rad_full_cov.argtypes = [c_vp, c_i, c_i, c_i, c_i, c_i, c_i, c_i, c_d]
            L.orc_rad_full_cov.restype = c_d
            L.orc_q32.argtypes = [c_i, c_f, c_f, c_d, c_d]
            L.orc_q32.restype = c_f
            L.orc_granularity_exponent.argtypes = [c_f, ctypes.POINTER(c_i)]
            L.orc_granularity_exponent.restype = c_i
            L.orc_round_pow2.argtypes = [c_f, c_i]
            L.orc_round_pow2.restype = c_f
            L.orc_round_element.argtypes = [c_f, c_f]
            L.orc_round_element.restype = c_f
            L.orc_reduce_precision_c64.argtypes = [c_vp, c_vp, c_l, c_l, c_l, c_d, c_d]
            L.orc_reduce_precision_c64.restype = None
            L.orc_granularity_map_c64.argtypes = [c_vp, c_vp, c_l, c_l, c_l, c_d, c_d]
            L.orc_granularity_map_c64.restype = None
            L.orc_round_int.argtypes = [ctypes.c_int32, c_i]
            L.orc_round_int.restype = ctypes.c_int32
            L.orc_compensation_min.argtypes = [c_vp, c_i, c_l, c_l, c_l, c_l, c_l]
            L.orc_compensation_min.restype = c_f
            L.orc_reduce_precision.argtypes = [c_vp, c_vp, c_i, c_l, c_l, c_l, c_d, c_d, c_i]
            L.orc_reduce_precision.restype = None
            L.orc_full_index.argtypes = [c_l, c_i, c_i, c_i]
            L.orc_full_index.restype = c_l
            L.orc_full_cov_matrix.argtypes = [c_vp, c_i, c_d, c_vp]
            L.orc_full_cov_matrix.restype = None
            L.orc_invert_spd.argtypes = [c_vp, c_l, c_vp]
            L.orc_invert_spd.restype = c_i
            L.orc_full_noise_var.argtypes = [c_vp, c_i, c_d, c_vp]
            L.orc_full_noise_var.restype = c_i
            L.orc_reduce_precision_full.argtypes = [c_vp, c_vp, c_i, c_l, c_l, c_l, c_d, c_d]
            L.orc_reduce_precision_full.restype = None
            L.orc_reorder_time.argtypes = [c_vp, c_vp, c_sz, c_sz, c_sz]
            L.orc_reorder_time.restype = None
            L.orc_bitshuffle.argtypes = [c_vp, c_vp, c_sz, c_sz, c_sz, c_i]
            L.orc_bitshuffle.restype = c_i
            L.orc_lz4_bound.argtypes = [c_sz]
            L.orc_lz4_bound.restype = c_sz
            L.orc_lz4_compress_block.argtypes = [c_vp, c_sz, c_vp, c_sz]
            L.orc_lz4_compress_block.restype = c_sz
            L.orc_lz4_decompress_block.argtypes = [c_vp, c_sz, c_vp, c_sz]
            L.orc_lz4_decompress_block.restype = c_i
            L.orc_compress_bound.argtypes = [c_sz, c_sz, c_sz]
            L.orc_compress_bound.restype = c_sz
            L.orc_compress.argtypes = [c_vp, c_sz, c_sz, c_sz, c_vp, c_sz, c_vp]
            L.orc_compress.restype = c_sz
            L.orc_decompress.argtypes = [c_vp, c_sz, c_vp, c_sz, c_sz, c_sz]
            L.orc_decompress.restype = c_i
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# -- Sec. 3.1 ---------------------------------------------------------------

def rad_simple_var(i: int, j: int, alpha: int, Vii: float, Vjj: float, N: float) -> float:
    """Eq. rad_simple on its diagonal; alpha 0 = Re, 1 = Im."""
    return lib().orc_rad_simple_var(i, j, alpha, Vii, Vjj, N)


def rad_full_cov(V: np.ndarray, alpha: int, i: int, j: int, beta: int, g: int, h: int,
                 N: float) -> float:
    """Eq. rad_full1-3: C_{alpha ij, beta gh} from the complex matrix V."""
    Vc = np.ascontiguousarray(V, dtype=np.complex128)
    n = Vc.shape[0]
    return lib().orc_rad_full_cov(_ptr(Vc.view(np.float64)), n, alpha, i, j, beta, g, h, N)


# -- Sec. 3.2 ---------------------------------------------------------------

def q32(is_auto: bool, Ai: float, Aj: float, f: float, N: float) -> np.float32:
    """q = 12 f s^2 in float32 with the operation order of reading R1."""
    return np.float32(lib().orc_q32(int(bool(is_auto)), Ai, Aj, f, N))


def granularity_exponent(q: float):
    """Largest k with 4^k < q (Eq. trunc_error), or None when q is unusable (R2)."""
    k = ctypes.c_int(0)
    ok = lib().orc_granularity_exponent(float(np.float32(q)), ctypes.byref(k))
    return k.value if ok else None


def round_pow2(x: float, k: int) -> np.float32:
    return np.float32(lib().orc_round_pow2(float(np.float32(x)), k))


def round_element(x: float, q: float) -> np.float32:
    return np.float32(lib().orc_round_element(float(np.float32(x)), float(np.float32(q))))


def reduce_precision_c64(vis: np.ndarray, N: float, f: float) -> np.ndarray:
    """Round a [F][P][T] complex64 cube (P = n(n+1)/2) per Sec. 6 steps 1-3."""
    vis = np.ascontiguousarray(vis, dtype=np.complex64)
    F, P, T = vis.shape
    n = _n_inputs(P)
    out = np.empty_like(vis)
    lib().orc_reduce_precision_c64(_ptr(vis), _ptr(out), F, n, T, N, f)
    return out


def round_int(x: int, k: int) -> int:
    """Integer data: nearest multiple of 2^k, ties to even (R17 on overflow)."""
    return int(lib().orc_round_int(int(x), int(k)))


def compensation_min(vis: np.ndarray, fr: int, t: int) -> np.float32:
    """Sec. 3.2: min over crosses of 1 - |V_ij|^2 / (V_ii V_jj) at (fr, t) (R18)."""
    F, P, T, is_int, a = _cube(vis)
    return np.float32(lib().orc_compensation_min(_ptr(a), is_int, F, _n_inputs(P), T, fr, t))


def reduce_precision(vis: np.ndarray, N: float, f: float, compensate: bool = False) -> np.ndarray:
    """Round a [F][P][T] cube of complex64, or of int32 (re, im) pairs given as
    an int32 array of shape [F][P][T][2], per Sec. 6 steps 1-3 (and the
    compensated f of Sec. 3.2 when asked)."""
    F, P, T, is_int, a = _cube(vis)
    out = np.empty_like(a)
    lib().orc_reduce_precision(_ptr(a), _ptr(out), is_int, F, _n_inputs(P), T, N, f,
                               int(bool(compensate)))
    return out


def _cube(vis):
    if vis.dtype == np.int32:
        a = np.ascontiguousarray(vis)
        assert a.ndim == 4 and a.shape[3] == 2
        F, P, T = a.shape[:3]
        return F, P, T, 1, a
    a = np.ascontiguousarray(vis, dtype=np.complex64)
    F, P, T = a.shape
    return F, P, T, 0, a


def granularity_map_c64(vis: np.ndarray, N: float, f: float) -> np.ndarray:
    """k per float of the cube, shape [F][P][T][2]; -1000 marks 'not rounded'."""
    vis = np.ascontiguousarray(vis, dtype=np.complex64)
    F, P, T = vis.shape
    out = np.empty((F, P, T, 2), dtype=np.int32)
    lib().orc_granularity_map_c64(_ptr(vis), _ptr(out), F, _n_inputs(P), T, N, f)
    return out


def _n_inputs(P: int) -> int:
    n = int(round(((8 * P + 1) ** 0.5 - 1) / 2))
    if n * (n + 1) // 2 != P:
        raise ValueError(f"{P} products is not n(n+1)/2")
    return n


# -- Sec. 3.1, full covariance (small arrays) ---------------------------------

def full_index(n: int, i: int, j: int, alpha: int) -> int:
    return lib().orc_full_index(n, i, j, alpha)


def full_cov_matrix(V: np.ndarray, N: float) -> np.ndarray:
    """M x M covariance (Eq. rad_full1-3) of the n^2 components of one sample."""
    V = np.ascontiguousarray(V, dtype=np.complex128)
    n = V.shape[0]
    C = np.empty((n * n, n * n))
    lib().orc_full_cov_matrix(_ptr(V), n, N, _ptr(C))
    return C


def invert_spd(A: np.ndarray):
    A = np.array(A, dtype=np.float64, order="C")
    out = np.empty_like(A)
    rc = lib().orc_invert_spd(_ptr(A), A.shape[0], _ptr(out))
    return rc, out


def full_noise_var(V: np.ndarray, N: float):
    """(rc, s^2 per component) of Eq. noise with the full covariance."""
    V = np.ascontiguousarray(V, dtype=np.complex128)
    n = V.shape[0]
    s2 = np.empty(n * n)
    rc = lib().orc_full_noise_var(_ptr(V), n, N, _ptr(s2))
    return rc, s2


def reduce_precision_full(vis: np.ndarray, N: float, f: float) -> np.ndarray:
    F, P, T, is_int, a = _cube(vis)
    out = np.empty_like(a)
    lib().orc_reduce_precision_full(_ptr(a), _ptr(out), is_int, F, _n_inputs(P), T, N, f)
    return out


# -- Sec. 2 ------------------------------------------------------------------

def reorder_time(a: np.ndarray) -> np.ndarray:
    """[T][...] (time slowest) -> [...][T] (time fastest) by plain loops."""
    a = np.ascontiguousarray(a)
    T = a.shape[0]
    S = a.size // T if T else 0
    out = np.empty(a.shape[1:] + (T,), dtype=a.dtype)
    lib().orc_reorder_time(_ptr(a), _ptr(out), T, S, a.itemsize)
    return out


# -- Sec. 4.2 ---------------------------------------------------------------

def bitshuffle(a: np.ndarray, block_elems: int = 0) -> np.ndarray:
    """Blocked bit transpose of a 1-D array of 1/2/4/8-byte elements (R9 tail)."""
    a = np.ascontiguousarray(a)
    out = np.empty_like(a)
    rc = lib().orc_bitshuffle(_ptr(a), _ptr(out), a.size, a.itemsize, block_elems, 0)
    if rc:
        raise ValueError("bad element size or block size")
    return out


def bitunshuffle(a: np.ndarray, block_elems: int = 0) -> np.ndarray:
    a = np.ascontiguousarray(a)
    out = np.empty_like(a)
    rc = lib().orc_bitshuffle(_ptr(a), _ptr(out), a.size, a.itemsize, block_elems, 1)
    if rc:
        raise ValueError("bad element size or block size")
    return out


# -- Sec. 4.1 ---------------------------------------------------------------

def lz4_bound(n: int) -> int:
    return lib().orc_lz4_bound(n)


def lz4_compress_block(data: bytes) -> bytes:
    src = np.frombuffer(bytes(data), dtype=np.uint8).copy()
    cap = lz4_bound(src.size)
    dst = np.empty(max(cap, 1), dtype=np.uint8)
    c = lib().orc_lz4_compress_block(_ptr(src) if src.size else 0, src.size, _ptr(dst), cap)
    return dst[:c].tobytes()


def lz4_decompress_block(data: bytes, n: int):
    """Decode one LZ4 block to exactly n bytes; returns (rc, bytes)."""
    src = np.frombuffer(bytes(data), dtype=np.uint8).copy()
    dst = np.zeros(max(n, 1), dtype=np.uint8)
    rc = lib().orc_lz4_decompress_block(_ptr(src) if src.size else 0, src.size, _ptr(dst), n)
    return rc, dst[:n].tobytes()


# -- framing (R11) ----------------------------------------------------------

def compress_bound(n: int, es: int, block_elems: int = 0) -> int:
    return lib().orc_compress_bound(n, es, block_elems)


def compress(a: np.ndarray, block_elems: int = 0, return_block_sizes: bool = False):
    """Bitshuffle + LZ4 every block of a 1-D array; returns the framed stream."""
    a = np.ascontiguousarray(a)
    n, es = a.size, a.itemsize
    cap = compress_bound(n, es, block_elems)
    out = np.empty(cap, dtype=np.uint8)
    B = block_elems or 4096 // es
    nblk = n // B + (1 if (n % B) >= 8 else 0)
    sizes = np.zeros(max(nblk, 1), dtype=np.uint32)
    c = lib().orc_compress(_ptr(a) if n else 0, n, es, block_elems, _ptr(out), cap, _ptr(sizes))
    if c == 0:
        raise ValueError("bad argument")
    if return_block_sizes:
        return out[:c].tobytes(), sizes[:nblk].copy()
    return out[:c].tobytes()


def decompress(stream: bytes, n: int, dtype, block_elems: int = 0):
    """Inverse of compress; returns (rc, array)."""
    src = np.frombuffer(bytes(stream), dtype=np.uint8).copy()
    out = np.zeros(n, dtype=dtype)
    rc = lib().orc_decompress(_ptr(src), src.size, _ptr(out) if n else 0, n,
                              out.itemsize, block_elems)
    return rc, out
