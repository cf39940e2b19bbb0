"""Thin Python binding of libbsgpu (include/bsgpu.h): argument marshalling only.

Every function here passes device pointers of PyTorch CUDA tensors, the
current CUDA stream and sizes to the C entry point of the same name (without
the ``bsgpu_`` prefix) and raises :class:`BsgpuError` on a nonzero status.
All computation happens in the CUDA kernels of libbsgpu; there is no CPU
fallback: importing this module fails if the library has not been built.
PyTorch provides device memory and streams only.
"""
from __future__ import annotations

import ctypes
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libbsgpu.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with "
                      "`python -m paper_1503_00638_gb300.build` (needs nvcc)")
_lib = ctypes.CDLL(_LIB_PATH)

OK, ERR_ARG, ERR_SPACE, ERR_CORRUPT, ERR_CUDA, ERR_TIMEOUT, ERR_ALIGN = 0, -1, -2, -3, -4, -5, -6
OP_COMPRESS, OP_DECOMPRESS, OP_COMPRESS_VIS, OP_REDUCE_PRECISION = 1, 2, 3, 4
VIS_F32, VIS_I32 = 0, 1
VIS_COMPENSATE = 1
VIS_TIME_SLOWEST = 2
VIS_FULL_COV = 4
_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_SPACE", -3: "ERR_CORRUPT", -4: "ERR_CUDA",
          -5: "ERR_TIMEOUT", -6: "ERR_ALIGN"}

_sz, _vp, _i, _i64, _d = ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "bsgpu_version": ([], ctypes.c_char_p),
    "bsgpu_compress_bound": ([_sz, _sz, _sz], _sz),
    "bsgpu_num_blocks": ([_sz, _sz, _sz], _sz),
    "bsgpu_workspace_size": ([_i, _sz, _sz, _sz], _sz),
    "bsgpu_vis_workspace_size": ([_i, _i64, _i64, _i64, _sz], _sz),
    "bsgpu_vis_workspace_size_ex": ([_i, _i64, _i64, _i64, _sz, _sz, _i], _sz),
    "bsgpu_status": ([_vp, _vp, ctypes.POINTER(_i)], _i),
    "bsgpu_reduce_precision_c64": ([_vp, _vp, _i64, _i64, _i64, _d, _d, _vp, _sz, _vp], _i),
    "bsgpu_reduce_precision_ex": ([_vp, _vp, _i, _i64, _i64, _i64, _d, _d, _i, _vp, _sz, _vp],
                                  _i),
    "bsgpu_bitshuffle": ([_vp, _vp, _sz, _sz, _sz, _vp], _i),
    "bsgpu_bitunshuffle": ([_vp, _vp, _sz, _sz, _sz, _vp], _i),
    "bsgpu_compress": ([_vp, _sz, _sz, _sz, _i, _vp, _sz, _vp, _vp, _vp, _sz, _vp], _i),
    "bsgpu_decompress": ([_vp, _sz, _vp, _sz, _sz, _sz, _vp, _vp, _sz, _vp], _i),
    "bsgpu_compress_vis": ([_vp, _i64, _i64, _i64, _d, _d, _sz, _i, _vp, _sz, _vp, _vp, _vp,
                            _sz, _vp], _i),
    "bsgpu_reorder_time": ([_vp, _vp, ctypes.c_uint64, ctypes.c_uint64, _sz, _vp], _i),
    "bsgpu_full_noise_var": ([_vp, _i, _i64, _i64, _i64, _d, _i, _vp, _vp, _sz, _vp], _i),
    "bsgpu_compress_vis_ex": ([_vp, _i, _i64, _i64, _i64, _d, _d, _i, _sz, _sz, _i, _vp, _sz,
                               _vp, _vp, _vp, _sz, _vp], _i),
    "bsgpu_compress_noalloc": ([_vp, _sz, _sz, _sz, _i, _vp, _sz, _vp, _vp, _vp], _i),
    "bsgpu_batch_table_bytes": ([ctypes.c_uint32], _sz),
    "bsgpu_batch_plan": ([_i, _vp, ctypes.c_uint32, _vp, _sz, ctypes.POINTER(ctypes.c_uint64),
                          ctypes.POINTER(_sz)], _i),
    "bsgpu_compress_batch": ([_vp, ctypes.c_uint32, ctypes.c_uint64, _i, _vp, _vp, _vp, _vp, _sz,
                              ctypes.c_uint32, _vp], _i),
    "bsgpu_decompress_batch": ([_vp, ctypes.c_uint32, ctypes.c_uint64, _vp, _vp, _vp, _vp, _sz,
                                ctypes.c_uint32, _vp], _i),
    "bsgpu_compress_batch_ex": ([_vp, ctypes.c_uint32, ctypes.c_uint64, _i, _vp, _vp, _vp, _vp,
                                 _sz, ctypes.c_uint32, ctypes.c_uint32, _vp], _i),
    "bsgpu_decompress_batch_ex": ([_vp, ctypes.c_uint32, ctypes.c_uint64, _vp, _vp, _vp, _vp, _sz,
                                   ctypes.c_uint32, ctypes.c_uint32, _vp], _i),
    "bsgpu_arena_create": ([ctypes.c_uint64, ctypes.c_uint64], _vp),
    "bsgpu_arena_destroy": ([_vp], None),
    "bsgpu_arena_alloc": ([_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)], _i),
    "bsgpu_arena_free": ([_vp, ctypes.c_uint64], _i),
    "bsgpu_arena_stats": ([_vp] + [ctypes.POINTER(ctypes.c_uint64)] * 4, _i),
}


class Chunk(ctypes.Structure):
    """bsgpu_chunk: one chunk of a batch (device pointers, sizes)."""
    _fields_ = [("in_ptr", ctypes.c_void_p), ("out_ptr", ctypes.c_void_p),
                ("n_elem", ctypes.c_uint64), ("in_bytes", ctypes.c_uint64),
                ("out_cap", ctypes.c_uint64), ("elem_size", ctypes.c_uint32),
                ("block_elems", ctypes.c_uint32), ("block_offsets", ctypes.c_void_p)]
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class BsgpuError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {_NAMES.get(code, code)} ({code})")
        self.code = code


def library_path() -> str:
    return _LIB_PATH


def _check(code: int, where: str):
    if code != 0:
        raise BsgpuError(code, where)


def _stream(stream) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _bytes_view(t: torch.Tensor) -> torch.Tensor:
    return t.reshape(-1).view(torch.uint8)


# -- queries -----------------------------------------------------------------

def version() -> str:
    return _lib.bsgpu_version().decode()


def compress_bound(n_elem: int, elem_size: int, block_elems: int = 0) -> int:
    return _lib.bsgpu_compress_bound(n_elem, elem_size, block_elems)


def num_blocks(n_elem: int, elem_size: int, block_elems: int = 0) -> int:
    return _lib.bsgpu_num_blocks(n_elem, elem_size, block_elems)


def workspace_size(op: int, n_elem: int, elem_size: int, block_elems: int = 0) -> int:
    return _lib.bsgpu_workspace_size(op, n_elem, elem_size, block_elems)


def vis_workspace_size(op: int, n_freq: int, n_inputs: int, n_time: int,
                       block_elems: int = 0) -> int:
    return _lib.bsgpu_vis_workspace_size(op, n_freq, n_inputs, n_time, block_elems)


def vis_workspace_size_ex(op: int, n_freq: int, n_inputs: int, n_time: int, elem_size: int = 4,
                          block_elems: int = 0, flags: int = 0) -> int:
    return _lib.bsgpu_vis_workspace_size_ex(op, n_freq, n_inputs, n_time, elem_size, block_elems,
                                            flags)


def status(ws: torch.Tensor, stream=None) -> int:
    """Device status word of a workspace (waits for the stream)."""
    st = ctypes.c_int(0)
    _check(_lib.bsgpu_status(_ptr(ws), _stream(stream), ctypes.byref(st)), "bsgpu_status")
    return st.value


def new_workspace(nbytes: int, device=None) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8,
                       device=device or torch.cuda.current_device())


# -- Sec. 3: precision reduction ---------------------------------------------

def reduce_precision_c64(vis: torch.Tensor, N: float, f: float, out: torch.Tensor | None = None,
                         ws: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Round a [n_freq][n_prod][n_time] complex64 cube (returns out)."""
    F, P, T = vis.shape
    n = _n_inputs(P)
    out = torch.empty_like(vis) if out is None else out
    need = vis_workspace_size(OP_REDUCE_PRECISION, F, n, T)
    ws = new_workspace(need, vis.device) if ws is None else ws
    _check(_lib.bsgpu_reduce_precision_c64(_ptr(vis), _ptr(out), F, n, T, float(N), float(f),
                                           _ptr(ws), ws.numel(), _stream(stream)),
           "bsgpu_reduce_precision_c64")
    return out


def _cube(vis: torch.Tensor, time_slowest: bool = False):
    """(n_freq, n_inputs, n_time, dtype code) of a complex64 [F][P][T] cube or
    an int32 [F][P][T][2] cube of (re, im) pairs ([T][F][P] / [T][F][P][2]
    when time_slowest)."""
    if vis.dtype == torch.complex64 and vis.dim() == 3:
        a, b, c = vis.shape
        F, P, T = (b, c, a) if time_slowest else (a, b, c)
        return F, _n_inputs(P), T, VIS_F32
    if vis.dtype == torch.int32 and vis.dim() == 4 and vis.shape[3] == 2:
        a, b, c, _ = vis.shape
        F, P, T = (b, c, a) if time_slowest else (a, b, c)
        return F, _n_inputs(P), T, VIS_I32
    raise ValueError("expected a complex64 [F][P][T] or int32 [F][P][T][2] cube")


def _flags(compensate=False, time_slowest=False, full_cov=False) -> int:
    return ((VIS_COMPENSATE if compensate else 0) | (VIS_TIME_SLOWEST if time_slowest else 0) |
            (VIS_FULL_COV if full_cov else 0))


def reduce_precision(vis: torch.Tensor, N: float, f: float, compensate: bool = False,
                     out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                     stream=None, time_slowest: bool = False,
                     full_cov: bool = False) -> torch.Tensor:
    """Round a complex64 or int32 cube, optionally with Sec. 3.2's
    compensated f, from the time-slowest order, or with the full-covariance
    noise of Sec. 3.1 (returns out, time fastest)."""
    F, n, T, dt = _cube(vis, time_slowest)
    flags = _flags(compensate, time_slowest, full_cov)
    if out is None:
        P = n * (n + 1) // 2
        shape = (F, P, T) if vis.dim() == 3 else (F, P, T, 2)
        out = torch.empty(shape, dtype=vis.dtype, device=vis.device)
    need = vis_workspace_size_ex(OP_REDUCE_PRECISION, F, n, T, 4, 0, flags)
    ws = new_workspace(need, vis.device) if ws is None else ws
    _check(_lib.bsgpu_reduce_precision_ex(_ptr(vis), _ptr(out), dt, F, n, T, float(N), float(f),
                                          flags, _ptr(ws), ws.numel(), _stream(stream)),
           "bsgpu_reduce_precision_ex")
    return out


def full_noise_var(vis: torch.Tensor, N: float, time_slowest: bool = False,
                   stream=None) -> torch.Tensor:
    """s^2 = 1/(C^-1)_kk of Eq. noise with the full covariance, as a
    [n_freq][n_time][n_inputs^2] float64 tensor."""
    F, n, T, dt = _cube(vis, time_slowest)
    flags = _flags(time_slowest=time_slowest)
    need = vis_workspace_size_ex(OP_REDUCE_PRECISION, F, n, T, 4, 0, flags | VIS_FULL_COV)
    if need == 0:
        raise BsgpuError(ERR_ARG, "bsgpu_vis_workspace_size_ex")
    ws = new_workspace(need, vis.device)
    s2 = torch.empty((F, T, n * n), dtype=torch.float64, device=vis.device)
    _check(_lib.bsgpu_full_noise_var(_ptr(vis), dt, F, n, T, float(N), flags, _ptr(s2), _ptr(ws),
                                     ws.numel(), _stream(stream)), "bsgpu_full_noise_var")
    return s2


def reorder_time(x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """[T][...] (time slowest) -> [...][T] (time fastest) for a contiguous
    tensor whose first axis is time (elements of 1, 2, 4 or 8 bytes; complex64
    counts as one 8-byte element)."""
    T = x.shape[0]
    S = x.numel() // T if T else 0
    if out is None:
        out = torch.empty(tuple(x.shape[1:]) + (T,), dtype=x.dtype, device=x.device)
    _check(_lib.bsgpu_reorder_time(_ptr(x), _ptr(out), T, S, x.element_size(), _stream(stream)),
           "bsgpu_reorder_time")
    return out


def _n_inputs(P: int) -> int:
    n = int(round(((8 * P + 1) ** 0.5 - 1) / 2))
    if n * (n + 1) // 2 != P:
        raise ValueError(f"{P} products is not n(n+1)/2")
    return n


# -- Sec. 4.2: Bitshuffle ----------------------------------------------------

def bitshuffle(x: torch.Tensor, block_elems: int = 0, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    out = torch.empty_like(x) if out is None else out
    _check(_lib.bsgpu_bitshuffle(_ptr(x), _ptr(out), x.numel(), x.element_size(), block_elems,
                                 _stream(stream)), "bsgpu_bitshuffle")
    return out


def bitunshuffle(x: torch.Tensor, block_elems: int = 0, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    out = torch.empty_like(x) if out is None else out
    _check(_lib.bsgpu_bitunshuffle(_ptr(x), _ptr(out), x.numel(), x.element_size(), block_elems,
                                   _stream(stream)), "bsgpu_bitunshuffle")
    return out


# -- Sec. 4.1 / 4.2.1: compress / decompress ----------------------------------

class Compressed:
    """A compressed stream on the device: `buf[:nbytes]` is the framed stream,
    `offsets` the per-block index (or None); `nbytes` is read lazily."""

    def __init__(self, buf, nbytes_dev, offsets, n_elem, elem_size, block_elems, ws):
        self.buf, self.nbytes_dev, self.offsets = buf, nbytes_dev, offsets
        self.n_elem, self.elem_size, self.block_elems, self.ws = n_elem, elem_size, block_elems, ws

    @property
    def nbytes(self) -> int:
        return int(self.nbytes_dev.item())

    def stream_bytes(self) -> torch.Tensor:
        return self.buf[: self.nbytes]


def compress(x: torch.Tensor, block_elems: int = 0, elem_size: int | None = None,
             out: torch.Tensor | None = None, with_offsets: bool = True,
             ws: torch.Tensor | None = None, stream=None, level: int = 0) -> Compressed:
    es = elem_size or x.element_size()
    n = x.numel() * x.element_size() // es
    cap = compress_bound(n, es, block_elems)
    if cap == 0:
        raise BsgpuError(ERR_ARG, "bsgpu_compress_bound")
    out = torch.empty(cap, dtype=torch.uint8, device=x.device) if out is None else out
    nb_dev = torch.zeros(1, dtype=torch.int64, device=x.device)
    nblk = num_blocks(n, es, block_elems)
    offs = torch.empty(max(nblk, 1), dtype=torch.int64, device=x.device) if with_offsets else None
    need = workspace_size(OP_COMPRESS, n, es, block_elems)
    ws = new_workspace(need, x.device) if ws is None else ws
    _check(_lib.bsgpu_compress(_ptr(x), n, es, block_elems, level, _ptr(out), out.numel(),
                               _ptr(nb_dev),
                               _ptr(offs), _ptr(ws), ws.numel(), _stream(stream)),
           "bsgpu_compress")
    return Compressed(out, nb_dev, offs, n, es, block_elems, ws)


def compress_vis(vis: torch.Tensor, N: float, f: float, block_elems: int = 0,
                 out: torch.Tensor | None = None, with_offsets: bool = True,
                 ws: torch.Tensor | None = None, stream=None, level: int = 0) -> Compressed:
    """Precision reduction + Bitshuffle + LZ4 of a complex64 cube (Sec. 6)."""
    F, P, T = vis.shape
    n_in = _n_inputs(P)
    n = 2 * F * P * T
    cap = compress_bound(n, 4, block_elems)
    if cap == 0:
        raise BsgpuError(ERR_ARG, "bsgpu_compress_bound")
    out = torch.empty(cap, dtype=torch.uint8, device=vis.device) if out is None else out
    nb_dev = torch.zeros(1, dtype=torch.int64, device=vis.device)
    nblk = num_blocks(n, 4, block_elems)
    offs = torch.empty(max(nblk, 1), dtype=torch.int64, device=vis.device) if with_offsets else None
    need = vis_workspace_size(OP_COMPRESS_VIS, F, n_in, T, block_elems)
    ws = new_workspace(need, vis.device) if ws is None else ws
    _check(_lib.bsgpu_compress_vis(_ptr(vis), F, n_in, T, float(N), float(f), block_elems,
                                   level, _ptr(out), out.numel(), _ptr(nb_dev), _ptr(offs), _ptr(ws),
                                   ws.numel(), _stream(stream)), "bsgpu_compress_vis")
    return Compressed(out, nb_dev, offs, n, 4, block_elems, ws)


def compress_vis_ex(vis: torch.Tensor, N: float, f: float, compensate: bool = False,
                    elem_size: int = 4, block_elems: int = 0, out: torch.Tensor | None = None,
                    with_offsets: bool = True, ws: torch.Tensor | None = None, stream=None,
                    level: int = 0, time_slowest: bool = False,
                    full_cov: bool = False) -> Compressed:
    """Precision reduction (complex64 or int32 cube, optionally compensated,
    optionally from the time-slowest order) + Bitshuffle + LZ4 with 4-byte
    components or 8-byte samples as elements."""
    F, n_in, T, dt = _cube(vis, time_slowest)
    flags = _flags(compensate, time_slowest, full_cov)
    n = F * (n_in * (n_in + 1) // 2) * T * 8 // elem_size
    cap = compress_bound(n, elem_size, block_elems)
    if cap == 0:
        raise BsgpuError(ERR_ARG, "bsgpu_compress_bound")
    out = torch.empty(cap, dtype=torch.uint8, device=vis.device) if out is None else out
    nb_dev = torch.zeros(1, dtype=torch.int64, device=vis.device)
    nblk = num_blocks(n, elem_size, block_elems)
    offs = torch.empty(max(nblk, 1), dtype=torch.int64, device=vis.device) if with_offsets else None
    need = vis_workspace_size_ex(OP_COMPRESS_VIS, F, n_in, T, elem_size, block_elems, flags)
    ws = new_workspace(need, vis.device) if ws is None else ws
    _check(_lib.bsgpu_compress_vis_ex(_ptr(vis), dt, F, n_in, T, float(N), float(f), flags,
                                      elem_size, block_elems, level, _ptr(out), out.numel(),
                                      _ptr(nb_dev), _ptr(offs), _ptr(ws), ws.numel(),
                                      _stream(stream)), "bsgpu_compress_vis_ex")
    return Compressed(out, nb_dev, offs, n, elem_size, block_elems, ws)


def decompress(stream_buf: torch.Tensor, in_bytes: int, n_elem: int, elem_size: int,
               block_elems: int = 0, offsets: torch.Tensor | None = None,
               out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """Decode a framed stream into a uint8 tensor of n_elem * elem_size bytes."""
    dev = stream_buf.device
    out = torch.empty(n_elem * elem_size, dtype=torch.uint8, device=dev) if out is None else out
    need = workspace_size(OP_DECOMPRESS, n_elem, elem_size, block_elems)
    if need == 0:
        raise BsgpuError(ERR_ARG, "bsgpu_workspace_size")
    ws = new_workspace(need, dev) if ws is None else ws
    _check(_lib.bsgpu_decompress(_ptr(stream_buf), in_bytes, _ptr(out), n_elem, elem_size,
                                 block_elems, _ptr(offsets), _ptr(ws), ws.numel(),
                                 _stream(stream)), "bsgpu_decompress")
    return out


def compress_noalloc(x: torch.Tensor, block_elems: int = 0, elem_size: int | None = None,
                     out: torch.Tensor | None = None, nbytes_dev: torch.Tensor | None = None,
                     offsets: torch.Tensor | None = None, stream=None, level: int = 0):
    """bsgpu_compress_noalloc: compress with the library's own fixed scratch
    (for callers that cannot allocate).  Returns (out, nbytes_dev, offsets);
    the caller may pass all three preallocated."""
    es = elem_size or x.element_size()
    n = x.numel() * x.element_size() // es
    cap = compress_bound(n, es, block_elems)
    if cap == 0:
        raise BsgpuError(ERR_ARG, "bsgpu_compress_bound")
    out = torch.empty(cap, dtype=torch.uint8, device=x.device) if out is None else out
    if nbytes_dev is None:
        nbytes_dev = torch.zeros(1, dtype=torch.int64, device=x.device)
    _check(_lib.bsgpu_compress_noalloc(_ptr(x), n, es, block_elems, level, _ptr(out), out.numel(),
                                       _ptr(nbytes_dev), _ptr(offsets), _stream(stream)),
           "bsgpu_compress_noalloc")
    return out, nbytes_dev, offsets


# -- batched codec (one persistent launch over many chunks) -------------------

def batch_table_bytes(n_chunks: int) -> int:
    return _lib.bsgpu_batch_table_bytes(n_chunks)


def batch_plan(op: int, chunks) -> tuple:
    """Validate a list of :class:`Chunk` for op and return (table image as a
    uint8 CPU tensor, n_items, workspace bytes).  Host only."""
    n = len(chunks)
    arr = (Chunk * n)(*chunks)
    table = torch.zeros(max(batch_table_bytes(n), 16), dtype=torch.uint8)
    n_items, ws = ctypes.c_uint64(0), ctypes.c_size_t(0)
    _check(_lib.bsgpu_batch_plan(op, ctypes.cast(arr, ctypes.c_void_p), n, table.data_ptr(),
                                 table.numel(), ctypes.byref(n_items), ctypes.byref(ws)),
           "bsgpu_batch_plan")
    return table, n_items.value, ws.value


def compress_batch(d_table: torch.Tensor, n_chunks: int, n_items: int, out_bytes: torch.Tensor,
                   offsets: torch.Tensor | None, status: torch.Tensor, ws: torch.Tensor,
                   level: int = 0, ctas_per_sm: int = 0, stream=None,
                   warps_per_cta: int = 1) -> None:
    _check(_lib.bsgpu_compress_batch_ex(_ptr(d_table), n_chunks, n_items, level, _ptr(out_bytes),
                                        _ptr(offsets), _ptr(status), _ptr(ws), ws.numel(),
                                        ctas_per_sm, warps_per_cta, _stream(stream)),
           "bsgpu_compress_batch_ex")


def decompress_batch(d_table: torch.Tensor, n_chunks: int, n_items: int,
                     in_bytes: torch.Tensor | None, offsets: torch.Tensor | None,
                     status: torch.Tensor, ws: torch.Tensor, ctas_per_sm: int = 0,
                     stream=None, warps_per_cta: int = 1) -> None:
    _check(_lib.bsgpu_decompress_batch_ex(_ptr(d_table), n_chunks, n_items, _ptr(in_bytes),
                                          _ptr(offsets), _ptr(status), _ptr(ws), ws.numel(),
                                          ctas_per_sm, warps_per_cta, _stream(stream)),
           "bsgpu_decompress_batch_ex")


class Arena:
    """Offsets of a fixed-capacity device arena (bsgpu_arena_*): host-side
    bookkeeping only; the caller owns the device allocation."""

    def __init__(self, capacity: int, align: int = 256):
        self._h = _lib.bsgpu_arena_create(capacity, align)
        if not self._h:
            raise BsgpuError(ERR_ARG, "bsgpu_arena_create")
        self.capacity, self.align = capacity // align * align, align

    def alloc(self, nbytes: int):
        """Offset of a new range, or None when nothing large enough is free."""
        off = ctypes.c_uint64(0)
        rc = _lib.bsgpu_arena_alloc(self._h, nbytes, ctypes.byref(off))
        if rc == ERR_SPACE:
            return None
        _check(rc, "bsgpu_arena_alloc")
        return off.value

    def free(self, offset: int) -> None:
        _check(_lib.bsgpu_arena_free(self._h, offset), "bsgpu_arena_free")

    def stats(self) -> dict:
        v = [ctypes.c_uint64(0) for _ in range(4)]
        _check(_lib.bsgpu_arena_stats(self._h, *[ctypes.byref(x) for x in v]), "bsgpu_arena_stats")
        return dict(zip(("used", "largest_free", "high_water", "free_ranges"),
                        (x.value for x in v)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.bsgpu_arena_destroy(h)
            self._h = None
