"""Batched codec engine: many independent chunks, one persistent launch each way.

Sec. 4.2.1 makes every block an independent unit of work; the batch calls of
libbsgpu run one persistent launch whose work queue covers every (chunk,
block) item of a batch.  This module is host orchestration around them:

* the output and round-trip arenas (one allocation each, chunks 256-byte
  aligned), the per-chunk lengths, block index and status words;
* the table images written by the C planner (``bsgpu_batch_plan``), copied
  once to the device;
* CUDA-graph capture of the compress launch, the decompress launch or both
  (the decompressor reads the compressor's per-chunk lengths on the device,
  so the pair needs no host round trip);
* an autotuner over the launch shape (resident one-warp CTAs per SM) and,
  optionally, the block size.

Every step of the codec runs in libbsgpu's kernels; nothing here touches the
data.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import bsgpu

ALIGN = 256


def _round(x: int, a: int = ALIGN) -> int:
    return (x + a - 1) // a * a


@dataclass
class TuneResult:
    ctas_per_sm: int
    ms: float
    table: dict


class BatchCodec:
    """Compress (and optionally round-trip) a fixed list of device buffers.

    inputs      : CUDA tensors, contiguous, 16-byte aligned (any dtype; their
                  bytes are the chunk)
    elem_sizes  : element size of each chunk (1, 2, 4 or 8)
    block_elems : one block size for all chunks or one per chunk (0 = 4096
                  bytes; at most 8192 bytes)
    level       : LZ4 match search (0 or 1), as bsgpu_compress
    round_trip  : also plan the decompression into a second arena
    """

    def __init__(self, inputs, elem_sizes, block_elems=0, level: int = 0,
                 round_trip: bool = True, with_offsets: bool = True):
        self.n = len(inputs)
        if self.n == 0:
            raise ValueError("empty batch")
        dev = inputs[0].device
        self.device = dev
        self.level = level
        self.inputs = inputs
        self.elem_sizes = [int(e) for e in elem_sizes]
        bl = block_elems if isinstance(block_elems, (list, tuple)) else [block_elems] * self.n
        self.block_elems = [int(b) for b in bl]
        self.n_elem = [x.numel() * x.element_size() // es for x, es in zip(inputs, self.elem_sizes)]
        self.in_bytes_total = sum(x.numel() * x.element_size() for x in inputs)
        caps = [bsgpu.compress_bound(n, es, b)
                for n, es, b in zip(self.n_elem, self.elem_sizes, self.block_elems)]
        if min(caps) == 0:
            raise bsgpu.BsgpuError(bsgpu.ERR_ARG, "bsgpu_compress_bound")
        self.caps = caps
        self.stream_off = []
        o = 0
        for c in caps:
            self.stream_off.append(o)
            o += _round(c)
        self.stream_arena = torch.empty(max(o, ALIGN), dtype=torch.uint8, device=dev)
        base = self.stream_arena.data_ptr()
        chunks = [bsgpu.Chunk(x.data_ptr(), base + off, n, 0, cap, es, b)
                  for x, off, n, cap, es, b in zip(inputs, self.stream_off, self.n_elem, caps,
                                                   self.elem_sizes, self.block_elems)]
        table, self.n_items, ws = bsgpu.batch_plan(bsgpu.OP_COMPRESS, chunks)
        self.table_c = table.to(dev)
        self.ws_c = bsgpu.new_workspace(ws, dev)
        self.out_bytes = torch.zeros(self.n, dtype=torch.int64, device=dev)
        self.offsets = (torch.zeros(self.n_items, dtype=torch.int64, device=dev)
                        if with_offsets else None)
        self.status_c = torch.zeros(self.n, dtype=torch.int32, device=dev)
        self.ctas_c = 0
        self.ctas_d = 0
        self.round_trip = round_trip
        if round_trip:
            self.dec_off = []
            o = 0
            for n, es in zip(self.n_elem, self.elem_sizes):
                self.dec_off.append(o)
                o += _round(n * es)
            self.dec_arena = torch.empty(max(o, ALIGN), dtype=torch.uint8, device=dev)
            dbase = self.dec_arena.data_ptr()
            dchunks = [bsgpu.Chunk(base + so, dbase + do, n, cap, 0, es, b)
                       for so, do, n, cap, es, b in zip(self.stream_off, self.dec_off,
                                                        self.n_elem, caps, self.elem_sizes,
                                                        self.block_elems)]
            table, n_items_d, ws = bsgpu.batch_plan(bsgpu.OP_DECOMPRESS, dchunks)
            assert n_items_d == self.n_items
            self.table_d = table.to(dev)
            self.ws_d = bsgpu.new_workspace(ws, dev)
            self.status_d = torch.zeros(self.n, dtype=torch.int32, device=dev)

    # -- launches ---------------------------------------------------------

    def compress(self, stream=None) -> None:
        bsgpu.compress_batch(self.table_c, self.n, self.n_items, self.out_bytes, self.offsets,
                             self.status_c, self.ws_c, self.level, self.ctas_c, stream)

    def decompress(self, stream=None) -> None:
        if not self.round_trip:
            raise RuntimeError("planned without round_trip")
        # stream lengths straight from the compressor's device array
        bsgpu.decompress_batch(self.table_d, self.n, self.n_items, self.out_bytes, self.offsets,
                               self.status_d, self.ws_d, self.ctas_d, stream)

    def capture(self, compress: bool = True, decompress: bool = True) -> torch.cuda.CUDAGraph:
        """A CUDA graph of the chosen launches on a side stream (replay with
        ``g.replay()``; the inputs are read at replay time)."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            # one eager run first: the library sets kernel attributes on first use
            if compress:
                self.compress(s)
            if decompress:
                self.decompress(s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            if compress:
                self.compress(s)
            if decompress:
                self.decompress(s)
        return g

    # -- results ----------------------------------------------------------

    def stream(self, i: int) -> torch.Tensor:
        """Chunk i's framed stream (reads its length from the device)."""
        o = self.stream_off[i]
        return self.stream_arena[o:o + int(self.out_bytes[i].item())]

    def output(self, i: int) -> torch.Tensor:
        o = self.dec_off[i]
        return self.dec_arena[o:o + self.n_elem[i] * self.elem_sizes[i]]

    def compressed_bytes(self) -> int:
        return int(self.out_bytes.sum().item())

    def statuses(self):
        st = self.status_c.cpu().tolist()
        return st, (self.status_d.cpu().tolist() if self.round_trip else None)

    # -- tuning -----------------------------------------------------------

    def _time(self, fn, reps: int) -> float:
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            start.record()
            fn()
            end.record()
            end.synchronize()
            best = min(best, start.elapsed_time(end))
        return best

    def autotune(self, candidates=(0, 8, 12, 16), reps: int = 3) -> tuple:
        """Pick the resident CTAs per SM of each launch by timing every
        candidate (0 = as many as fit).  Returns (compress, decompress) as
        :class:`TuneResult`."""
        res = []
        for which in ("c", "d") if self.round_trip else ("c",):
            table = {}
            for k in candidates:
                if which == "c":
                    self.ctas_c = k
                    table[k] = self._time(self.compress, reps)
                else:
                    self.ctas_d = k
                    table[k] = self._time(self.decompress, reps)
            best = min(table, key=table.get)
            if which == "c":
                self.ctas_c = best
            else:
                self.ctas_d = best
            res.append(TuneResult(best, table[best], table))
        return tuple(res)


def choose_block_elems(inputs, elem_sizes, candidates_bytes=(2048, 4096, 8192), level: int = 0,
                       reps: int = 3, ratio_slack: float = 0.02) -> tuple:
    """Block size (bytes, the same for every chunk) with the fastest round
    trip among those whose compressed size is within ``ratio_slack`` of the
    smallest.  Returns (best block bytes, {bytes: (ms, compressed bytes)})."""
    results = {}
    for bb in candidates_bytes:
        blocks = [bb // es for es in elem_sizes]
        eng = BatchCodec(inputs, elem_sizes, blocks, level=level)
        eng.autotune(reps=1)

        def both():
            eng.compress()
            eng.decompress()
        ms = eng._time(both, reps)
        results[bb] = (ms, eng.compressed_bytes())
        del eng
    smallest = min(v[1] for v in results.values())
    ok = [b for b, v in results.items() if v[1] <= smallest * (1 + ratio_slack)]
    best = min(ok, key=lambda b: results[b][0])
    return best, results
