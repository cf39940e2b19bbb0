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
* an autotuner over the launch shape (warps per CTA and resident CTAs per
  SM, each launch on its own) and over the block size (``tune``).

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
    warps_per_cta: int = 1


# Launch shapes the tuner times: (warps per CTA, CTAs per SM); 0 CTAs = as many
# as fit.  With 96 registers a thread, at most 20 warps are resident per SM
# (the kernels' launch bounds), so the shapes span 8 to 20 warps per SM in
# CTAs of one, two or four warps.
SHAPES = ((1, 8), (1, 12), (1, 16), (1, 0), (2, 4), (2, 6), (2, 8), (2, 0), (4, 2), (4, 3),
          (4, 4), (4, 0))


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
        self.warps_c = 1
        self.warps_d = 1
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
                             self.status_c, self.ws_c, self.level, self.ctas_c, stream,
                             warps_per_cta=self.warps_c)

    def decompress(self, stream=None) -> None:
        if not self.round_trip:
            raise RuntimeError("planned without round_trip")
        # stream lengths straight from the compressor's device array
        bsgpu.decompress_batch(self.table_d, self.n, self.n_items, self.out_bytes, self.offsets,
                               self.status_d, self.ws_d, self.ctas_d, stream,
                               warps_per_cta=self.warps_d)

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

    def autotune(self, shapes=SHAPES, reps: int = 3) -> tuple:
        """Pick the launch shape (warps per CTA, CTAs per SM) of each launch by
        timing every candidate; a bare int k in `shapes` means (1, k).
        Returns (compress, decompress) as :class:`TuneResult`, whose table
        maps "WxC" (W warps per CTA, C CTAs per SM, 0 = as many as fit) to
        the best time in ms."""
        shapes = [(1, k) if isinstance(k, int) else tuple(k) for k in shapes]
        res = []
        for which in ("c", "d") if self.round_trip else ("c",):
            table = {}
            for w, k in shapes:
                if which == "c":
                    self.warps_c, self.ctas_c = w, k
                    table[f"{w}x{k}"] = (self._time(self.compress, reps), w, k)
                else:
                    self.warps_d, self.ctas_d = w, k
                    table[f"{w}x{k}"] = (self._time(self.decompress, reps), w, k)
            best = min(table, key=lambda key: table[key][0])
            ms, w, k = table[best]
            if which == "c":
                self.warps_c, self.ctas_c = w, k
            else:
                self.warps_d, self.ctas_d = w, k
            res.append(TuneResult(k, ms, {key: v[0] for key, v in table.items()}, w))
        return tuple(res)


def choose_block_elems(inputs, elem_sizes, candidates_bytes=(2048, 4096, 8192), level: int = 0,
                       reps: int = 3, ratio_slack: float = 0.02) -> tuple:
    """Block size (bytes, the same for every chunk) with the fastest round
    trip among those whose compressed size is within ``ratio_slack`` of the
    smallest.  Returns (best block bytes, {bytes: (ms, compressed bytes)})."""
    best, table, _ = tune(inputs, elem_sizes, candidates_bytes, level=level, reps=reps,
                          ratio_slack=ratio_slack)
    return best, {b: (v["round_trip_ms"], v["compressed_bytes"]) for b, v in table.items()}


def tune(inputs, elem_sizes, candidates_bytes=(2048, 4096, 8192), level: int = 0,
         shapes=SHAPES, reps: int = 2, ratio_slack: float = 0.02, keep: bool = True) -> tuple:
    """The batch autotuner: for every candidate block size (bytes, the same
    for every chunk; Sec. 4.2.1 makes it the tunable of the method) tune the
    launch shape of each launch (:meth:`BatchCodec.autotune`), then time the
    round trip with the chosen shapes.  The block size chosen is the fastest
    round trip among those whose compressed size is within ``ratio_slack``
    of the smallest (a smaller block may be faster but compress worse).
    Returns (best block bytes, {bytes: record}, the codec of the best block
    size with its shapes set, or None when keep is False)."""
    results, engines = {}, {}
    for bb in candidates_bytes:
        blocks = [bb // es for es in elem_sizes]
        eng = BatchCodec(inputs, elem_sizes, blocks, level=level)
        tc, td = eng.autotune(shapes, reps=reps)

        def both():
            eng.compress()
            eng.decompress()
        ms = eng._time(both, reps)
        results[bb] = {"round_trip_ms": ms, "compressed_bytes": eng.compressed_bytes(),
                       "compress": {"warps_per_cta": tc.warps_per_cta, "ctas_per_sm": tc.ctas_per_sm,
                                    "ms": tc.ms, "candidates_ms": tc.table},
                       "decompress": {"warps_per_cta": td.warps_per_cta,
                                      "ctas_per_sm": td.ctas_per_sm, "ms": td.ms,
                                      "candidates_ms": td.table}}
        if keep:
            engines[bb] = eng
        else:
            del eng
    smallest = min(v["compressed_bytes"] for v in results.values())
    ok = [b for b, v in results.items() if v["compressed_bytes"] <= smallest * (1 + ratio_slack)]
    best = min(ok, key=lambda b: results[b]["round_trip_ms"])
    chosen = engines.pop(best) if keep else None
    engines.clear()
    return best, results, chosen
