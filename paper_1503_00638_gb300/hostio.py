"""Compressing visibility cubes that live in host memory.

The paper stores data in chunks, each compressed on its own (HDF5 chunks,
Sec. 2.3; blocks within a chunk, Sec. 4.2.1).  `HostVisCodec` does the same
with frequency slabs of a host cube: every slab is one framed stream (as
``bsgpu_compress_vis`` writes it) with its block index, and slabs are
software-pipelined so that the upload of one slab, the kernels of another and
the download of a third overlap, and uploads run beside downloads.  Each kind
of copy (cube up, stream down, stream up, cube down) has a CUDA stream of
its own besides the kernels' stream, so that no copy waits behind another
kind's in one queue (measured on the CHIME-shaped cube: 88 GB/s round trip
with one upload and one download stream, 103 GB/s with one per kind).  Slabs are independent: the noise of Sec. 3.1 only needs a
slab's own autocorrelations.

`HostBatchCodec` does the same for the batch workload: groups of chunks,
one batched launch per group and direction (measured on 447 chunks of the
batch generator, 4.3 GB: 90 GB/s round trip, against 44 GB/s with the
copies and launches one after another on one stream).

Host orchestration only (pinned buffers, streams, events); the rounding,
shuffling and coding run in libbsgpu's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import bsgpu


@dataclass
class Chunk:
    freq: tuple           # (f0, f1)
    nbytes: int           # stream length
    stream: torch.Tensor  # pinned host bytes [nbytes]
    index: torch.Tensor   # pinned host int64 block offsets


class HostVisCodec:
    """Round + compress a [F][P][T] complex64 host cube slab by slab, and
    decompress such slabs back into host memory, with copies and kernels
    overlapped.

    slab_freq : frequencies per slab (one stream each)
    depth     : slabs in flight (device buffers are allocated per slot)
    """

    def __init__(self, n_freq: int, n_inputs: int, n_time: int, N: float, f: float,
                 block_elems: int = 2048, level: int = 0, slab_freq: int = 64, depth: int = 3,
                 device="cuda"):
        self.F, self.n_in, self.T = n_freq, n_inputs, n_time
        self.P = n_inputs * (n_inputs + 1) // 2
        self.N, self.f, self.B, self.level = float(N), float(f), block_elems, level
        self.slabs = [(f0, min(n_freq, f0 + slab_freq)) for f0 in range(0, n_freq, slab_freq)]
        self.depth = min(depth, len(self.slabs))
        dev = torch.device(device)
        self.dev = dev
        sf = slab_freq
        self.slab_elems = sf * self.P * n_time * 2          # float32 components
        self.cap = bsgpu.compress_bound(self.slab_elems, 4, block_elems)
        self.nblk = bsgpu.num_blocks(self.slab_elems, 4, block_elems)
        wsc = bsgpu.vis_workspace_size(bsgpu.OP_COMPRESS_VIS, sf, n_inputs, n_time, block_elems)
        wsd = bsgpu.workspace_size(bsgpu.OP_DECOMPRESS, self.slab_elems, 4, block_elems)
        self.slot = []
        for _ in range(self.depth):
            self.slot.append({
                "vis": torch.empty((sf, self.P, n_time), dtype=torch.complex64, device=dev),
                "stream": torch.empty(self.cap, dtype=torch.uint8, device=dev),
                "offs": torch.empty(max(self.nblk, 1), dtype=torch.int64, device=dev),
                "nb": torch.zeros(1, dtype=torch.int64, device=dev),
                "h_nb": torch.zeros(1, dtype=torch.int64).pin_memory(),
                "ws_c": bsgpu.new_workspace(wsc, dev),
                "ws_d": bsgpu.new_workspace(wsd, dev),
                "out": torch.empty(self.slab_elems * 4, dtype=torch.uint8, device=dev),
                "ev_in": torch.cuda.Event(), "ev_c": torch.cuda.Event(),
                "ev_d2h": torch.cuda.Event(), "ev_dc": torch.cuda.Event(),
                "free": torch.cuda.Event(),
            })
        self.s_k = torch.cuda.Stream(device=dev)       # kernels
        self.s_upc = torch.cuda.Stream(device=dev)     # cube slabs up
        self.s_dns = torch.cuda.Stream(device=dev)     # streams and indexes down
        self.s_ups = torch.cuda.Stream(device=dev)     # streams and indexes up
        self.s_dnc = torch.cuda.Stream(device=dev)     # decoded slabs down
        self.h_streams = [torch.empty(self.cap, dtype=torch.uint8).pin_memory() for _ in self.slabs]
        self.h_index = [torch.empty(max(self.nblk, 1), dtype=torch.int64).pin_memory()
                        for _ in self.slabs]

    # -- helpers ------------------------------------------------------------

    def _compress_slab(self, sl, F):
        b = bsgpu
        b._check(b._lib.bsgpu_compress_vis(
            sl["vis"].data_ptr(), F, self.n_in, self.T, self.N, self.f, self.B, self.level,
            sl["stream"].data_ptr(), self.cap, sl["nb"].data_ptr(), sl["offs"].data_ptr(),
            sl["ws_c"].data_ptr(), sl["ws_c"].numel(), self.s_k.cuda_stream), "bsgpu_compress_vis")

    def _decompress_slab(self, sl, F, L):
        b = bsgpu
        n = F * self.P * self.T * 2
        b._check(b._lib.bsgpu_decompress(
            sl["stream"].data_ptr(), L, sl["out"].data_ptr(), n, 4, self.B, sl["offs"].data_ptr(),
            sl["ws_d"].data_ptr(), sl["ws_d"].numel(), self.s_k.cuda_stream), "bsgpu_decompress")

    # -- the pipelined round trip -------------------------------------------

    def round_trip(self, h_vis: torch.Tensor, h_out: torch.Tensor, lag: int = 1) -> list:
        """Compress the pinned host cube h_vis ([F][P][T] complex64) slab by slab
        into pinned host streams, then decompress every stream (read back from
        host memory) into the pinned host tensor h_out (same shape), with
        uploads, kernels and downloads of different slabs overlapped.
        Returns the chunks (freq range, length, host stream and index)."""
        n = len(self.slabs)
        # slab k reuses the slot of slab k - depth, whose copies back are
        # enqueued `lag` steps after its kernels: the slot must be free first
        lag = max(0, min(lag, self.depth - 1))
        lens = [0] * n
        for sl in self.slot:
            sl["free"].record(self.s_dnc)
        for step in range(n + lag):
            k = step
            if k < n:
                sl = self.slot[k % self.depth]
                f0, f1 = self.slabs[k]
                F = f1 - f0
                self.s_upc.wait_event(sl["free"])
                with torch.cuda.stream(self.s_upc):
                    sl["vis"][:F].copy_(h_vis[f0:f1], non_blocking=True)
                    sl["ev_in"].record(self.s_upc)
                self.s_k.wait_event(sl["ev_in"])
                with torch.cuda.stream(self.s_k):
                    self._compress_slab(sl, F)
                    sl["h_nb"].copy_(sl["nb"], non_blocking=True)
                    sl["ev_c"].record(self.s_k)
            j = step - lag
            if j >= 0:
                sl = self.slot[j % self.depth]
                f0, f1 = self.slabs[j]
                F = f1 - f0
                sl["ev_c"].synchronize()              # the stream length, for exact copies
                L = int(sl["h_nb"][0])
                lens[j] = L
                nb = bsgpu.num_blocks(F * self.P * self.T * 2, 4, self.B)
                self.s_dns.wait_event(sl["ev_c"])
                with torch.cuda.stream(self.s_dns):
                    self.h_streams[j][:L].copy_(sl["stream"][:L], non_blocking=True)
                    self.h_index[j][:nb].copy_(sl["offs"][:nb], non_blocking=True)
                    sl["ev_d2h"].record(self.s_dns)
                # decompression reads the stream back from host memory
                self.s_ups.wait_event(sl["ev_d2h"])
                with torch.cuda.stream(self.s_ups):
                    sl["stream"][:L].copy_(self.h_streams[j][:L], non_blocking=True)
                    sl["offs"][:nb].copy_(self.h_index[j][:nb], non_blocking=True)
                    sl["ev_in"].record(self.s_ups)
                self.s_k.wait_event(sl["ev_in"])
                with torch.cuda.stream(self.s_k):
                    self._decompress_slab(sl, F, L)
                    sl["ev_dc"].record(self.s_k)
                self.s_dnc.wait_event(sl["ev_dc"])
                with torch.cuda.stream(self.s_dnc):
                    nbytes = F * self.P * self.T * 8
                    h_out.view(torch.uint8).reshape(-1)[f0 * self.P * self.T * 8:
                                                       f0 * self.P * self.T * 8 + nbytes].copy_(
                        sl["out"][:nbytes], non_blocking=True)
                    sl["free"].record(self.s_dnc)
        torch.cuda.synchronize(self.dev)
        return [Chunk(self.slabs[j], lens[j], self.h_streams[j][:lens[j]],
                      self.h_index[j][:bsgpu.num_blocks((self.slabs[j][1] - self.slabs[j][0]) *
                                                         self.P * self.T * 2, 4, self.B)])
                for j in range(n)]

    def statuses(self):
        return [(bsgpu.status(sl["ws_c"]), bsgpu.status(sl["ws_d"])) for sl in self.slot]

    def bytes_moved(self, chunks):
        """(host-to-device, device-to-host) bytes of one round trip."""
        cube = self.F * self.P * self.T * 8
        streams = sum(c.nbytes for c in chunks)
        idx = sum(c.index.numel() * 8 for c in chunks)
        return cube + streams + idx, streams + idx + cube + 8 * len(chunks)


def chunk_groups(sizes, group_bytes: int):
    """Consecutive chunks in groups of at most group_bytes (a chunk larger
    than that is a group of its own): [(first, end), ...] covering all."""
    groups, i, n = [], 0, len(sizes)
    while i < n:
        j, acc = i, 0
        while j < n and (j == i or acc + sizes[j] <= group_bytes):
            acc += sizes[j]
            j += 1
        groups.append((i, j))
        i = j
    return groups


class HostBatchCodec:
    """Round trip of many chunks that live in pinned host memory (the batch
    workload: uneven sizes and element widths), in groups of consecutive
    chunks: each group is one `engine.BatchCodec` (one persistent launch per
    direction over every block of its chunks), and the upload of one group,
    the kernels of another and the downloads of a third overlap, with one
    CUDA stream per kind of copy as in `HostVisCodec`.  Every chunk's stream
    (its exact length) and block index go to host memory and are read back
    from there for the decompression, so the round trip moves what storing
    the streams would.

    sizes       : bytes of each chunk
    elem_sizes  : element size of each chunk (1, 2, 4 or 8)
    block_elems : block size (elements) of each chunk, or one for all
    group_bytes : uncompressed bytes per group (a group holds at least one chunk)
    launch      : (warps per CTA, CTAs per SM) of the compress and the
                  decompress launch, e.g. the autotuner's choice
    """

    def __init__(self, sizes, elem_sizes, block_elems, level: int = 0,
                 group_bytes: int = 512 << 20, launch=((1, 0), (1, 0)), device="cuda"):
        from . import engine
        self.dev = torch.device(device)
        self.sizes = [int(s) for s in sizes]
        self.es = [int(e) for e in elem_sizes]
        n = len(self.sizes)
        bl = block_elems if isinstance(block_elems, (list, tuple)) else [block_elems] * n
        self.groups = chunk_groups(self.sizes, group_bytes)
        self.codecs = []
        for g0, g1 in self.groups:
            xs = [torch.empty(self.sizes[k], dtype=torch.uint8, device=self.dev) for k in range(g0, g1)]
            c = engine.BatchCodec(xs, self.es[g0:g1], list(bl[g0:g1]), level=level)
            (c.warps_c, c.ctas_c), (c.warps_d, c.ctas_d) = launch
            self.codecs.append(c)
        self.s_k = torch.cuda.Stream(device=self.dev)
        self.s_upc = torch.cuda.Stream(device=self.dev)   # chunks up
        self.s_dns = torch.cuda.Stream(device=self.dev)   # streams down
        self.s_ups = torch.cuda.Stream(device=self.dev)   # streams up
        self.s_dnc = torch.cuda.Stream(device=self.dev)   # chunks down
        self.h_len = [torch.empty(c.n, dtype=torch.int64).pin_memory() for c in self.codecs]
        self.h_streams = [[torch.empty(cap, dtype=torch.uint8).pin_memory() for cap in c.caps]
                          for c in self.codecs]
        self.h_index = [torch.empty(max(c.n_items, 1), dtype=torch.int64).pin_memory()
                        for c in self.codecs]
        self.lens = [None] * len(self.codecs)

    def round_trip(self, h_in, h_out, lag: int = 1) -> None:
        """Compress the pinned host chunks h_in (uint8 tensors of `sizes`) into
        pinned host streams and decompress those back into the pinned host
        tensors h_out, group by group with copies and kernels overlapped."""
        G = len(self.codecs)
        lag = max(0, lag)
        ev = [{k: torch.cuda.Event() for k in ("in", "c", "d2h", "up", "dc")} for _ in range(G)]
        for step in range(G + lag):
            g = step
            if g < G:
                c, (g0, _) = self.codecs[g], self.groups[g]
                with torch.cuda.stream(self.s_upc):
                    for k, x in enumerate(c.inputs):
                        x.copy_(h_in[g0 + k], non_blocking=True)
                    ev[g]["in"].record(self.s_upc)
                self.s_k.wait_event(ev[g]["in"])
                with torch.cuda.stream(self.s_k):
                    c.compress(self.s_k)
                    self.h_len[g].copy_(c.out_bytes, non_blocking=True)
                    ev[g]["c"].record(self.s_k)
            j = step - lag
            if j >= 0:
                c, (g0, _) = self.codecs[j], self.groups[j]
                ev[j]["c"].synchronize()               # the stream lengths, for exact copies
                lens = self.h_len[j].tolist()
                self.lens[j] = lens
                self.s_dns.wait_event(ev[j]["c"])
                with torch.cuda.stream(self.s_dns):
                    for k, L in enumerate(lens):
                        o = c.stream_off[k]
                        self.h_streams[j][k][:L].copy_(c.stream_arena[o:o + L], non_blocking=True)
                    self.h_index[j][:c.n_items].copy_(c.offsets, non_blocking=True)
                    ev[j]["d2h"].record(self.s_dns)
                self.s_ups.wait_event(ev[j]["d2h"])
                with torch.cuda.stream(self.s_ups):
                    for k, L in enumerate(lens):
                        o = c.stream_off[k]
                        c.stream_arena[o:o + L].copy_(self.h_streams[j][k][:L], non_blocking=True)
                    c.offsets.copy_(self.h_index[j][:c.n_items], non_blocking=True)
                    c.out_bytes.copy_(self.h_len[j], non_blocking=True)
                    ev[j]["up"].record(self.s_ups)
                self.s_k.wait_event(ev[j]["up"])
                with torch.cuda.stream(self.s_k):
                    c.decompress(self.s_k)
                    ev[j]["dc"].record(self.s_k)
                self.s_dnc.wait_event(ev[j]["dc"])
                with torch.cuda.stream(self.s_dnc):
                    for k in range(c.n):
                        h_out[g0 + k].copy_(c.output(k), non_blocking=True)
        torch.cuda.synchronize(self.dev)

    def statuses(self):
        return [c.statuses() for c in self.codecs]

    def bytes_moved(self):
        """(host-to-device, device-to-host) bytes of one round trip."""
        data = sum(self.sizes)
        streams = sum(sum(l) for l in self.lens if l)
        idx = sum(8 * c.n_items for c in self.codecs)
        lens = sum(8 * c.n for c in self.codecs)
        return data + streams + idx + lens, streams + idx + data + lens
