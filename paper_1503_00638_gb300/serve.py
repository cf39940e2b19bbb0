"""Serving compress / decompress requests on one GPU.

Requests arrive over time; each names a device buffer (elements to compress,
or a framed stream to decompress) that stays where the client put it.  The
server's device memory is one arena of fixed capacity (the admission cap)
from which every admitted request reserves its output; a request waits while
its output does not fit.

* :class:`BatchingServer` (continuous batching): whenever fewer than `depth`
  batches are in flight and requests wait, it admits waiting requests in
  arrival order while their outputs fit (and the batch has room), then
  launches ONE persistent batch launch for all admitted compressions and one
  for all admitted decompressions (libbsgpu's batch calls; Sec. 4.2.1's
  independent blocks of every request share the GPU).  A request completes
  when its batch's completion event is observed.
* :class:`SerialServer`: the plain pipeline, one request at a time through
  the single-stream calls (bsgpu_compress / bsgpu_decompress).

A request may carry a deadline for its admission, and a client may cancel
a request (set its ``cancelled`` flag, from any thread) while it waits: a
request that is still waiting past its deadline, or cancelled, leaves the
queue without touching the GPU, with status ``EXPIRED`` or ``CANCELLED``
(host-side failures: nothing on the device waits for it).  A request already
admitted completes normally.

Latency is measured from arrival to the observed completion.  Each request's
output is the same bytes alone or in any mix (tests check it); ``on_done``
sees it before its range returns to the arena.  Host orchestration only:
every step on the data runs in libbsgpu's kernels.
"""
from __future__ import annotations

import collections
import statistics
import time
from dataclasses import dataclass, field

import torch

from . import bsgpu

ALIGN = 256
EXPIRED = -101     # status of a request still waiting at its deadline
CANCELLED = -102   # status of a request cancelled while waiting


def _round(x: int) -> int:
    return (x + ALIGN - 1) // ALIGN * ALIGN


@dataclass
class Request:
    rid: int
    kind: str                 # "compress" or "decompress"
    arrival: float            # seconds after the start of the run
    data: torch.Tensor        # device bytes: the elements, or the framed stream
    n_elem: int
    elem_size: int
    block_elems: int = 0
    level: int = 0
    index: torch.Tensor | None = None   # decompress: the stream's block index
    deadline: float | None = None       # latest admission time (seconds after the start)
    cancelled: bool = False             # set by the client to withdraw a waiting request
    # filled in by the server
    admitted: float | None = None
    done: float | None = None
    status: int | None = None
    out_off: int | None = None
    out_cap: int = 0
    out_len: int = 0
    extra: dict = field(default_factory=dict)

    def n_blocks(self) -> int:
        return bsgpu.num_blocks(self.n_elem, self.elem_size, self.block_elems)

    def stream_cap(self) -> int:
        return bsgpu.compress_bound(self.n_elem, self.elem_size, self.block_elems)

    def out_bytes_needed(self) -> int:
        """Compress: the stream's worst case, then its block index (kept with
        the stream so that decompression starts every block at once)."""
        if self.kind == "compress":
            return _round(self.stream_cap()) + 8 * self.n_blocks()
        return self.n_elem * self.elem_size

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def nbytes(self) -> int:
        """Uncompressed bytes of the request."""
        return self.n_elem * self.elem_size


def latency_summary(reqs) -> dict:
    reqs = [r for r in reqs if r.status not in (EXPIRED, CANCELLED)]
    lat = sorted(r.latency for r in reqs)
    q = lambda p: lat[min(len(lat) - 1, int(p * len(lat)))]  # noqa: E731
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {"n": len(lat), "p50_ms": 1e3 * q(0.50), "p99_ms": 1e3 * q(0.99),
            "mean_ms": 1e3 * statistics.mean(lat), "max_ms": 1e3 * lat[-1],
            "gbs": sum(r.nbytes for r in reqs) / span / 1e9, "span_s": span}


class _Server:
    def __init__(self, cap_bytes: int, device="cuda", on_done=None):
        self.device = torch.device(device)
        self.cap = cap_bytes // ALIGN * ALIGN
        self.pool = torch.empty(self.cap, dtype=torch.uint8, device=self.device)
        self.arena = bsgpu.Arena(self.cap, ALIGN)
        self.on_done = on_done
        self.stream = torch.cuda.Stream(device=self.device)

    def output(self, r: Request) -> torch.Tensor:
        return self.pool[r.out_off:r.out_off + r.out_len]

    def output_index(self, r: Request) -> torch.Tensor:
        """A compress request's block index (n_blocks uint64s)."""
        o = r.out_off + _round(r.stream_cap())
        return self.pool[o:o + 8 * r.n_blocks()].view(torch.int64)

    def _index_ptr(self, r: Request):
        if r.kind == "compress":
            return self.pool.data_ptr() + r.out_off + _round(r.stream_cap()) if r.n_blocks() else None
        return r.index.data_ptr() if r.index is not None else None

    def _reserve(self, r: Request) -> bool:
        need = r.out_bytes_needed()
        if need > self.cap:
            raise ValueError(f"request {r.rid} needs {need} bytes, more than the cap")
        off = self.arena.alloc(need)
        if off is None:
            return False
        r.out_off, r.out_cap = off, need
        return True

    def _purge(self, waiting, now: float) -> int:
        """Withdraw waiting requests that are cancelled or past their deadline."""
        gone = [r for r in waiting
                if r.cancelled or (r.deadline is not None and now > r.deadline)]
        for r in gone:
            waiting.remove(r)
            r.status = CANCELLED if r.cancelled else EXPIRED
            r.done = now
        return len(gone)

    def _finish(self, r: Request, now: float):
        r.done = now
        if self.on_done:
            self.on_done(self, r)
        self.arena.free(r.out_off)

    def run(self, requests, idle_sleep: float = 20e-6):
        """Serve `requests` (sorted by arrival) in real time; returns them
        with admitted / done / status / out_len filled in."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        waiting = collections.deque()
        t0 = time.perf_counter()
        nxt, n_done = 0, 0
        while n_done < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                waiting.append(reqs[nxt])
                nxt += 1
            n_done += self._retire(now)
            if waiting:
                n_done += self._purge(waiting, now)
            launched = self._launch(waiting, now) if waiting else False
            if not launched and not self._busy():
                if nxt < len(reqs):
                    wait = reqs[nxt].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 1e-3))
            elif not launched:
                time.sleep(idle_sleep)
        torch.cuda.synchronize(self.device)
        return reqs


class _Slot:
    """Everything one in-flight batch owns: table images (pinned host and
    device), per-chunk lengths and statuses, block index, workspaces."""

    def __init__(self, dev, max_chunks: int):
        tb = bsgpu.batch_table_bytes(max_chunks)
        self.h_table_c = torch.empty(tb, dtype=torch.uint8).pin_memory()
        self.h_table_d = torch.empty(tb, dtype=torch.uint8).pin_memory()
        self.d_table_c = torch.empty(tb, dtype=torch.uint8, device=dev)
        self.d_table_d = torch.empty(tb, dtype=torch.uint8, device=dev)
        self.out_bytes = torch.zeros(max_chunks, dtype=torch.int64, device=dev)
        self.status_c = torch.zeros(max_chunks, dtype=torch.int32, device=dev)
        self.status_d = torch.zeros(max_chunks, dtype=torch.int32, device=dev)
        self.h_out_bytes = torch.zeros(max_chunks, dtype=torch.int64).pin_memory()
        self.h_status_c = torch.zeros(max_chunks, dtype=torch.int32).pin_memory()
        self.h_status_d = torch.zeros(max_chunks, dtype=torch.int32).pin_memory()
        self.ws_c = None
        self.ws_d = None
        self.event = torch.cuda.Event()
        self.reqs_c, self.reqs_d = [], []

    def workspace(self, which: str, nbytes: int, dev):
        cur = self.ws_c if which == "c" else self.ws_d
        if cur is None or cur.numel() < nbytes:
            cur = bsgpu.new_workspace(nbytes, dev)
            if which == "c":
                self.ws_c = cur
            else:
                self.ws_d = cur
        return cur


class BatchingServer(_Server):
    """Continuous batching with one persistent launch per batch and kind.

    cap_bytes  : the admission cap (bytes of request outputs on the device)
    depth      : batches in flight at once (>= 2 lets the host prepare the
                 next batch while the GPU runs the current one)
    max_chunks : requests per batch
    """

    def __init__(self, cap_bytes: int = 40 << 30, depth: int = 2, max_chunks: int = 4096,
                 min_block_bytes: int = 1024, device="cuda", on_done=None, ctas_per_sm: int = 0):
        super().__init__(cap_bytes, device, on_done)
        self.max_chunks = max_chunks
        self.min_block_bytes = min_block_bytes
        self.slots = [_Slot(self.device, max_chunks) for _ in range(depth)]
        self.free_slots = collections.deque(self.slots)
        self.inflight = collections.deque()
        self.ctas_per_sm = ctas_per_sm
        self.batches = []

    def _busy(self) -> bool:
        return bool(self.inflight)

    def _launch(self, waiting, now) -> bool:
        if not self.free_slots:
            return False
        slot = self.free_slots[0]
        batch = []
        while waiting and len(batch) < self.max_chunks:
            r = waiting[0]
            if r.block_elems * r.elem_size > 8192:
                raise ValueError("batched requests take blocks of at most 8192 bytes")
            if r.elem_size * (r.block_elems or 4096 // r.elem_size) < self.min_block_bytes:
                raise ValueError("block smaller than the server's min_block_bytes")
            if not self._reserve(r):
                break
            r.admitted = now
            batch.append(waiting.popleft())
        if not batch:
            return False
        self.free_slots.popleft()
        base = self.pool.data_ptr()
        slot.reqs_c = [r for r in batch if r.kind == "compress"]
        slot.reqs_d = [r for r in batch if r.kind == "decompress"]
        s = self.stream
        levels = {r.level for r in slot.reqs_c}
        if len(levels) > 1:
            raise ValueError("one LZ4 level per server")
        with torch.cuda.stream(s):
            if slot.reqs_c:
                ch = [bsgpu.Chunk(r.data.data_ptr(), base + r.out_off, r.n_elem, 0,
                                  r.stream_cap(), r.elem_size, r.block_elems, self._index_ptr(r))
                      for r in slot.reqs_c]
                table, n_items, ws = bsgpu.batch_plan(bsgpu.OP_COMPRESS, ch)
                slot.h_table_c[:table.numel()].copy_(table)
                slot.d_table_c[:table.numel()].copy_(slot.h_table_c[:table.numel()],
                                                     non_blocking=True)
                wsb = slot.workspace("c", ws, self.device)
                bsgpu.compress_batch(slot.d_table_c, len(ch), n_items, slot.out_bytes,
                                     None, slot.status_c, wsb, levels.pop(),
                                     self.ctas_per_sm, s)
                k = len(ch)
                slot.h_out_bytes[:k].copy_(slot.out_bytes[:k], non_blocking=True)
                slot.h_status_c[:k].copy_(slot.status_c[:k], non_blocking=True)
            if slot.reqs_d:
                ch = [bsgpu.Chunk(r.data.data_ptr(), base + r.out_off, r.n_elem, r.data.numel(),
                                  0, r.elem_size, r.block_elems, self._index_ptr(r))
                      for r in slot.reqs_d]
                table, n_items, ws = bsgpu.batch_plan(bsgpu.OP_DECOMPRESS, ch)
                slot.h_table_d[:table.numel()].copy_(table)
                slot.d_table_d[:table.numel()].copy_(slot.h_table_d[:table.numel()],
                                                     non_blocking=True)
                wsb = slot.workspace("d", ws, self.device)
                # requests without an index have their block chains walked first
                bsgpu.decompress_batch(slot.d_table_d, len(ch), n_items, None, None,
                                       slot.status_d, wsb, self.ctas_per_sm, s)
                k = len(ch)
                slot.h_status_d[:k].copy_(slot.status_d[:k], non_blocking=True)
            slot.event.record(s)
        self.inflight.append(slot)
        self.batches.append((now, len(slot.reqs_c), len(slot.reqs_d)))
        return True

    def _retire(self, now) -> int:
        n = 0
        while self.inflight and self.inflight[0].event.query():
            slot = self.inflight.popleft()
            t = now
            for k, r in enumerate(slot.reqs_c):
                r.status = int(slot.h_status_c[k])
                r.out_len = int(slot.h_out_bytes[k])
                self._finish(r, t)
            for k, r in enumerate(slot.reqs_d):
                r.status = int(slot.h_status_d[k])
                r.out_len = r.n_elem * r.elem_size
                self._finish(r, t)
            n += len(slot.reqs_c) + len(slot.reqs_d)
            slot.reqs_c, slot.reqs_d = [], []
            self.free_slots.append(slot)
        return n


class SerialServer(_Server):
    """The plain pipeline: one request at a time, in arrival order, through
    the single-stream calls (bsgpu_compress / bsgpu_decompress, called
    directly so that nothing is allocated per request); the next starts when
    the previous has completed."""

    def __init__(self, cap_bytes: int = 40 << 30, device="cuda", on_done=None):
        super().__init__(cap_bytes, device, on_done)
        self.cur = None
        self.event = torch.cuda.Event()
        self.nb_dev = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.h_nb = torch.zeros(1, dtype=torch.int64).pin_memory()
        self.h_st = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.ws = bsgpu.new_workspace(1 << 20, self.device)

    def _busy(self) -> bool:
        return self.cur is not None

    def _ws(self, nbytes):
        if self.ws.numel() < nbytes:
            self.ws = bsgpu.new_workspace(nbytes, self.device)
        return self.ws

    def _launch(self, waiting, now) -> bool:
        if self.cur is not None or not self._reserve(waiting[0]):
            return False
        r = waiting.popleft()
        r.admitted = now
        s = self.stream
        out = self.pool.data_ptr() + r.out_off
        lib = bsgpu._lib
        with torch.cuda.stream(s):
            if r.kind == "compress":
                ws = self._ws(bsgpu.workspace_size(bsgpu.OP_COMPRESS, r.n_elem, r.elem_size,
                                                   r.block_elems))
                bsgpu._check(lib.bsgpu_compress(r.data.data_ptr(), r.n_elem, r.elem_size,
                                                r.block_elems, r.level, out, r.stream_cap(),
                                                self.nb_dev.data_ptr(), self._index_ptr(r),
                                                ws.data_ptr(), ws.numel(), s.cuda_stream),
                             "bsgpu_compress")
                self.h_nb.copy_(self.nb_dev, non_blocking=True)
            else:
                ws = self._ws(bsgpu.workspace_size(bsgpu.OP_DECOMPRESS, r.n_elem, r.elem_size,
                                                   r.block_elems))
                bsgpu._check(lib.bsgpu_decompress(r.data.data_ptr(), r.data.numel(), out,
                                                  r.n_elem, r.elem_size, r.block_elems,
                                                  self._index_ptr(r), ws.data_ptr(), ws.numel(),
                                                  s.cuda_stream), "bsgpu_decompress")
            self.h_st.copy_(ws[:4].view(torch.int32), non_blocking=True)
            self.event.record(s)
        self.cur = r
        return True

    def _retire(self, now) -> int:
        if self.cur is None or not self.event.query():
            return 0
        r, self.cur = self.cur, None
        r.status = int(self.h_st[0])
        r.out_len = int(self.h_nb[0]) if r.kind == "compress" else r.n_elem * r.elem_size
        self._finish(r, now)
        return 1
