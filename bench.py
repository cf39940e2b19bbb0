"""Benchmark: compress + decompress of a CHIME-Pathfinder-shaped visibility cube.

One step = the whole hot path on one batch: precision reduction (Sec. 3),
Bitshuffle + LZ4 with framing (Sec. 4) in one fused pass, then LZ4 decode +
un-Bitshuffle of the stream (the inverse), all through the C-ABI.

Workload: 1024 freq x 8256 products (128 inputs) x 16 time samples of
complex64 (1.08 GB), N = 2^17, f = 0.01, seed = rank; synthetic data (the
CHIME data of Sec. 5 is not available).  The input (1.08 GB) is larger than
L2 (129 MB), so nothing is flushed between steps.

value = uncompressed bytes of all ranks / (max over ranks of the timed
region) in GB/s.  Ranks are independent replicas on their own cubes (weak
scaling; no collective on the data path).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl bsgpu|reference]

``--workload serve`` measures serving: Poisson arrivals, 70 % compress and
30 % decompress requests of rounded visibility data with sizes log-uniform in
[16 KiB, 256 MiB], admission capped at 40 GB of device memory; p50/p99
latency and GB/s of the continuous-batching server against the
one-at-a-time pipeline, with the arrival rate swept up to saturation.

``--workload batch`` measures the batched engine instead: 4096 chunks of
log-uniform sizes in [64 KiB, 64 MiB] (about 40 GB), element sizes 2, 4 or 8
bytes at random, half rounded visibility cubes (16 inputs x 64 time
samples, N = 2^16, f = 0.01) and half random walks, compressed and
decompressed by one persistent launch each, replayed from a CUDA graph.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "compress+decompress GB/s (uncompressed bytes) & % HBM roofline; served p50/p99 latency"
WORKLOAD = "chime-pathfinder-shaped visibilities 1024 freq x 8256 prod (128 inputs) x 16 time c64"
BLOCK_ELEMS = 2048   # 8192-byte blocks of float32 components
LEVEL = 0            # LZ4 search level


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="bsgpu", choices=["bsgpu", "reference"])
    p.add_argument("--f", type=float, default=0.01)
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--cpu-freqs", type=int, default=128,
                   help="frequencies of the cube the oracle baseline processes")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--freqs", type=int, default=1024,
                   help="frequencies of the cube (1024 = the full workload; fewer only for "
                        "profiling runs)")
    p.add_argument("--workload", default="chime",
                   choices=["chime", "batch", "serve", "shuffle", "round"] + sorted(VARIANTS))
    p.add_argument("--requests", type=int, default=3000,
                   help="serve workload: requests per arrival-rate point")
    p.add_argument("--chunks", type=int, default=4096,
                   help="batch workload: number of chunks (4096 = the full workload)")
    p.add_argument("--sub-chunks", type=int, default=1024,
                   help="chunks of the batch record in the default run's line")
    p.add_argument("--sub-requests", type=int, default=800,
                   help="requests per point of the serving record in the default run's line")
    p.add_argument("--no-sweep", action="store_true",
                   help="shuffle workload: leave out the codec-only size x block grid")
    p.add_argument("--no-sub", action="store_true",
                   help="leave the batch and serving records out of the default run's line")
    p.add_argument("--batch-fixed", default="",
                   help="BLOCK_BYTES:WxC -- the batch workload with this one block size and "
                        "launch shape (W warps per CTA, C CTAs per SM, 0 = as many as fit) "
                        "instead of the autotuner's choice; for profiling one launch shape")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# -- clocks sampled while the GPU works ---------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            if not (t0 <= ts <= t1):
                continue
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# -- the oracle as the CPU baseline / reference arm ---------------------------

def oracle_round_trip(cfg, n_freq, f, seed):
    """Oracle (plain C, one core): round + compress + decompress of the first
    n_freq frequencies of the cube; returns (bytes, seconds, ratio)."""
    import oracle
    from paper_1503_00638_gb300 import synth
    vis = synth.visibilities(cfg, 0, n_freq)
    t0 = time.perf_counter()
    r = oracle.reduce_precision_c64(vis, cfg.n_samp, f)
    flat = r.view(np.float32).reshape(-1)
    s = oracle.compress(flat, BLOCK_ELEMS)
    rc, back = oracle.decompress(s, flat.size, np.float32, BLOCK_ELEMS)
    dt = time.perf_counter() - t0
    if rc != 0 or not np.array_equal(back.view(np.uint32), flat.view(np.uint32)):
        raise RuntimeError("oracle round trip failed")
    return vis.nbytes, dt, len(s) / vis.nbytes


def oracle_round_trip_cores(cfg, n_freq, f, threads):
    """The same oracle round trip over all host cores: the frequencies split
    into `threads` slabs, each rounded, compressed into its own stream and
    decompressed by one thread (the oracle's C calls release the GIL), as
    the paper runs blocks in parallel over cores.  Returns (bytes, seconds)."""
    import concurrent.futures as cf
    import oracle
    from paper_1503_00638_gb300 import synth
    vis = synth.visibilities(cfg, 0, n_freq)
    edges = [n_freq * k // threads for k in range(threads + 1)]
    slabs = [(edges[k], edges[k + 1]) for k in range(threads) if edges[k + 1] > edges[k]]

    def work(ab):
        a, b = ab
        r = oracle.reduce_precision_c64(vis[a:b], cfg.n_samp, f)
        flat = r.view(np.float32).reshape(-1)
        s = oracle.compress(flat, BLOCK_ELEMS)
        rc, back = oracle.decompress(s, flat.size, np.float32, BLOCK_ELEMS)
        return rc == 0 and np.array_equal(back.view(np.uint32), flat.view(np.uint32))

    with cf.ThreadPoolExecutor(max_workers=len(slabs)) as ex:
        t0 = time.perf_counter()
        ok = all(ex.map(work, slabs))
        dt = time.perf_counter() - t0
    if not ok:
        raise RuntimeError("oracle round trip failed")
    return vis.nbytes, dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def run_reference(args, rank):
    from paper_1503_00638_gb300 import synth
    if rank != 0:
        return
    cfg = synth.VisConfig(1024, 128, 16, 2 ** 17, args.f, seed=0, drift=True)
    # size each step's sample so that the whole run stays near two minutes
    _, t8, _ = oracle_round_trip(cfg, 8, args.f, 0)
    per_freq = t8 / 8
    nf = int(120.0 / (args.steps + 0.25 * args.warmup) / per_freq)
    nf = max(1, min(args.cpu_freqs, nf))
    for _ in range(args.warmup):
        oracle_round_trip(cfg, max(1, nf // 4), args.f, 0)
    times, nbytes = [], 0
    for _ in range(args.steps):
        nbytes, dt, ratio = oracle_round_trip(cfg, nf, args.f, 0)
        times.append(dt)
    total = sum(times)
    value = nbytes * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"first {nf} of 1024 frequencies",
                   "f": args.f, "N": 2 ** 17, "block_bytes": BLOCK_ELEMS * 4},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{nf} of 1024 frequencies ({nbytes / 1e6:.1f} MB) per step"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "ratio": ratio,
    }
    print(json.dumps(line), flush=True)


# -- traffic recorded from an ncu capture of the current kernel source ----------

# the sources the profiled compress kernel is compiled from
KERNEL_SOURCES = ("kernels.cu", "kernels.cuh", "compress_fast.cuh", "codec.cuh", "common.cuh",
                  "lz4_warp.cuh", "shuffle.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1503_00638_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_profile(scale_units, key="dram_bytes_per_launch"):
    """A per-launch figure of the compress kernel from profiles/traffic.json
    (DRAM bytes, or warp instructions with key="inst_per_launch"), if it was
    taken on the current kernel source; scaled to this launch."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash() or key not in d:
        return None
    return d[key] / d["units_per_launch"] * scale_units


def recorded_traffic(scale_units):
    return recorded_profile(scale_units)


def issue_peak_ginst(sm_mhz):
    """Warp instructions per second the SMs can issue: 4 schedulers per SM,
    one instruction per scheduler per cycle."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return sms * 4 * (sm_mhz or 2070.0) * 1e6 / 1e9


# -- the batched-engine workload ------------------------------------------------

BATCH_WORKLOAD = ("batch of 4096 chunks, log-uniform 64 KiB..64 MiB (~40 GB), elem 2/4/8 B, "
                  "half rounded visibilities (16 inputs x 64 time), half random walks")
BATCH_BLOCK_BYTES = 8192                     # the serving workload's block size
BATCH_BLOCK_CANDIDATES = (2048, 4096, 8192)  # the batch autotuner's block sizes (bytes)


def batch_specs(n_chunks, seed):
    """(bytes, elem size, kind) per chunk; sizes log-uniform on [64 KiB, 64 MiB]."""
    from paper_1503_00638_gb300 import synth
    return synth.batch_specs(n_chunks, seed)


def batch_inputs(specs, seed, device="cuda", keep_raw=False):
    """Device buffers of the chunks: rounded visibility cubes (16 inputs x 64
    time, as many frequencies as the size needs, cut to size) or random walks.
    With keep_raw, also {chunk: (host cube, config)} for the smallest
    visibility chunk of each element size (for the oracle's check of the
    rounding)."""
    import torch
    from paper_1503_00638_gb300 import bsgpu, synth
    xs, raw, keep = [], {}, {}
    for k, (nb, es, kind) in enumerate(specs):
        if kind == "vis" and (es not in keep or nb < specs[keep[es]][0]):
            keep[es] = k
    per_freq = synth.n_products(16) * 64 * 8
    for k, (nb, es, kind) in enumerate(specs):
        if kind == "vis":
            F = -(-nb // per_freq)
            cfg = synth.VisConfig(F, 16, 64, 2 ** 16, 0.01, seed=seed * 100003 + k)
            cube = synth.visibilities_torch(cfg, device)
            r = bsgpu.reduce_precision_c64(cube, cfg.n_samp, cfg.f)
            x = r.view(torch.uint8).reshape(-1)[:nb].clone()
            if keep_raw and keep.get(es) == k:
                raw[k] = (cube.cpu().numpy(), cfg)
            del cube, r
        else:
            x = synth.random_walk_torch(nb // es, es, seed=seed * 100003 + k, device=device)
        xs.append(x)
    return (xs, raw) if keep_raw else xs


def oracle_batch_checks(eng, xs, specs, raw, block_bytes):
    """The oracle against the batch run: the GPU rounding of the smallest
    visibility chunk of each element size against the oracle's rounding of
    its raw cube, and the oracle's strict decoder on the GPU stream of the
    smallest chunk of every (element size, kind) pair."""
    import oracle
    rounding_ok = True
    for k, (cube, cfg) in raw.items():
        want = oracle.reduce_precision_c64(cube, cfg.n_samp, cfg.f).view(np.uint8).reshape(-1)
        rounding_ok &= bool(np.array_equal(xs[k].cpu().numpy(), want[:specs[k][0]]))
    pick = {}
    for k, (nb, es, kind) in enumerate(specs):
        if (es, kind) not in pick or nb < specs[pick[(es, kind)]][0]:
            pick[(es, kind)] = k
    udt = {2: np.uint16, 4: np.uint32, 8: np.uint64}
    decode_ok = True
    for (es, kind), k in pick.items():
        a = xs[k].cpu().numpy().view(udt[es])
        rc, back = oracle.decompress(eng.stream(k).cpu().numpy().tobytes(), a.size, a.dtype,
                                     block_bytes // es)
        decode_ok &= rc == 0 and bool(np.array_equal(back, a))
    return {"rounding_vs_oracle": {"chunks": len(raw), "bit_exact": rounding_ok},
            "oracle_decodes": {"chunks": len(pick),
                               "pairs": sorted(f"{es}B-{kind}" for es, kind in pick),
                               "exact": decode_ok}}


def oracle_batch_sample(xs, specs, block_bytes=BATCH_BLOCK_BYTES, seconds=15.0):
    """The oracle compressing and decompressing whole chunks, in order, until
    about `seconds` have passed; returns (bytes, seconds, chunks)."""
    import oracle
    done, t_used, n = 0, 0.0, 0
    for x, (nb, es, _) in zip(xs, specs):
        a = x.cpu().numpy().view({2: np.uint16, 4: np.uint32, 8: np.uint64}[es])
        t0 = time.perf_counter()
        s = oracle.compress(a, block_bytes // es)
        rc, back = oracle.decompress(s, a.size, a.dtype, block_bytes // es)
        t_used += time.perf_counter() - t0
        if rc != 0 or not np.array_equal(back, a):
            raise RuntimeError("oracle round trip failed")
        done += nb
        n += 1
        if t_used > seconds:
            break
    return done, t_used, n


def run_batch(args, rank, world, local, barrier, gpu_index, chunks=None, steps=None,
              warmup=None, cpu=True):
    """The batched engine on `chunks` chunks of the batch generator: the
    autotuner picks the block size and each launch's shape, then compress +
    decompress of the whole batch is timed as one CUDA-graph replay per step.
    Returns the record (rank 0 prints it for --workload batch)."""
    import torch
    import torch.distributed as dist
    from paper_1503_00638_gb300 import bsgpu, engine

    chunks = chunks or args.chunks
    steps = steps or args.steps
    warmup = args.warmup if warmup is None else warmup
    specs = batch_specs(chunks, rank)
    xs, raw = batch_inputs(specs, rank, keep_raw=True)
    es_l = [es for _, es, _ in specs]
    nbytes = sum(nb for nb, _, _ in specs)
    if args.batch_fixed:
        # one given launch, no tuning (profiles of a single launch shape)
        fb, fs = args.batch_fixed.split(":")
        fw, fc = (int(v) for v in fs.split("x"))
        block_bytes = int(fb)
        shape = {"warps_per_cta": fw, "ctas_per_sm": fc}
        tune_table = {block_bytes: {"compress": dict(shape), "decompress": dict(shape),
                                    "note": "fixed by --batch-fixed, not tuned"}}
    else:
        # the autotuner: block size x warps per CTA x CTAs per SM, each launch
        # tuned on its own (one codec at a time, so that a 40 GB batch fits)
        block_bytes, tune_table, _ = engine.tune(xs, es_l, BATCH_BLOCK_CANDIDATES, level=LEVEL,
                                                 reps=2, keep=False)
    torch.cuda.empty_cache()
    bl = [block_bytes // es for es in es_l]
    eng = engine.BatchCodec(xs, es_l, bl, level=LEVEL)
    chosen = tune_table[block_bytes]
    eng.warps_c, eng.ctas_c = chosen["compress"]["warps_per_cta"], chosen["compress"]["ctas_per_sm"]
    eng.warps_d, eng.ctas_d = (chosen["decompress"]["warps_per_cta"],
                               chosen["decompress"]["ctas_per_sm"])
    eng.compress()
    eng.decompress()
    sc, sd = eng.statuses()
    if any(sc) or any(sd):
        raise RuntimeError("batch status after tuning")
    # correctness of what is timed: sampled chunks round-trip exactly
    for i in range(0, eng.n, max(1, eng.n // 64)):
        if not torch.equal(eng.output(i), xs[i]):
            raise RuntimeError(f"batch round trip failed on chunk {i}")
    slen = eng.compressed_bytes()
    graph = eng.capture()
    stream = torch.cuda.current_stream()

    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    for _ in range(warmup):
        graph.replay()
    t_soak0 = time.time()
    torch.cuda.synchronize()
    # split timing of the two launches (eager, events on the launching stream)
    c_ms, d_ms = [], []
    for _ in range(3):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        eng.compress(stream)
        e1.record(stream)
        eng.decompress(stream)
        e2.record(stream)
        e2.synchronize()
        c_ms.append(e0.elapsed_time(e1))
        d_ms.append(e1.elapsed_time(e2))
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        graph.replay()
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall1 = time.time()
    ms = start.elapsed_time(end)
    sc, sd = eng.statuses()
    if any(sc) or any(sd):
        raise RuntimeError("batch status after timed steps")
    clk = clocks.summary(t_soak0, t_wall1)
    clocks.stop()
    ms_t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = nbytes * world * steps / (ms_max / 1e3) / 1e9

    hbm, peak_kind = peaks()
    cm, dm = statistics.median(c_ms), statistics.median(d_ms)
    alg_c = nbytes + slen + 8 * eng.n_items + 8 * eng.n
    alg_d = slen + 8 * eng.n_items + nbytes
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms_max / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD if chunks == 4096
                   else f"{BATCH_WORKLOAD} (first {chunks} chunks, {nbytes / 1e9:.1f} GB)",
                   "chunks": eng.n, "items": eng.n_items, "bytes": nbytes,
                   "block_bytes": block_bytes, "level": LEVEL,
                   "launch": {"compress": {"warps_per_cta": eng.warps_c,
                                           "ctas_per_sm": eng.ctas_c},
                              "decompress": {"warps_per_cta": eng.warps_d,
                                             "ctas_per_sm": eng.ctas_d}},
                   "autotuner": {"block_bytes_candidates": list(BATCH_BLOCK_CANDIDATES),
                                 "shapes": [f"{w}x{k}" for w, k in engine.SHAPES],
                                 "shape_note": "WxC = W warps per CTA, C CTAs per SM (0 = as "
                                               "many as fit)",
                                 "rule": "fastest round trip among block sizes within 2% of "
                                         "the smallest compressed size",
                                 "per_block_bytes": tune_table},
                   "l2": f"inputs ({nbytes / 1e9:.1f} GB) larger than L2; no flush",
                   "step": "compress + decompress batch, one CUDA-graph replay",
                   "parallelism": f"replicas x{world}"},
        "compress_gbs": nbytes / (cm / 1e3) / 1e9,
        "decompress_gbs": nbytes / (dm / 1e3) / 1e9,
        "ratio": slen / nbytes,
        "roofline": {"bound": "hbm", "kernel": "compress_batch_kernel",
                     "achieved": alg_c / (cm / 1e3) / 1e9, "peak": hbm, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": alg_c / (cm / 1e3) / 1e9 / hbm, "traffic": None,
                     "algorithmic_bytes": alg_c},
        "decompress_roofline": {"bound": "hbm", "kernel": "decompress_batch_kernel",
                                "achieved": alg_d / (dm / 1e3) / 1e9, "peak": hbm,
                                "unit": "GB/s", "frac": alg_d / (dm / 1e3) / 1e9 / hbm},
        "gpu_launches": 2 * steps,
        "clocks": clk,
        "wall_s_timed": t_wall1 - t_wall0,
    }
    if rank == 0:
        line["parity"] = oracle_batch_checks(eng, xs, specs, raw, block_bytes)
    if rank == 0 and world == 1 and cpu and not args.no_cpu_baseline:
        nb_cpu, dt, n_cpu = oracle_batch_sample(xs, specs, block_bytes)
        line["cpu_baseline"] = {"value": nb_cpu / dt / 1e9, "unit": "GB/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"first {n_cpu} chunks ({nb_cpu / 1e6:.1f} MB): "
                                          "compress+decompress"}
    return line


# -- the serving workload --------------------------------------------------------

SERVE_WORKLOAD = ("serving: Poisson arrivals, 70% compress / 30% decompress, rounded "
                  "visibilities (16 inputs x 64 time), sizes log-uniform 16 KiB..256 MiB, "
                  "admission cap 40 GB")


def serve_pool(n_payloads, seed):
    """Distinct request payloads (rounded visibility bytes, 4-byte elements)
    with their compressed streams and block indexes."""
    import torch
    from paper_1503_00638_gb300 import bsgpu
    rng = np.random.default_rng([seed, 5])
    sizes = np.exp(rng.uniform(np.log(16 << 10), np.log(256 << 20), n_payloads)).astype(np.int64)
    specs = [(int(b) // 4 * 4, 4, "vis") for b in sizes]
    xs = batch_inputs(specs, seed + 17)
    comp = []
    for x in xs:
        c = bsgpu.compress(x, BATCH_BLOCK_BYTES // 4, elem_size=4)
        comp.append((c.buf[:c.nbytes].clone(), c.offsets.clone()))
        del c
    torch.cuda.synchronize()
    return xs, comp


def serve_requests(xs, comp, n, rate, seed):
    from paper_1503_00638_gb300 import serve
    rng = np.random.default_rng([seed, 6])
    t = 0.0
    reqs = []
    for i in range(n):
        if rate:
            t += rng.exponential(1.0 / rate)
        k = int(rng.integers(len(xs)))
        x = xs[k]
        if rng.random() < 0.7:
            reqs.append(serve.Request(i, "compress", t, x, x.numel() // 4, 4,
                                      BATCH_BLOCK_BYTES // 4))
        else:
            st, idx = comp[k]
            reqs.append(serve.Request(i, "decompress", t, st, x.numel() // 4, 4,
                                      BATCH_BLOCK_BYTES // 4, index=idx))
    return reqs


def batch_launch(rec):
    """Block size and launch shapes a batch record chose (for its end-to-end step)."""
    lc = rec["config"]["launch"]
    return {"block_bytes": rec["config"]["block_bytes"],
            "shapes": ((lc["compress"]["warps_per_cta"], lc["compress"]["ctas_per_sm"]),
                       (lc["decompress"]["warps_per_cta"], lc["decompress"]["ctas_per_sm"]))}


def run_batch_e2e(args, chunks, launch):
    """End to end with host buffers through `hostio.HostBatchCodec` on the
    leading chunks of the batch generator up to 4 GB (pinned host copies of
    the whole 40 GB are not kept): inputs, streams with their lengths and
    block index, and outputs all cross the host link.  Measured as a step of
    its own, after the other batch and serving measurements of the run."""
    import torch
    from paper_1503_00638_gb300 import hostio
    specs = batch_specs(chunks, 0)
    sub, acc = 0, 0
    while sub < len(specs) and acc + specs[sub][0] <= (4 << 30):
        acc += specs[sub][0]
        sub += 1
    sub = max(sub, 1)
    xs_sub = batch_inputs(specs[:sub], 0)
    es_l = [es for _, es, _ in specs[:sub]]
    bl = [launch["block_bytes"] // es for es in es_l]
    h_in = [x.reshape(-1).view(torch.uint8).cpu().pin_memory() for x in xs_sub]
    del xs_sub
    h_out = [torch.empty_like(h).pin_memory() for h in h_in]
    hb = hostio.HostBatchCodec([h.numel() for h in h_in], es_l, bl, level=LEVEL,
                               launch=launch["shapes"])
    e2e_t = []
    sub_bytes = sum(specs[i][0] for i in range(sub))
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hb.round_trip(h_in, h_out)
        if k:
            e2e_t.append(time.perf_counter() - t0)
    ok = all(torch.equal(h_out[i], h_in[i]) for i in range(0, sub, 7))
    ok = ok and all(sc == [0] * len(sc) and sd == [0] * len(sd) for sc, sd in hb.statuses())
    h2d, d2h = hb.bytes_moved()
    del hb, h_in, h_out
    torch.cuda.empty_cache()
    return {"value": sub_bytes / statistics.median(e2e_t) / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "chunks": sub,
            "round_trip_ok": ok,
            "api": "hostio.HostBatchCodec.round_trip (groups of about 512 MB, pipelined; "
                   "streams, lengths and block index through host memory)"}


def run_serve(args, rank, world, gpu_index, requests=None, payloads=256):
    """Serving: the continuous-batching server and the one-at-a-time
    pipeline on the same request lists (every request present at t = 0, then
    Poisson arrivals at 0.1 .. 0.9 of the batching server's saturation).
    Returns the record."""
    import torch
    from paper_1503_00638_gb300 import serve
    n_req = requests or args.requests
    xs, comp = serve_pool(payloads, rank)
    mean_bytes = statistics.mean(x.numel() for x in xs)   # payloads are drawn uniformly
    cap = 40 << 30
    bsrv = serve.BatchingServer(cap_bytes=cap, depth=2)
    ssrv = serve.SerialServer(cap_bytes=cap)
    for srv in (bsrv, ssrv):          # warm-up (kernel attributes, workspaces)
        srv.run(serve_requests(xs, comp, 64, 0.0, 99))
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    t_0 = time.time()
    # saturation: every request present at t = 0
    # both servers run the identical request list at every point
    sat_b = serve.latency_summary(bsrv.run(serve_requests(xs, comp, n_req, 0.0, 1)))
    sat_s = serve.latency_summary(ssrv.run(serve_requests(xs, comp, n_req, 0.0, 1)))
    lam_sat = sat_b["gbs"] * 1e9 / mean_bytes
    sweep = []
    for frac in (0.1, 0.3, 0.5, 0.7, 0.9):
        lam = frac * lam_sat
        point = {"rate_per_s": lam, "offered_gbs": lam * mean_bytes / 1e9, "frac_of_sat": frac}
        rb = bsrv.run(serve_requests(xs, comp, n_req, lam, 2))
        point["batching"] = serve.latency_summary(rb)
        point["batching"]["batches"] = len(bsrv.batches)
        bsrv.batches.clear()
        rs = ssrv.run(serve_requests(xs, comp, n_req, lam, 2))
        point["serial"] = serve.latency_summary(rs)
        for r in rb + rs:
            if r.status != 0:
                raise RuntimeError(f"request {r.rid} status {r.status}")
        sweep.append(point)
    t_1 = time.time()
    clk = clocks.summary(t_0, t_1)
    clocks.stop()
    half = [p for p in sweep if p["frac_of_sat"] == 0.5][0]
    line = {
        "metric": METRIC, "value": sat_b["gbs"], "unit": "GB/s", "n_gpus": world,
        "steps": n_req, "warmup": 64, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD, "payloads": len(xs), "requests": n_req,
                   "same_requests": "both servers run the identical request list at every point",
                   "mean_request_bytes": mean_bytes, "block_bytes": BATCH_BLOCK_BYTES,
                   "admission_cap_bytes": cap, "batch_depth": 2,
                   "value": "batching server GB/s with every request present at t = 0",
                   "parallelism": f"replicas x{world}"},
        "serving": {"saturation": {"batching": sat_b, "serial": sat_s},
                    "p50_ms_at_half_saturation": {"batching": half["batching"]["p50_ms"],
                                                  "serial": half["serial"]["p50_ms"]},
                    "p99_ms_at_half_saturation": {"batching": half["batching"]["p99_ms"],
                                                  "serial": half["serial"]["p99_ms"]},
                    "sweep": sweep},
        "clocks": clk,
    }
    return line


# -- variants of the visibility path (the int32 path, the fused reorder, the
#    compensated f, 8-byte samples, the full covariance) ------------------------

VARIANTS = {
    "chime-int32": {"dtype": "i32", "es": 4, "tslow": False, "comp": False, "full": False,
                    "what": "int32 (re, im) cube (the CHIME-shaped cube x 4096, rounded to integers)"},
    "chime-tslow": {"dtype": "f32", "es": 4, "tslow": True, "comp": False, "full": False,
                    "what": "complex64 cube in the instrument's order [T][F][P], reorder fused"},
    "chime-compensated": {"dtype": "f32", "es": 4, "tslow": False, "comp": True, "full": False,
                          "what": "complex64 cube, compensated f of Sec. 3.2 per sample"},
    "chime-samples8": {"dtype": "f32", "es": 8, "tslow": False, "comp": False, "full": False,
                       "what": "complex64 cube bitshuffled as 8-byte samples"},
    "chime-tslow-t40": {"dtype": "f32", "es": 4, "tslow": True, "comp": False, "full": False,
                        "F": 512, "T": 40,
                        "what": "complex64 cube of 512 freq x 8256 products x 40 time in the "
                                "instrument's [T][F][P] order, reorder fused"},
    "chime-t40": {"dtype": "f32", "es": 4, "tslow": False, "comp": False, "full": False,
                  "F": 512, "T": 40,
                  "what": "complex64 cube of 512 freq x 8256 products x 40 time (a time axis "
                          "that is not a multiple of 16)"},
    "fullcov8": {"dtype": "f32", "es": 4, "tslow": False, "comp": False, "full": True, "n_in": 8,
                 "what": "8-input array, 1024 freq x 36 products x 64 time, full covariance"},
    "fullcov16": {"dtype": "f32", "es": 4, "tslow": False, "comp": False, "full": True,
                  "n_in": 16,
                  "what": "16-input array, 1024 freq x 136 products x 64 time, full covariance"},
}


def run_variant(args, rank, world, gpu_index, barrier):
    import torch
    import torch.distributed as dist
    import numpy as _np
    from paper_1503_00638_gb300 import bsgpu, synth
    v = VARIANTS[args.workload]
    if v["full"]:
        cfg = synth.VisConfig(1024, v["n_in"], 64, 2 ** 16, args.f, seed=rank, rho=0.5)
        host = synth.visibilities_physical(cfg)
    else:
        cfg = synth.VisConfig(v.get("F", 1024), 128, v.get("T", 16), 2 ** 17, args.f, seed=rank,
                              drift=True)
        host = synth.visibilities_int(cfg, 4096.0) if v["dtype"] == "i32" else synth.visibilities(cfg)
    F, n_in, T = cfg.n_freq, cfg.n_inputs, cfg.n_time
    host_in = _np.ascontiguousarray(_np.moveaxis(host, 2, 0)) if v["tslow"] else host
    nbytes = host.nbytes
    es = v["es"]
    B = 8192 // es
    n_el = nbytes // es
    flags = ((bsgpu.VIS_COMPENSATE if v["comp"] else 0) |
             (bsgpu.VIS_TIME_SLOWEST if v["tslow"] else 0) |
             (bsgpu.VIS_FULL_COV if v["full"] else 0))
    dt = bsgpu.VIS_I32 if v["dtype"] == "i32" else bsgpu.VIS_F32
    pin = torch.from_numpy(host_in).pin_memory()
    d_in = pin.cuda()
    stream = torch.cuda.current_stream()
    cap = bsgpu.compress_bound(n_el, es, B)
    nblk = bsgpu.num_blocks(n_el, es, B)
    comp = torch.empty(cap, dtype=torch.uint8, device="cuda")
    offs = torch.empty(max(nblk, 1), dtype=torch.int64, device="cuda")
    nb_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws_c = bsgpu.new_workspace(bsgpu.vis_workspace_size_ex(bsgpu.OP_COMPRESS_VIS, F, n_in, T, es,
                                                           B, flags))
    ws_d = bsgpu.new_workspace(bsgpu.workspace_size(bsgpu.OP_DECOMPRESS, n_el, es, B))
    dec = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    lib = bsgpu._lib

    def compress():
        bsgpu._check(lib.bsgpu_compress_vis_ex(
            d_in.data_ptr(), dt, F, n_in, T, cfg.n_samp, cfg.f, flags, es, B, LEVEL,
            comp.data_ptr(), cap, nb_dev.data_ptr(), offs.data_ptr(), ws_c.data_ptr(),
            ws_c.numel(), stream.cuda_stream), "bsgpu_compress_vis_ex")

    def decompress(slen):
        bsgpu._check(lib.bsgpu_decompress(
            comp.data_ptr(), slen, dec.data_ptr(), n_el, es, B, offs.data_ptr(), ws_d.data_ptr(),
            ws_d.numel(), stream.cuda_stream), "bsgpu_decompress")

    compress()
    slen = int(nb_dev.item())
    decompress(slen)
    torch.cuda.synchronize()
    if bsgpu.status(ws_c) or bsgpu.status(ws_d):
        raise RuntimeError("variant status")
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        compress()
        decompress(slen)
    torch.cuda.synchronize()
    # soak ~1 s under load so the clock sampler sees the working clock
    t_soak0 = time.time()
    while time.time() - t_soak0 < 1.0:
        compress()
        decompress(slen)
        torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    # inputs that fit in L2 (the full-covariance cubes) are timed cold: a
    # write of 2 x L2 before each launch, outside the launch's events
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    small = nbytes + cap < 2 * l2
    flush = torch.empty(2 * l2 if small else 0, dtype=torch.uint8, device="cuda")
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        if small:
            flush.zero_()
        evs[k][0].record(stream)
        compress()
        evs[k][1].record(stream)
        if small:
            flush.zero_()
        evs[k][2].record(stream)
        decompress(slen)
        evs[k][3].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall1 = time.time()
    clk = clocks.summary(t_soak0, t_wall1)
    clocks.stop()
    if bsgpu.status(ws_c) or bsgpu.status(ws_d):
        raise RuntimeError("variant status after timed steps")
    cm = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    dm = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    # with flushes, the step is the two launches' own time
    ms = start.elapsed_time(end) if not small else args.steps * (cm + dm)
    ms_t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    # the output is the time-fastest rounded cube
    ref = bsgpu.reduce_precision(d_in, cfg.n_samp, cfg.f, compensate=v["comp"],
                                 time_slowest=v["tslow"], full_cov=v["full"])
    ok = bool(torch.equal(ref.view(torch.uint8).reshape(-1), dec))
    # end to end, one stream: upload, compress, download the stream, upload it,
    # decompress, download the cube
    h_stream = torch.empty(cap, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    e2e_t = []
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_in.view(torch.uint8).reshape(-1).copy_(pin.view(torch.uint8).reshape(-1),
                                                 non_blocking=True)
        compress()
        L = int(nb_dev.item())
        h_stream[:L].copy_(comp[:L], non_blocking=True)
        comp[:L].copy_(h_stream[:L], non_blocking=True)
        decompress(L)
        h_out.copy_(dec, non_blocking=True)
        torch.cuda.synchronize()
        if k:
            e2e_t.append(time.perf_counter() - t0)
    hbm, peak_kind = peaks()
    autos = F * n_in * T * 4
    alg_c = nbytes + slen + nblk * 8 + autos
    alg_d = slen + nblk * 8 + nbytes
    line = {
        "metric": METRIC, "value": nbytes * world * args.steps / (ms_max / 1e3) / 1e9,
        "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i32" if v["dtype"] == "i32" else "f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {v['what']}", "f": cfg.f, "N": cfg.n_samp,
                   "elem_bytes": es, "block_bytes": 8192, "cube_bytes": nbytes,
                   "l2": (f"inputs ({nbytes / 1e9:.3f} GB) fit in L2: L2 flushed (a "
                          f"{2 * l2 / 1e6:.0f} MB write) before every timed launch"
                          if small else
                          f"inputs ({nbytes / 1e9:.2f} GB) larger than L2; no flush"),
                   "parallelism": f"replicas x{world}"},
        "compress_gbs": nbytes / (cm / 1e3) / 1e9, "decompress_gbs": nbytes / (dm / 1e3) / 1e9,
        "ratio": slen / nbytes, "round_trip_ok": ok,
        "roofline": {"bound": "hbm", "kernel": "compress (round + shuffle + LZ4)",
                     "achieved": alg_c / (cm / 1e3) / 1e9, "peak": hbm, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": alg_c / (cm / 1e3) / 1e9 / hbm, "traffic": None,
                     "algorithmic_bytes": alg_c},
        "decompress_roofline": {"bound": "hbm", "achieved": alg_d / (dm / 1e3) / 1e9,
                                "peak": hbm, "unit": "GB/s",
                                "frac": alg_d / (dm / 1e3) / 1e9 / hbm},
        "e2e": {"value": nbytes * world / statistics.median(e2e_t) / 1e9, "unit": "GB/s",
                "h2d_bytes_per_step": nbytes + slen, "d2h_bytes_per_step": slen + nbytes + 8},
        # per step: the tables, the compensated c or the full-covariance q
        # when asked, one compress kernel (no shortened block at these
        # sizes), one decompress kernel
        "gpu_launches": args.steps * (3 + int(v["comp"]) + int(v["full"])),
        "clocks": clk, "wall_s_timed": t_wall1 - t_wall0,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        fs = 2 if v["full"] else 16
        sub = host[:fs]
        t0 = time.perf_counter()
        if v["full"]:
            r = oracle.reduce_precision_full(sub, cfg.n_samp, cfg.f)
        else:
            src = oracle.reorder_time(_np.ascontiguousarray(_np.moveaxis(sub, 2, 0))) \
                if v["tslow"] else sub
            r = oracle.reduce_precision(src, cfg.n_samp, cfg.f, v["comp"])
        flat = _np.ascontiguousarray(r).view(_np.uint32 if es == 4 else _np.uint64).reshape(-1)
        st = oracle.compress(flat, B)
        rc, back = oracle.decompress(st, flat.size, flat.dtype, B)
        dt_cpu = time.perf_counter() - t0
        if rc or not _np.array_equal(back, flat):
            raise RuntimeError("oracle round trip")
        line["cpu_baseline"] = {"value": sub.nbytes / dt_cpu / 1e9, "unit": "GB/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"first {fs} of {F} frequencies ({sub.nbytes / 1e6:.1f} "
                                          "MB): round+compress+decompress"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_round(args, rank, world, gpu_index, barrier):
    """Precision reduction alone (Sec. 3, `bsgpu_reduce_precision_c64`) on the
    CHIME-shaped cube: each sample is read once and written once (16 bytes)
    beside the autos, so the kernel is HBM-bound."""
    import torch
    import torch.distributed as dist
    from paper_1503_00638_gb300 import bsgpu, synth
    cfg = synth.VisConfig(1024, 128, 16, 2 ** 17, args.f, seed=rank, drift=True)
    d = torch.from_numpy(synth.visibilities(cfg)).cuda()
    out = torch.empty_like(d)
    F, P, T = d.shape
    ws = bsgpu.new_workspace(bsgpu.vis_workspace_size(bsgpu.OP_REDUCE_PRECISION, F, 128, T))
    stream = torch.cuda.current_stream()
    hbm, peak_kind = peaks()
    for _ in range(args.warmup):
        bsgpu.reduce_precision_c64(d, cfg.n_samp, cfg.f, out=out, ws=ws)
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    # soak ~1 s under load so the clock sampler sees the working clock
    t_soak0 = time.time()
    while time.time() - t_soak0 < 1.0:
        for _ in range(20):
            bsgpu.reduce_precision_c64(d, cfg.n_samp, cfg.f, out=out, ws=ws)
        torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        evs[k][0].record(stream)
        bsgpu.reduce_precision_c64(d, cfg.n_samp, cfg.f, out=out, ws=ws)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall1 = time.time()
    clk = clocks.summary(t_soak0, t_wall1)
    clocks.stop()
    ms = [e[0].elapsed_time(e[1]) for e in evs]
    t = torch.tensor([statistics.mean(ms)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    mean_ms = float(t.item())
    nbytes = d.numel() * 8
    alg = 2 * nbytes + F * 128 * T * 4
    # sampled frequencies against the oracle (bit for bit)
    ok = bsgpu.status(ws) == 0
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        host = d.cpu().numpy()
        for fr in (0, F - 1):
            want = oracle.reduce_precision_c64(host[fr:fr + 1], cfg.n_samp, cfg.f)
            ok &= bool(np.array_equal(out[fr:fr + 1].cpu().numpy().view(np.uint32),
                                      want.view(np.uint32)))
    # the post-acquisition reorder alone (bsgpu_reorder_time) on the same
    # cube in the instrument's [T][F P] order: 16 bytes per sample moved
    ts = torch.empty((T, F, P), dtype=torch.complex64, device="cuda")
    ts.copy_(d.permute(2, 0, 1))
    back = torch.empty_like(d)
    for _ in range(args.warmup):
        bsgpu.reorder_time(ts, out=back)
    evr = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        evr[k][0].record(stream)
        bsgpu.reorder_time(ts, out=back)
        evr[k][1].record(stream)
    torch.cuda.synchronize()
    r_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evr)
    reorder_ok = bool(torch.equal(back, d))
    del ts, back
    line = {
        "metric": "precision reduction GB/s (uncompressed bytes) & % HBM roofline",
        "value": nbytes * world / (mean_ms / 1e3) / 1e9, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "round: the CHIME-shaped cube (1024 freq x 8256 products x 16 "
                               "time, complex64), f as given, out of place",
                   "f": cfg.f, "N": cfg.n_samp, "l2": "inputs (1.08 GB) larger than L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "kernel_ms": {"mean": statistics.mean(ms), "median": statistics.median(ms),
                      "best": min(ms)},
        "matches_oracle_sampled": ok,
        "reorder": {"gbs": nbytes / (r_ms / 1e3) / 1e9, "frac": 2 * nbytes / (r_ms / 1e3) / 1e9 / hbm,
                    "ms": r_ms, "round_trip_ok": reorder_ok,
                    "what": "bsgpu_reorder_time, [T][F P] -> [F P][T], complex64"},
        "roofline": {"bound": "hbm", "kernel": "reduce_precision_kernel",
                     "achieved": alg / (mean_ms / 1e3) / 1e9, "peak": hbm,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": alg / (mean_ms / 1e3) / 1e9 / hbm, "traffic": None,
                     "algorithmic_bytes": alg},
        "gpu_launches": args.steps * 2,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_shuffle(args, rank, world, gpu_index, barrier):
    """Bitshuffle and un-Bitshuffle alone (Sec. 4.2), timed separately on
    random walks of 1-, 2-, 4- and 8-byte elements (1 GiB each, 8 KiB
    blocks): every byte is read once and written once, so these kernels
    are HBM-bound.  The same arrays then go through the whole codec
    (Bitshuffle + LZ4, Sec. 4.2.1), compress and decompress timed apart."""
    import torch
    import torch.distributed as dist
    from paper_1503_00638_gb300 import bsgpu, synth
    nbytes = 1 << 30
    stream = torch.cuda.current_stream()
    hbm, peak_kind = peaks()
    per_es, fwd_ms, inv_ms = {}, [], []
    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)
    t_soak0 = time.time()
    ok_all = True
    for es in (1, 2, 4, 8):
        x = synth.random_walk_torch(nbytes // es, es, seed=rank * 16 + es)
        if x.element_size() != es:
            x = x.view({1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}[es])
        B = 8192 // es
        y, z = torch.empty_like(x), torch.empty_like(x)
        for _ in range(args.warmup):
            bsgpu.bitshuffle(x, B, out=y)
            bsgpu.bitunshuffle(y, B, out=z)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            evs[k][0].record(stream)
            bsgpu.bitshuffle(x, B, out=y)
            evs[k][1].record(stream)
            bsgpu.bitunshuffle(y, B, out=z)
            evs[k][2].record(stream)
        torch.cuda.synchronize()
        barrier()
        f_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
        i_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
        ok = bool(torch.equal(x, z))
        # the whole codec on the same array (Bitshuffle + LZ4 level 0 and back)
        n = nbytes // es
        cap, nblk = bsgpu.compress_bound(n, es, B), bsgpu.num_blocks(n, es, B)
        cbuf = torch.empty(cap, dtype=torch.uint8, device="cuda")
        offs = torch.empty(max(nblk, 1), dtype=torch.int64, device="cuda")
        nbd = torch.zeros(1, dtype=torch.int64, device="cuda")
        wsc = bsgpu.new_workspace(bsgpu.workspace_size(bsgpu.OP_COMPRESS, n, es, B))
        wsd = bsgpu.new_workspace(bsgpu.workspace_size(bsgpu.OP_DECOMPRESS, n, es, B))
        lib = bsgpu._lib

        def comp():
            bsgpu._check(lib.bsgpu_compress(x.data_ptr(), n, es, B, LEVEL, cbuf.data_ptr(), cap,
                                            nbd.data_ptr(), offs.data_ptr(), wsc.data_ptr(),
                                            wsc.numel(), stream.cuda_stream), "bsgpu_compress")

        def dec(L):
            bsgpu._check(lib.bsgpu_decompress(cbuf.data_ptr(), L, z.data_ptr(), n, es, B,
                                              offs.data_ptr(), wsd.data_ptr(), wsd.numel(),
                                              stream.cuda_stream), "bsgpu_decompress")

        comp()
        L = int(nbd.item())
        for _ in range(args.warmup):
            comp()
            dec(L)
        z.zero_()
        torch.cuda.synchronize()
        for k in range(args.steps):
            evs[k][0].record(stream)
            comp()
            evs[k][1].record(stream)
            dec(L)
            evs[k][2].record(stream)
        torch.cuda.synchronize()
        c_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
        d_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
        ok_c = bool(torch.equal(x, z)) and bsgpu.status(wsc) == 0 and bsgpu.status(wsd) == 0
        ok_all &= ok and ok_c
        fwd_ms.append(f_ms)
        inv_ms.append(i_ms)
        per_es[str(es)] = {"shuffle_gbs": nbytes / (f_ms / 1e3) / 1e9,
                           "unshuffle_gbs": nbytes / (i_ms / 1e3) / 1e9,
                           "shuffle_frac": 2 * nbytes / (f_ms / 1e3) / 1e9 / hbm,
                           "unshuffle_frac": 2 * nbytes / (i_ms / 1e3) / 1e9 / hbm,
                           "round_trip_ok": ok,
                           "codec_compress_gbs": nbytes / (c_ms / 1e3) / 1e9,
                           "codec_decompress_gbs": nbytes / (d_ms / 1e3) / 1e9,
                           "codec_ratio": L / nbytes, "codec_round_trip_ok": ok_c}
        del x, y, z, cbuf, offs, wsc, wsd
        torch.cuda.empty_cache()
    t_wall1 = time.time()
    clk = clocks.summary(t_soak0, t_wall1)
    clocks.stop()
    step_ms = sum(fwd_ms) + sum(inv_ms)
    t = torch.tensor([step_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    step_ms = float(t.item())
    f4 = fwd_ms[2]
    line = {
        "metric": "bitshuffle + unshuffle GB/s (uncompressed bytes) & % HBM roofline",
        "value": 4 * nbytes * world / (step_ms / 1e3) / 1e9,
        "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "shuffle: random walks x_{t+1} = x_t +- 2^k, k ~ U{0..6}, of 1-, "
                               "2-, 4- and 8-byte integers, 1 GiB each, 8 KiB blocks",
                   "l2": "inputs (1.07 GB) larger than L2; no flush",
                   "step": "Bitshuffle + un-Bitshuffle of each of the four arrays",
                   "parallelism": f"replicas x{world}"},
        "per_elem_size": per_es, "round_trip_ok": ok_all,
        "roofline": {"bound": "hbm", "kernel": "shuffle_kernel (4-byte elements)",
                     "achieved": 2 * nbytes / (f4 / 1e3) / 1e9, "peak": hbm,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": 2 * nbytes / (f4 / 1e3) / 1e9 / hbm, "traffic": None,
                     "algorithmic_bytes": 2 * nbytes},
        "gpu_launches": args.steps * 8,
        "clocks": clk,
    }
    if not args.no_sweep:
        line["sweep"] = codec_sweep(args, hbm)
    if rank == 0:
        print(json.dumps(line), flush=True)


SWEEP_SIZES = tuple((1 << 20) * 4 ** k for k in range(6)) + (4 * 10 ** 9,)   # 1 MiB .. 1 GiB, 4 GB
SWEEP_BLOCKS = (1024, 2048, 4096, 8192)


def codec_sweep(args, hbm):
    """The codec-only grid: uint8 / uint16 / int32 / float64 random walks of
    1 MiB to 4 GB (x4 steps) in blocks of 1024 .. 8192 elements; Bitshuffle,
    un-Bitshuffle, compress (Bitshuffle + LZ4) and decompress each timed on
    its own with CUDA events (median of the repetitions).  Sizes that fit in
    L2 are timed cold: a write of 2 x L2 precedes every timed launch.  Each
    smaller array is the start of the 4 GB one.  Every point checks both
    round trips."""
    import torch
    from paper_1503_00638_gb300 import bsgpu, synth
    stream = torch.cuda.current_stream()
    lib = bsgpu._lib
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    flush = torch.empty(2 * l2, dtype=torch.uint8, device="cuda")
    grid = []
    for es in (1, 2, 4, 8):
        nmax = max(SWEEP_SIZES) // es
        x = synth.random_walk_device(nmax, es, seed=40 + es, floating=(es == 8))
        y, z = torch.empty_like(x), torch.empty_like(x)
        cap = bsgpu.compress_bound(nmax, es, min(SWEEP_BLOCKS))
        cbuf = torch.empty(cap, dtype=torch.uint8, device="cuda")
        offs = torch.empty(bsgpu.num_blocks(nmax, es, min(SWEEP_BLOCKS)), dtype=torch.int64,
                           device="cuda")
        nbd = torch.zeros(1, dtype=torch.int64, device="cuda")
        wsc = bsgpu.new_workspace(bsgpu.workspace_size(bsgpu.OP_COMPRESS, nmax, es,
                                                       min(SWEEP_BLOCKS)))
        wsd = bsgpu.new_workspace(bsgpu.workspace_size(bsgpu.OP_DECOMPRESS, nmax, es,
                                                       min(SWEEP_BLOCKS)))
        for size in SWEEP_SIZES:
            n = size // es
            cold = size < 2 * l2
            reps = 3 if size >= (1 << 30) else 5
            for B in SWEEP_BLOCKS:
                ops = {
                    "shuffle": lambda: lib.bsgpu_bitshuffle(x.data_ptr(), y.data_ptr(), n, es, B,
                                                            stream.cuda_stream),
                    "unshuffle": lambda: lib.bsgpu_bitunshuffle(y.data_ptr(), z.data_ptr(), n, es,
                                                                B, stream.cuda_stream),
                    "compress": lambda: lib.bsgpu_compress(
                        x.data_ptr(), n, es, B, LEVEL, cbuf.data_ptr(), cap, nbd.data_ptr(),
                        offs.data_ptr(), wsc.data_ptr(), wsc.numel(), stream.cuda_stream),
                }
                times = {}
                for name in ("shuffle", "unshuffle", "compress", "decompress"):
                    if name == "decompress":
                        L = int(nbd.item())
                        fn = (lambda L=L: lib.bsgpu_decompress(
                            cbuf.data_ptr(), L, z.data_ptr(), n, es, B, offs.data_ptr(),
                            wsd.data_ptr(), wsd.numel(), stream.cuda_stream))
                    else:
                        fn = ops[name]
                    bsgpu._check(fn(), name)            # warm-up
                    if name == "unshuffle":
                        ok_sh = bool(torch.equal(z[:n * es], x[:n * es]))
                    ts = []
                    for _ in range(reps):
                        if cold:
                            flush.zero_()
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        bsgpu._check(fn(), name)
                        e1.record(stream)
                        e1.synchronize()
                        ts.append(e0.elapsed_time(e1))
                    times[name] = statistics.median(ts)
                L = int(nbd.item())
                ok_c = (bool(torch.equal(z[:n * es], x[:n * es])) and bsgpu.status(wsc) == 0
                        and bsgpu.status(wsd) == 0)
                nb = n * es
                grid.append({
                    "elem_bytes": es, "bytes": nb, "block_elems": B, "l2_cold": cold,
                    "shuffle_gbs": nb / times["shuffle"] / 1e6,
                    "shuffle_frac": 2 * nb / times["shuffle"] / 1e6 / hbm,
                    "unshuffle_gbs": nb / times["unshuffle"] / 1e6,
                    "unshuffle_frac": 2 * nb / times["unshuffle"] / 1e6 / hbm,
                    "compress_gbs": nb / times["compress"] / 1e6,
                    "compress_frac": (nb + L) / times["compress"] / 1e6 / hbm,
                    "decompress_gbs": nb / times["decompress"] / 1e6,
                    "decompress_frac": (nb + L) / times["decompress"] / 1e6 / hbm,
                    "ratio": L / nb, "round_trips_ok": ok_sh and ok_c})
        del x, y, z, cbuf, offs, wsc, wsd
        torch.cuda.empty_cache()
    return {"sizes": list(SWEEP_SIZES), "blocks": list(SWEEP_BLOCKS), "elem_bytes": [1, 2, 4, 8],
            "values": "uint8 / uint16 / int32 random walks (wrapping), float64 random walk",
            "timing": "CUDA events per launch, median of 5 (3 at 1 GiB and up); L2 flushed "
                      "before each launch when the array is under 2 x L2",
            "grid": grid}


# -- the GPU arm ----------------------------------------------------------------

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_1503_00638_gb300 import build as _build
    _build.build()
    from paper_1503_00638_gb300 import bsgpu, synth

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    gpu_index = local
    vis_dev_env = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis_dev_env:
        try:
            gpu_index = int(vis_dev_env.split(",")[local])
        except ValueError:
            gpu_index = local
    if args.workload in VARIANTS:
        run_variant(args, rank, world, gpu_index, barrier)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload == "serve":
        line = run_serve(args, rank, world, gpu_index)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload == "round":
        run_round(args, rank, world, gpu_index, barrier)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload == "shuffle":
        run_shuffle(args, rank, world, gpu_index, barrier)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload == "batch":
        line = run_batch(args, rank, world, local, barrier, gpu_index)
        line["e2e"] = run_batch_e2e(args, args.chunks, batch_launch(line))
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    cfg = synth.VisConfig(1024, 128, 16, 2 ** 17, args.f, seed=rank, drift=True)
    F, n_in, T = args.freqs, cfg.n_inputs, cfg.n_time
    vis_h = synth.visibilities(cfg, 0, F)
    nbytes = vis_h.nbytes
    n_fl = nbytes // 4
    vis_pin = torch.from_numpy(vis_h).pin_memory()
    vis = vis_pin.cuda()
    stream = torch.cuda.current_stream()

    cap = bsgpu.compress_bound(n_fl, 4, BLOCK_ELEMS)
    nblk = bsgpu.num_blocks(n_fl, 4, BLOCK_ELEMS)
    comp = torch.empty(cap, dtype=torch.uint8, device="cuda")
    offs = torch.empty(nblk, dtype=torch.int64, device="cuda")
    ws_c = bsgpu.new_workspace(bsgpu.vis_workspace_size(bsgpu.OP_COMPRESS_VIS, F, n_in, T,
                                                        BLOCK_ELEMS))
    ws_d = bsgpu.new_workspace(bsgpu.workspace_size(bsgpu.OP_DECOMPRESS, n_fl, 4, BLOCK_ELEMS))
    dec = torch.empty(nbytes, dtype=torch.uint8, device="cuda")

    def step(ev=None):
        # C entry points directly, so that the timed loop allocates nothing
        if ev:
            ev[0].record(stream)
        bsgpu._check(bsgpu._lib.bsgpu_compress_vis(
            vis.data_ptr(), F, n_in, T, cfg.n_samp, cfg.f, BLOCK_ELEMS, LEVEL, comp.data_ptr(), cap,
            nb_dev.data_ptr(), offs.data_ptr(), ws_c.data_ptr(), ws_c.numel(),
            stream.cuda_stream), "compress_vis")
        if ev:
            ev[1].record(stream)
        bsgpu._check(bsgpu._lib.bsgpu_decompress(
            comp.data_ptr(), stream_len[0], dec.data_ptr(), n_fl, 4, BLOCK_ELEMS,
            offs.data_ptr(), ws_d.data_ptr(), ws_d.numel(), stream.cuda_stream), "decompress")
        if ev:
            ev[2].record(stream)

    nb_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    # first compression fixes the stream length the decompressions read
    stream_len = [cap]
    bsgpu._check(bsgpu._lib.bsgpu_compress_vis(
        vis.data_ptr(), F, n_in, T, cfg.n_samp, cfg.f, BLOCK_ELEMS, LEVEL, comp.data_ptr(), cap,
        nb_dev.data_ptr(), offs.data_ptr(), ws_c.data_ptr(), ws_c.numel(), stream.cuda_stream),
        "compress_vis")
    stream_len[0] = int(nb_dev.item())
    if bsgpu.status(ws_c) != 0:
        raise RuntimeError("compress status")

    clocks = ClockSampler(gpu_index)
    clocks.start()
    time.sleep(0.3)

    for _ in range(args.warmup):
        step()
    # soak ~1 s under load so the clock sampler sees the working clock
    t_soak0 = time.time()
    while time.time() - t_soak0 < 1.0:
        for _ in range(10):
            step()
        torch.cuda.synchronize()
    if bsgpu.status(ws_c) != 0 or bsgpu.status(ws_d) != 0:
        raise RuntimeError("device status after warm-up")
    # correctness of the steady state: the output is the rounded cube
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall1 = time.time()
    ms = start.elapsed_time(end)
    comp_ms = [e[0].elapsed_time(e[1]) for e in evs]
    dec_ms = [e[1].elapsed_time(e[2]) for e in evs]
    if bsgpu.status(ws_c) != 0 or bsgpu.status(ws_d) != 0:
        raise RuntimeError("device status after timed steps")
    clk = clocks.summary(t_soak0, t_wall1)
    clocks.stop()

    ms_t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    total_bytes = nbytes * world
    value = total_bytes * args.steps / (ms_max / 1e3) / 1e9

    # end to end through the C-ABI with host buffers: H2D input, compress,
    # D2H stream; H2D stream, decompress, D2H output
    comp_h = torch.empty(cap, dtype=torch.uint8).pin_memory()
    dec_h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    slen = stream_len[0]
    e2e_times = []
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vis.view(torch.uint8).reshape(-1).copy_(vis_pin.view(torch.uint8).reshape(-1),
                                               non_blocking=True)
        bsgpu._check(bsgpu._lib.bsgpu_compress_vis(
            vis.data_ptr(), F, n_in, T, cfg.n_samp, cfg.f, BLOCK_ELEMS, LEVEL, comp.data_ptr(), cap,
            nb_dev.data_ptr(), offs.data_ptr(), ws_c.data_ptr(), ws_c.numel(),
            stream.cuda_stream), "compress_vis")
        slen = int(nb_dev.item())          # the stream length (8-byte read)
        comp_h[:slen].copy_(comp[:slen], non_blocking=True)
        comp[:slen].copy_(comp_h[:slen], non_blocking=True)
        bsgpu._check(bsgpu._lib.bsgpu_decompress(
            comp.data_ptr(), slen, dec.data_ptr(), n_fl, 4, BLOCK_ELEMS, offs.data_ptr(),
            ws_d.data_ptr(), ws_d.numel(), stream.cuda_stream), "decompress")
        dec_h.copy_(dec, non_blocking=True)
        torch.cuda.synchronize()
        if k:
            e2e_times.append(time.perf_counter() - t0)
    e2e_value = total_bytes / statistics.median(e2e_times) / 1e9
    # the round trip returns the rounded cube
    ok_rt = bool(torch.equal(dec_h[:1 << 20], dec[:1 << 20].cpu()))

    # end to end through the host-buffer API (hostio.HostVisCodec): slabs of
    # 64 frequencies, each its own stream (the paper's chunked storage),
    # uploads / kernels / downloads of different slabs overlapped
    from paper_1503_00638_gb300 import hostio
    del comp_h, dec_h
    h_out = torch.empty_like(vis_pin).pin_memory()
    codec = hostio.HostVisCodec(F, n_in, T, cfg.n_samp, cfg.f, block_elems=BLOCK_ELEMS,
                                level=LEVEL, slab_freq=64, depth=3)
    pipe_times = []
    chunks = None
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        chunks = codec.round_trip(vis_pin, h_out)
        if k:
            pipe_times.append(time.perf_counter() - t0)
    if any(st != (0, 0) for st in codec.statuses()):
        raise RuntimeError("host codec status")
    pipe_h2d, pipe_d2h = codec.bytes_moved(chunks)
    pipe_value = total_bytes / statistics.median(pipe_times) / 1e9
    ok_pipe = bool(torch.equal(h_out.view(torch.uint8).reshape(-1)[:1 << 20],
                               dec[:1 << 20].cpu()))

    hbm, peak_kind = peaks()
    comp_avg_ms = statistics.mean(comp_ms)
    dec_avg_ms = statistics.mean(dec_ms)
    # algorithmic bytes of one compress launch: read the cube, write the stream
    # and the block index, read the autos table (n_in x T floats per freq)
    autos_bytes = F * n_in * T * 4
    alg_c = nbytes + slen + nblk * 8 + autos_bytes
    achieved = alg_c / (comp_avg_ms / 1e3) / 1e9
    alg_d = slen + nblk * 8 + nbytes
    traffic = recorded_traffic(nblk)
    # the compress kernel against the instruction-issue ceiling (the bound
    # that holds for it, DRAM being at ~10 %): warp instructions per launch
    # from the profile of the same source, over the measured launch time
    inst = recorded_profile(nblk, "inst_per_launch")
    issue_line = None
    if inst:
        peak_i = issue_peak_ginst(clk.get("sm_mhz"))
        ach_i = inst / (comp_avg_ms / 1e3) / 1e9
        issue_line = {"bound": "issue", "kernel": "compress_fast_kernel", "achieved": ach_i,
                      "peak": peak_i, "unit": "G warp-instructions/s", "frac": ach_i / peak_i,
                      "inst_per_launch": inst}

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if F == 1024 else f"{WORKLOAD} (first {F} freq)",
                   "f": cfg.f, "N": 2 ** 17, "block_bytes": BLOCK_ELEMS * 4,
                   "cube_bytes": nbytes,
                   "l2": f"inputs ({nbytes / 1e9:.2f} GB) larger than L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "compress_gbs": nbytes / (comp_avg_ms / 1e3) / 1e9,
        "decompress_gbs": nbytes / (dec_avg_ms / 1e3) / 1e9,
        "kernel_ms": {"compress": {"mean": comp_avg_ms, "median": statistics.median(comp_ms),
                                   "best": min(comp_ms)},
                      "decompress": {"mean": dec_avg_ms, "median": statistics.median(dec_ms),
                                     "best": min(dec_ms)}},
        "ratio": slen / nbytes,
        "roofline": {"bound": "hbm", "kernel": "compress_fast_kernel (fused round+shuffle+LZ4)",
                     "achieved": achieved, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "algorithmic_bytes": alg_c},
        "decompress_roofline": {"bound": "hbm", "achieved": alg_d / (dec_avg_ms / 1e3) / 1e9,
                                "peak": hbm, "unit": "GB/s",
                                "frac": alg_d / (dec_avg_ms / 1e3) / 1e9 / hbm},
        "issue_roofline": issue_line,
        "e2e": {"value": pipe_value, "unit": "GB/s", "h2d_bytes_per_step": pipe_h2d,
                "d2h_bytes_per_step": pipe_d2h, "round_trip_ok": ok_pipe,
                "api": "hostio.HostVisCodec.round_trip (64-frequency slabs, pipelined)",
                "unpipelined": {"value": e2e_value, "h2d_bytes_per_step": nbytes + slen,
                                "d2h_bytes_per_step": slen + nbytes + 8,
                                "round_trip_ok": ok_rt,
                                "api": "bsgpu_compress_vis / bsgpu_decompress, one stream"}},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
        "wall_s_timed": t_wall1 - t_wall0,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nb_cpu, dt, ratio = oracle_round_trip(cfg, args.cpu_freqs, cfg.f, rank)
        line["cpu_baseline"] = {"value": nb_cpu / dt / 1e9, "unit": "GB/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"first {args.cpu_freqs} of 1024 frequencies "
                                          f"({nb_cpu / 1e6:.1f} MB): round+compress+decompress",
                                "ratio": ratio}
        nc = host_cores()
        nf_all = min(1024, args.cpu_freqs * nc)
        nb_all, dt_all = oracle_round_trip_cores(cfg, nf_all, cfg.f, nc)
        line["cpu_baseline_all_cores"] = {
            "value": nb_all / dt_all / 1e9, "unit": "GB/s", "cores": nc, "kind": "oracle",
            "sample": f"first {nf_all} of 1024 frequencies ({nb_all / 1e6:.1f} MB) in {nc} "
                      f"frequency slabs, one thread each: round+compress+decompress"}
    if rank == 0 and world == 1:
        line["ratio_vs_oracle"], orc_stream = ratio_side_by_side(cfg, vis_h, args)
        line["decompress_no_index"] = time_no_index(
            bsgpu, [("gpu stream", comp[:slen]), ("oracle stream", orc_stream)], dec, n_fl,
            nbytes, dec_avg_ms)
    if world == 1 and not args.no_sub:
        # the batched engine and the server, at stated sizes, in the same line
        del comp, dec, ws_c, ws_d, offs
        torch.cuda.empty_cache()
        b = run_batch(args, rank, world, local, barrier, gpu_index, chunks=args.sub_chunks,
                      steps=5, warmup=3, cpu=False)
        line["batch"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "compress_gbs",
                                           "decompress_gbs", "ratio", "roofline",
                                           "decompress_roofline", "config", "parity",
                                           "clocks", "gpu_launches") if k in b}
        torch.cuda.empty_cache()
        sv = run_serve(args, rank, world, gpu_index, requests=args.sub_requests, payloads=128)
        line["serving"] = {"value_gbs_at_saturation": sv["value"], "unit": "GB/s",
                           "config": sv["config"], "clocks": sv["clocks"], **sv["serving"]}
        torch.cuda.empty_cache()
        line["batch"]["e2e"] = run_batch_e2e(args, args.sub_chunks, batch_launch(b))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def ratio_side_by_side(cfg, vis, args):
    """Compression ratio of the GPU encoder and of the oracle's greedy encoder
    on the whole CHIME-shaped cube at f = 1e-3, 1e-2 and 0.1 (the oracle over
    all host cores, one frequency slab each; blocks never straddle slabs, so
    the per-slab streams add up to the whole stream less their headers).
    Also returns the oracle's whole-cube stream at f = args.f (the slabs'
    blocks after one header)."""
    import concurrent.futures as cf
    import torch
    import oracle
    from paper_1503_00638_gb300 import bsgpu
    F = vis.shape[0]
    d = torch.from_numpy(vis).cuda()
    out, whole = {}, None
    for f in sorted({1e-3, 1e-2, 0.1, args.f}):
        c = bsgpu.compress_vis(d, cfg.n_samp, f, BLOCK_ELEMS)
        g = c.nbytes

        def slab(fr):
            r = oracle.reduce_precision_c64(vis[fr:fr + 1], cfg.n_samp, f)
            return oracle.compress(r.view(np.float32).reshape(-1), BLOCK_ELEMS)[12:]

        with cf.ThreadPoolExecutor(max_workers=host_cores()) as ex:
            parts = list(ex.map(slab, range(F)))
        o = 12 + sum(len(p) for p in parts)
        out[str(f)] = {"gpu": g / vis.nbytes, "oracle": o / vis.nbytes}
        if f == args.f:
            whole = (vis.nbytes.to_bytes(8, "big") + (BLOCK_ELEMS * 4).to_bytes(4, "big")
                     + b"".join(parts))
        del c, parts
    del d
    return out, whole


def time_no_index(bsgpu, streams, want, n_fl, nbytes, indexed_ms, reps=5):
    """Decompression of whole-cube streams WITHOUT their block index (the
    device first recovers it from the chain of length fields: the parallel
    segment walk, checked, else the staged serial walk), next to the same
    stream decoded with its index; each output is checked against `want`."""
    import torch
    out = {"indexed_decompress_gbs": nbytes / (indexed_ms / 1e3) / 1e9}
    dec = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    for name, st in streams:
        d = st if isinstance(st, torch.Tensor) else torch.frombuffer(bytearray(st),
                                                                      dtype=torch.uint8).cuda()
        ws = bsgpu.new_workspace(bsgpu.workspace_size(bsgpu.OP_DECOMPRESS, n_fl, 4, BLOCK_ELEMS))
        bsgpu.decompress(d, d.numel(), n_fl, 4, BLOCK_ELEMS, offsets=None, out=dec, ws=ws)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bsgpu.decompress(d, d.numel(), n_fl, 4, BLOCK_ELEMS, offsets=None, out=dec, ws=ws)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ok = bool(torch.equal(dec, want)) and bsgpu.status(ws) == 0
        ms = statistics.median(ts)
        # the same stream with its block index (read off the length fields
        # on the host), for the decoder's own time on it
        h = d.cpu().numpy()
        offs, D = [], 12
        while len(offs) < bsgpu.num_blocks(n_fl, 4, BLOCK_ELEMS):
            offs.append(D)
            D += 4 + int.from_bytes(h[D:D + 4].tobytes(), "big")
        od = torch.tensor(offs, dtype=torch.int64, device="cuda")
        ti = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bsgpu.decompress(d, d.numel(), n_fl, 4, BLOCK_ELEMS, offsets=od, out=dec, ws=ws)
            e1.record()
            e1.synchronize()
            ti.append(e0.elapsed_time(e1))
        ok = ok and bool(torch.equal(dec, want))
        mi = statistics.median(ti)
        out[name] = {"ms": ms, "gbs": nbytes / (ms / 1e3) / 1e9, "exact": ok,
                     "with_index_ms": mi, "with_index_gbs": nbytes / (mi / 1e3) / 1e9,
                     "index_recovery_ms": ms - mi, "stream_bytes": int(d.numel())}
        del d, ws, od
    return out


if __name__ == "__main__":
    main()
