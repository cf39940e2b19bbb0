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

def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1503_00638_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(scale_units):
    """dram bytes per launch of the compress kernel from profiles/traffic.json,
    if it was taken on the current kernel source; scaled to this launch."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    per_unit = d["dram_bytes_per_launch"] / d["units_per_launch"]
    return per_unit * scale_units


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

    gpu_index = local
    vis_dev_env = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis_dev_env:
        try:
            gpu_index = int(vis_dev_env.split(",")[local])
        except ValueError:
            gpu_index = local
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

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if F == 1024 else f"{WORKLOAD} (first {F} freq)",
                   "f": cfg.f, "N": 2 ** 17, "block_bytes": BLOCK_ELEMS * 4,
                   "cube_bytes": nbytes, "l2": "inputs (1.08 GB) larger than L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "compress_gbs": nbytes / (comp_avg_ms / 1e3) / 1e9,
        "decompress_gbs": nbytes / (dec_avg_ms / 1e3) / 1e9,
        "ratio": slen / nbytes,
        "roofline": {"bound": "hbm", "kernel": "compress_fast_kernel (fused round+shuffle+LZ4)",
                     "achieved": achieved, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "algorithmic_bytes": alg_c},
        "decompress_roofline": {"bound": "hbm", "achieved": alg_d / (dec_avg_ms / 1e3) / 1e9,
                                "peak": hbm, "unit": "GB/s",
                                "frac": alg_d / (dec_avg_ms / 1e3) / 1e9 / hbm},
        "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": nbytes + slen,
                "d2h_bytes_per_step": slen + nbytes + 8, "round_trip_ok": ok_rt},
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
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
