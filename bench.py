"""Benchmark: Wallace normal generation on one GB300 (per rank), JSON line out.

Workload (one "step"): 4096 independent streams (one CTA each), pool N = 4096,
R = 2 passes per block, seeds 1..4096 (rank r adds 4096 r), each stream
returning its next 2^20 FP32 values -- 2^32 N(0,1) values per step written to
HBM.  Streams persist across steps (a generator is created once and drawn
from many times); creation (seeding, initialisation, 8 warm-up blocks) runs
before the timed region and is reported separately.

Reported: whole-job variates/s (value), the generate kernel's achieved HBM
GB/s against the measured copy peak (roofline), the same metric delivered to
pinned host memory through wn_generate_host (e2e), the project's own
Box-Muller/Philox generator on the same GPU and shape (comparison), and the
FP64 CPU oracle timed on the host's cores on a bounded sample (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--kernel-only times the generate steps alone (for ncu captures); with it,
--pool/--passes/--dtype/--in-place select another workload of the kernel
(e.g. the 16-bit precision workload's pools: --pool 16384 --passes 3
--dtype bf16).

For N > 1 run under torch.distributed.run; ranks shard streams (weak scaling)
and only the timing is reduced (max over ranks).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# every run times the library's tuners afresh (no choices from earlier processes)
os.environ["WN_TUNE_CACHE"] = "off"

METRIC = "N(0,1) variates/s on 1 GB300, % of HBM-write roofline, vs Box–Muller same GPU"
STREAMS, POOL_N, PASSES_R, PER_STREAM = 4096, 4096, 2, 1 << 20
WARMUP_BLOCKS = 8
HDR_BYTES = 96
KERNEL_SOURCES = ("wn_group.cuh", "wn_gen.cuh", "wn_device.cuh")


ESIZE = {"f32": 4, "bf16": 2, "f16": 2}


def _workload(streams, per_stream, pool=POOL_N, passes=PASSES_R, dtype="f32"):
    return (f"many_streams: {streams} streams x pool N={pool}, R={passes} passes/block, "
            f"seeds SplitMix64(1..{streams}), {per_stream} {dtype.upper()} variates per stream per step")


def _config(streams=STREAMS, per_stream=PER_STREAM, pool=POOL_N, passes=PASSES_R, dtype="f32"):
    out_bytes = streams * per_stream * ESIZE[dtype]
    return {"workload": _workload(streams, per_stream, pool, passes, dtype), "streams": streams, "pool_N": pool,
            "passes_R": passes, "variates_per_stream_per_step": per_stream,
            "variates_per_step": streams * per_stream,
            "output": f"{dtype.upper()}, [stream][value] contiguous in HBM",
            "l2": "flushed (256 MiB write) between steps, outside the per-step events; "
                  f"{out_bytes / 2**30:.3g} GiB of output per step"}


def kernel_source_hash():
    """sha256 over the generate kernel's sources (profiles record it)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1005_2314_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _algorithmic_bytes(streams, per_stream, pool=POOL_N, esize=4):
    """Bytes one generate launch must move: the output values plus reading and
    writing each stream's pool and header once."""
    return streams * (per_stream * esize + 2 * pool * 4 + 2 * HDR_BYTES)


def _l1_roofline(values_per_s, passes, esize, sm_mhz, sms):
    """The shared-memory side of the kernel: L1 data-pipe wavefronts the method
    needs per value against one 128-byte wavefront per cycle per SM.  Each
    pass gathers one 4-byte value per lane (one wavefront per 32 values) and
    stores four per lane as 16 bytes (one wavefront per 32 values); the output
    stores add 32 esize bytes per 32 values (esize/4 wavefronts).  Pool loads,
    tables and the scale are a few per block and left out."""
    if not sm_mhz:
        return None
    wf = (2.0 * passes + esize / 4.0) / 32.0
    achieved = values_per_s * wf
    peak = sms * sm_mhz * 1e6
    return {"bound": "l1_data_pipe", "achieved": round(achieved / 1e9, 2), "peak": round(peak / 1e9, 2),
            "unit": "G wavefronts/s", "frac": round(achieved / peak, 4), "wavefronts_per_value": wf,
            "peak_kind": f"{sms} SMs x 1 wavefront per cycle at the sampled {sm_mhz:.0f} MHz"}


def _traffic_per_launch(streams, per_stream):
    """DRAM bytes per launch from the committed ncu summary (a capture with the
    same per-stream count on fewer streams, scaled by streams: every stream of
    the launch moves the same bytes); None when the summary is missing, was
    taken at another per-stream count, or the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "generate_many_streams_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        if t["source_sha256"] != kernel_source_hash() or t["per_stream"] != per_stream:
            return None
        return int(t["dram_bytes_per_stream"] * streams)
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (test infrastructure, timed as a reported baseline)
# ---------------------------------------------------------------------------

def _cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(n_streams: int, per_stream: int, steps: int, warmup: int, threads: int):
    """Times the FP64 oracle on `n_streams` streams of the bench workload,
    each step returning the next `per_stream` values of every stream, spread
    over `threads` host threads (the oracle releases the GIL).  Returns the
    per-step times in seconds."""
    import concurrent.futures
    import numpy as np
    import oracle

    streams = [oracle.Stream(POOL_N, PASSES_R, seed=i + 1, warmup=WARMUP_BLOCKS) for i in range(n_streams)]
    bufs = [np.empty(per_stream, dtype=np.float64) for _ in range(threads)]
    groups = [streams[t::threads] for t in range(threads)]
    lib = oracle.lib()

    def work(t):
        buf = bufs[t]
        for s in groups[t]:
            lib.orc_generate(s._h, buf.ctypes.data, per_stream)

    times = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        for i in range(warmup + steps):
            t0 = time.perf_counter()
            list(ex.map(work, range(threads)))
            dt = time.perf_counter() - t0
            if i >= warmup:
                times.append(dt)
    return times


# ---------------------------------------------------------------------------
# Rank logic (weak scaling: ranks shard independent streams)
# ---------------------------------------------------------------------------

def rank_seeds(rank: int, streams: int):
    """Seeds of rank `rank`'s streams: disjoint ranges, 1-based."""
    return [rank * streams + i + 1 for i in range(streams)]


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Maximum of a per-rank float over all ranks (the timing reduction)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def _timed(torch, stream, flush, fn, reps):
    """Median CUDA-event time (ms) of fn() on `stream`, L2 flushed before each."""
    ms = []
    for i in range(reps):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ms.append((a, b))
    torch.cuda.synchronize()
    t = sorted(x.elapsed_time(y) for x, y in ms)
    return t[len(t) // 2]


def other_workloads(wn, torch, dev, stream, flush, sm_mhz=None, headline_value=None):
    """The method's other workloads on this GPU, each timed with CUDA events:
    one stream (pool 1024, R=2, 2^24 FP32 in one call); 4096 streams of pool
    16384, R=3, 2^21 values each in BF16 and in FP16 (with Box-Muller at the
    same shape and type); the same 16-bit outputs at the headline's shape
    (pool 4096, R=2, 2^20 each); the plane-rotation form at that shape; and
    the fused GBM consumer (2^20 paths x 252 steps, pool 4096, R=2, normals
    never written to memory)."""
    peak, _ = _peaks()
    res = {}
    # single stream: a serial chain of blocks on one SM
    h1 = wn.wn_create(1024, 2, 1)
    wn.wn_set_cuda_stream(h1, stream)
    n1 = 1 << 24
    o1 = torch.empty(n1, dtype=torch.float32, device=dev)
    shape1 = wn.wn_get_config_ex(h1)  # a lone stream's default: the chain mode
    wn.wn_generate_ex(o1, n1, h1, wn.WN_F32, stream)
    t1 = _timed(torch, stream, flush, lambda: wn.wn_generate_ex(o1, n1, h1, wn.WN_F32, stream), 5)
    res["single_stream"] = {"value": n1 / (t1 / 1e3), "unit": "variates/s", "ms_per_call": t1,
                            "ns_per_block": t1 * 1e6 / math.ceil(n1 / 1023),
                            "config": "1 stream, pool N=1024, R=2, seed 1, 2^24 FP32 per call",
                            "shape": list(shape1)}
    wn.wn_destroy(h1)
    del o1
    # 16-bit outputs from an FP32 pool
    S3, N3, R3, per3 = 4096, 16384, 3, 1 << 21
    h3 = wn.wn_create_streams([N3] * S3, [R3] * S3, list(range(1, S3 + 1)), WARMUP_BLOCKS, stream)
    o3 = torch.empty(S3 * per3, dtype=torch.bfloat16, device=dev)
    prec = {}
    for dt, name, tdt in ((wn.WN_BF16, "bf16", torch.bfloat16), (wn.WN_F16, "f16", torch.float16)):
        o = o3.view(tdt)
        shape3 = wn.wn_get_config_ex(h3)  # default: group mode, 4 warps x 32 quadruples per lane
        wn.wn_generate_ex(o, per3, h3, dt, stream)
        t3 = _timed(torch, stream, flush, lambda: wn.wn_generate_ex(o, per3, h3, dt, stream), 5)
        tb = _timed(torch, stream, flush, lambda: wn.wn_boxmuller(o, per3, S3, 1, dt, stream), 5)
        v = S3 * per3 / (t3 / 1e3)
        l1 = _l1_roofline(v, R3, 2, sm_mhz, torch.cuda.get_device_properties(dev).multi_processor_count)
        prec[name] = {"value": v, "unit": "variates/s", "ms_per_step": t3, "shape": list(shape3),
                      "hbm_frac": round(v * 2 / 1e9 / peak, 4), "l1_frac": l1["frac"] if l1 else None,
                      "boxmuller_value": S3 * per3 / (tb / 1e3), "wallace_over_boxmuller": tb / t3}
    prec["config"] = "4096 streams x pool N=16384, R=3, 2^21 values each (2^33 per type), FP32 pool, 16-bit RN output"
    res["precision"] = prec
    wn.wn_destroy(h3)
    del o3
    # the 16-bit outputs at the headline's shape (4096 streams x pool 4096,
    # R = 2, 2^20 values each): what halving the bytes per value buys
    S2, N2, R2, per2 = 4096, 4096, 2, 1 << 20
    h2 = wn.wn_create_streams([N2] * S2, [R2] * S2, list(range(1, S2 + 1)), WARMUP_BLOCKS, stream)
    o2 = torch.empty(S2 * per2, dtype=torch.bfloat16, device=dev)
    pc2 = {}
    for dt, name, tdt in ((wn.WN_BF16, "bf16", torch.bfloat16), (wn.WN_F16, "f16", torch.float16)):
        o = o2.view(tdt)
        wn.wn_generate_ex(o, per2, h2, dt, stream)
        t2 = _timed(torch, stream, flush, lambda: wn.wn_generate_ex(o, per2, h2, dt, stream), 5)
        v = S2 * per2 / (t2 / 1e3)
        l1 = _l1_roofline(v, R2, 2, sm_mhz, torch.cuda.get_device_properties(dev).multi_processor_count)
        pc2[name] = {"value": v, "unit": "variates/s", "ms_per_step": t2, "shape": list(wn.wn_get_config_ex(h2)),
                     "hbm_frac": round(v * 2 / 1e9 / peak, 4), "l1_frac": l1["frac"] if l1 else None,
                     "over_fp32_headline": round(v / headline_value, 4) if headline_value else None}
    pc2["config"] = "4096 streams x pool N=4096, R=2, 2^20 values each (2^32 per type), FP32 pool, 16-bit RN output"
    res["precision_c2"] = pc2
    # the plane-rotation form (Section 5.3, rann4) at the headline's shape, FP32
    hr = wn.wn_create_ex([N2] * S2, [R2] * S2, list(range(1, S2 + 1)), WARMUP_BLOCKS, update="rotation",
                         cuda_stream=stream)
    o = o2.view(torch.float32)[: S2 * per2 // 2]
    perr = per2 // 2
    wn.wn_generate_ex(o, perr, hr, wn.WN_F32, stream)
    tr = _timed(torch, stream, flush, lambda: wn.wn_generate_ex(o, perr, hr, wn.WN_F32, stream), 5)
    v = S2 * perr / (tr / 1e3)
    res["rotation"] = {"value": v, "unit": "variates/s", "ms_per_step": tr, "shape": list(wn.wn_get_config_ex(hr)),
                       "hbm_frac": round(v * 4 / 1e9 / peak, 4),
                       "config": "4096 streams x pool N=4096, R=2, 2^19 FP32 values each, plane rotations "
                                 "(general kernel; gathers 2-way bank-conflicted)"}
    wn.wn_destroy(hr)
    wn.wn_destroy(h2)
    del o2
    # fused consumer: geometric Brownian motion driven in-kernel
    # 585 paths per stream (7 steps per block): 1793 streams, four full waves of
    # 3 CTAs per SM (measured 0.249 ms against 0.263 for 455 per stream, whose
    # 2305 streams leave a sixth wave almost empty)
    N5, R5, ppg, steps, paths = 4096, 2, 585, 252, 1 << 20
    G = -(-paths // ppg)
    h5 = wn.wn_create_streams([N5] * G, [R5] * G, list(range(1, G + 1)), WARMUP_BLOCKS, stream)
    st = torch.empty(G * ppg, dtype=torch.float32, device=dev)
    args5 = (0.05, 0.2, 1.0 / 252)
    wn.wn_gbm(st, h5, ppg, steps, 100.0, *args5, stream)
    t5 = _timed(torch, stream, flush, lambda: wn.wn_gbm(st, h5, ppg, steps, 100.0, *args5, stream), 5)
    gv = G * ppg * steps / (t5 / 1e3)
    # the consumer writes nothing per value: its bound is the shared-memory
    # side alone (2R wavefronts per 32 values, no output wavefronts)
    gl1 = _l1_roofline(gv, R5, 0, sm_mhz, torch.cuda.get_device_properties(dev).multi_processor_count)
    res["gbm"] = {"value": gv, "unit": "normals consumed/s", "ms_per_call": t5,
                  "paths_per_s": G * ppg / (t5 / 1e3), "l1_frac": gl1["frac"] if gl1 else None,
                  "config": f"{G * ppg} paths ({G} streams x {ppg}) x 252 steps, pool N=4096, R=2, "
                            "S0=100, mu=0.05, sigma=0.2, dt=1/252"}
    wn.wn_destroy(h5)
    return res



def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1005_2314_gb300 as wn

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    STREAMS, PER_STREAM = args.streams, args.per_stream
    POOL, R, DT = args.pool, args.passes, args.dtype
    wdt = {"f32": wn.WN_F32, "bf16": wn.WN_BF16, "f16": wn.WN_F16}[DT]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[DT]
    seeds = rank_seeds(rank, STREAMS)

    t0 = time.perf_counter()
    h = wn.wn_create_streams([POOL] * STREAMS, [R] * STREAMS, seeds, WARMUP_BLOCKS, stream)
    create_s = time.perf_counter() - t0
    if args.shape:
        qt, th = (int(v) for v in args.shape.split(","))
        wn.wn_set_config_ex(h, qt, th, (wn.WN_CFG_IN_PLACE if args.in_place else 0) |
                            (wn.WN_CFG_GROUP if args.group else 0))
    elif args.autotune:  # the library's autotuner times the shapes on a copy of the state
        wn.wn_autotune(h, min(PER_STREAM, 1 << 17), wdt, stream)
    # otherwise the library's default shape for the pool size (the autotuner's
    # pick on GB300; fixed, so that a profiler's slowdown cannot change it)
    shape = wn.wn_get_config_ex(h)
    out = torch.empty(STREAMS * PER_STREAM, dtype=tdt, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        if args.method == "boxmuller":  # the comparison generator on the same shape (--kernel-only)
            wn.wn_boxmuller(out, PER_STREAM, STREAMS, 1, wdt, stream)
        else:
            wn.wn_generate_ex(out, PER_STREAM, h, wdt, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    variates = STREAMS * PER_STREAM
    value = world * variates * args.steps / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps

    # roofline of the generate kernel (the step is exactly one launch of it)
    peak, peak_kind = _peaks()
    algo = _algorithmic_bytes(STREAMS, PER_STREAM, POOL, ESIZE[DT])
    achieved = algo / (ms_per_step / 1e3) / 1e9
    default_kernel = (POOL, R, DT) == (POOL_N, PASSES_R, "f32")
    traffic = _traffic_per_launch(STREAMS, PER_STREAM) if default_kernel else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": algo,
                "kernel": (f"wn::group_kernel ({DT.upper()} out, {shape[1] // 32} warps x {shape[0]} quadruples "
                           f"per lane per stream, no control warp, in-place pool)" if shape[2] & 2 else
                           f"wn::chain_kernel ({DT.upper()} out, {shape[1] // 32} compute warps x {shape[0]} "
                           f"quadruples per lane + scale, store and draw warps per stream)" if shape[2] & 4 else
                           f"wn::generate_kernel ({DT.upper()} out, {shape[0]} quadruples x {shape[1]} compute "
                           f"threads + 1 control warp per stream{', in-place pool' if shape[2] else ''})")}
    if args.method == "boxmuller":
        roofline["kernel"] = f"wn::boxmuller_kernel ({DT.upper()} out, Philox4x32-10)"
        roofline["algorithmic_bytes_per_launch"] = algo = STREAMS * PER_STREAM * ESIZE[DT]
        roofline["achieved"] = round(algo / (ms_per_step / 1e3) / 1e9, 1)
        roofline["frac"] = round(roofline["achieved"] / peak, 4)
        roofline["traffic"] = None
    if args.kernel_only:
        wn.wn_destroy(h)
        return {"metric": METRIC, "value": value, "unit": "variates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step,
                "config": _config(STREAMS, PER_STREAM, POOL, R, DT),
                "roofline": roofline, "gpu_launches": args.steps, "kernel_only": True}

    # context: a plain write of the same bytes by torch (fill_), i.e. what a
    # write-only stream reaches on this GPU
    fill_ms = []
    for i in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(i & 0xFF)
        a.record(stream)
        out.fill_(float(i))
        b.record(stream)
        fill_ms.append((a, b))
    torch.cuda.synchronize()
    fill_gbs = out.numel() * 4 / (min(x.elapsed_time(y) for x, y in fill_ms) / 1e3) / 1e9

    # the conventional comparison on the same GPU and shape
    bm_out = out
    for _ in range(3):
        wn.wn_boxmuller(bm_out, PER_STREAM, STREAMS, 1, wn.WN_F32, stream)
    bm_ms = []
    for i in range(max(5, args.steps // 2)):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        wn.wn_boxmuller(bm_out, PER_STREAM, STREAMS, 1, wn.WN_F32, stream)
        b.record(stream)
        bm_ms.append((a, b))
    torch.cuda.synchronize()
    bm_step = sum(a.elapsed_time(b) for a, b in bm_ms) / len(bm_ms)
    bm_value = variates / (bm_step / 1e3)

    # e2e: values delivered to pinned host memory through the public API
    e2e = None
    try:
        host = torch.empty(STREAMS * PER_STREAM, dtype=torch.float32, pin_memory=True)
        wn.wn_generate_host(host, PER_STREAM, h, wn.WN_F32, stream)
        torch.cuda.synchronize()
        e_steps = max(3, min(args.steps, 10))
        t = time.perf_counter()
        for _ in range(e_steps):
            wn.wn_generate_host(host, PER_STREAM, h, wn.WN_F32, stream)
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t, world, dev)
        e2e = {"value": world * variates * e_steps / dt, "unit": "variates/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": variates * 4, "steps": e_steps,
               "how": "wn_generate_host into pinned host memory (the kernel stores straight into it over "
                      "the host link); host wall clock"}
        del host
    except Exception as ex:  # pinned allocation can fail on small hosts
        e2e = {"value": None, "unit": "variates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
               "error": str(ex)[:200]}

    # the other workloads of the method, one line each (the headline stays the
    # many-streams FP32 step above)
    configs = None
    if not args.no_configs:
        configs = other_workloads(wn, torch, dev, stream, flush, clk.summary()["sm_mhz"], value / world)

    # the batched uneven-request workload: 10,000 streams, pool from
    # {1024, 4096, 16384}, R from {1, 2, 4}, log-uniform lengths 2^10..2^24,
    # FP32 packed contiguously; one captured graph of persistent kernels
    batched = None
    if not args.no_batch:
        from paper_1005_2314_gb300.workloads import packed_offsets, uneven_batch
        bN, bR, bc = uneven_batch(10000, seed=12345)
        boff = packed_offsets(bc)
        btotal = int(bc.sum())
        del out, bm_out
        bout = torch.empty(btotal, dtype=torch.float32, device=dev)
        hb = wn.wn_create_streams(bN, bR, [rank * 10000 + i + 1 for i in range(10000)], WARMUP_BLOCKS, stream)
        wn.wn_autotune_batch(bout, bc, boff, hb, wn.WN_F32, stream)
        plan = wn.wn_get_batch_plan(hb)
        wn.wn_generate_batch(bout, bc, boff, hb, wn.WN_F32, True, stream)  # captures the graph
        torch.cuda.synchronize()
        bms = []
        for i in range(7):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            wn.wn_generate_batch(bout, bc, boff, hb, wn.WN_F32, True, stream)  # graph replay
            b.record(stream)
            bms.append((a, b))
        torch.cuda.synchronize()
        bts = sorted(x.elapsed_time(y) for x, y in bms)
        bt = bts[len(bts) // 2]
        batched = {"value": btotal / (bt / 1e3), "unit": "variates/s", "ms_per_replay": bt,
                   "ms_min": bts[0], "ms_max": bts[-1], "spread": round(bts[-1] / bts[0] - 1, 4),
                   "replays": len(bts), "variates_per_replay": btotal, "streams": 10000,
                   "achieved_gbs": round(btotal * 4 / (bt / 1e3) / 1e9, 1),
                   "longest_request": int(bc.max()),
                   "plan": {"chains": int(plan[0]), "chains_per_sm": int(plan[1])},
                   "how": "wn_generate_batch with use_graph: per pool size one persistent kernel (atomic claim, "
                          "longest request first), groups forked on branch streams, captured once and replayed; "
                          "launch shapes from wn_autotune_batch; median of 7 replays (min, max and spread beside it)"}
        wn.wn_destroy(hb)
        del bout

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = _cpu_cores()
        ns, per = 1024, PER_STREAM
        times = oracle_sample(ns, per, steps=1, warmup=0, threads=cores)
        cpu = {"value": ns * per / times[0], "unit": "variates/s", "cores": cores, "kind": "oracle",
               "sample": f"{ns} of the {STREAMS} streams, next 2^20 values each after creation "
                         f"(1/4 of one step), FP64 oracle, {cores} threads"}

    line = {"metric": METRIC, "value": value, "unit": "variates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(STREAMS, PER_STREAM),
            "roofline": roofline,
            "l1_roofline": _l1_roofline(value / world, PASSES_R, 4, clk.summary()["sm_mhz"],
                                        torch.cuda.get_device_properties(dev).multi_processor_count),
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "comparison": {"boxmuller_philox4x32_10": {"value": bm_value, "unit": "variates/s",
                                                       "ms_per_step": bm_step,
                                                       "wallace_over_boxmuller": value / world / bm_value}},
            "batched_uneven": batched,
            "workloads": configs,
            "create_s": create_s,
            "context": {"torch_fill_write_gbs": round(fill_gbs, 1),
                        "frac_of_fill": round(achieved / fill_gbs, 4)}}
    wn.wn_destroy(h)
    return line


def run_reference(args, rank, world):
    """The oracle on the host's cores: same metric and workload, each step a
    bounded sample (256 of the 4096 streams, their next 2^20 values)."""
    if rank != 0:
        return None
    cores = _cpu_cores()
    ns = 256
    times = oracle_sample(ns, PER_STREAM, steps=args.steps, warmup=args.warmup, threads=cores)
    total = sum(times)
    value = ns * PER_STREAM * args.steps / total
    sample = (f"each step: {ns} of the {STREAMS} streams, their next 2^20 values (1/16 of the workload), "
              f"FP64 oracle over {cores} host threads")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "variates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(),
            "cpu_baseline": {"value": value, "unit": "variates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "variates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched uneven-request leg")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the single-stream, 16-bit and fused-GBM workload legs")
    ap.add_argument("--streams", type=int, default=STREAMS, help="streams per GPU (default 4096)")
    ap.add_argument("--per-stream", type=int, default=PER_STREAM, help="values per stream per step")
    ap.add_argument("--shape", default="",
                    help="launch shape 'quadruples,threads' instead of autotuning (e.g. 8,128)")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time only the generate steps (for ncu captures of the generate kernel)")
    ap.add_argument("--pool", type=int, default=POOL_N, help="pool size N (--kernel-only runs)")
    ap.add_argument("--passes", type=int, default=PASSES_R, help="passes per block R (--kernel-only runs)")
    ap.add_argument("--dtype", choices=sorted(ESIZE), default="f32", help="output type (--kernel-only runs)")
    ap.add_argument("--in-place", action="store_true", help="with --shape: the in-place pool layout")
    ap.add_argument("--method", choices=["wallace", "boxmuller"], default="wallace",
                    help="--kernel-only: time Wallace's generator or the Box-Muller comparison on the same shape")
    ap.add_argument("--group", action="store_true",
                    help="with --shape 'quadruples per lane,threads': the group-mode kernel")
    ap.add_argument("--autotune", action="store_true",
                    help="main workload: wn_autotune's pick instead of the library default shape")
    args = ap.parse_args()
    if ((args.pool, args.passes, args.dtype) != (POOL_N, PASSES_R, "f32") or args.method != "wallace") \
            and not args.kernel_only:
        ap.error("--pool/--passes/--dtype/--method select another workload for --kernel-only runs only")
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    import __graft_entry__
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
        if rank == 0:
            __graft_entry__.build()
        torch.distributed.barrier()
    else:
        __graft_entry__.build()
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
