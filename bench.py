#!/usr/bin/env python
"""Realtime factor of the lunar-pulse hot path on GB300.

A step is one block of station data through the whole path (beamform +
de-disperse, noise level, inverse FFT + synthesis FIR + envelope trigger,
history shift): 48 stations x 2 pols x 488 subbands x 65536 frames of complex
int8 (6.14 GB, 0.336 s of data) into 50 beams.  The realtime factor is the
block duration divided by the device time per block.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp16|fp32]

With N > 1 (torchrun) every rank runs its own replica on its own GPU (the
streams are independent; there is no exchange step) and rank 0 reports the
whole-job rate from the slowest rank's time.  --impl reference times the FP64
CPU oracle on bounded samples of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

FS_HZ = 200e6
M = 1024
# algorithmic work per output sample of the synthesis kernel: inverse FFT
# 5 N log2 N / N = 50 FLOP (the paper's radix-2 count), 16-tap complex FIR
# with real taps 64 FLOP, envelope |u|^2 and compare 4 FLOP
SYNTH_FLOP_PER_SAMPLE = 50 + 64 + 4
SMS = 152
FP32_LANES_PER_SM = 128


def measured_peaks():
    """The measured peaks file (copy bandwidth, bf16 GEMM, clocks), or {}."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def write4_bandwidth():
    """Streaming bandwidth (GB/s) of a kernel that reads every word once and
    writes it four times (the beamformer's mix), from profiles/hbm_mix.json, or
    None when it was not measured."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "hbm_mix.json")))
        return float(rec["forms"]["fan4"]["gbs"])
    except (OSError, ValueError, KeyError):
        return None


def fp32_peak():
    """FP32 FMA peak (TFLOP/s, SM MHz it was measured at, note): the measurement of
    the peak microbenchmark (profiles/fp32_peak.json) when recorded, else unit
    counts at the maximum SM clock."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "fp32_peak.json")))
        form = rec["forms"][rec["peak_form"]]
        mhz = form["clocks"].get("sm_mhz")
        return (float(rec["peak_tflops"]), mhz,
                f"measured: {rec['peak_form'].upper()} chains on all SMs "
                f"(python -m paper_1612_06592_gb300.microbench.peaks, median SM clock {mhz} MHz; "
                f"{rec['reading']})")
    except (OSError, ValueError, KeyError):
        mhz = float(measured_peaks().get("sm_max_mhz", 2070.0))
        return (SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, mhz,
                f"unit counts: {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 FLOP x {mhz:.0f} MHz "
                "(no measurement recorded)")


def fp32_peak_tflops():
    return fp32_peak()[0]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--shard", default="beams", choices=["beams", "replicas"],
                    help="N > 1: beams (each rank runs its share of the 50 beams on the same "
                         "block, triggers merged on rank 0; strong scaling) or replicas (every "
                         "rank the whole problem on its own block; weak scaling)")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16", choices=["fp16", "fp32"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-frames", type=int, default=16384)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--serve-blocks", type=int, default=200,
                    help="blocks of the realtime serving leg (p50/p99 latency); 0 skips it")
    ap.add_argument("--stress-blocks", type=int, default=1,
                    help="blocks of the stress leg (200 beams x 8 trials x 262144 frames, "
                         "recall and roofline) added to the default line; 0 skips it")
    ap.add_argument("--workload", default="precision", choices=["precision", "stress", "two-stage"],
                    help="precision: the 48x488x50 headline block; stress: 200 beams x 8 "
                         "trials x 262144 frames with injected pulses (recall)")
    ap.add_argument("--synth-frames", type=int, default=0,
                    help="fixed synthesis frames per thread block (0: autotune; -1: the "
                         "balanced tiling, one block per SM)")
    ap.add_argument("--fine", action="store_true",
                    help="fine (channel-domain) de-dispersion filter on (a separate line, "
                         "not the headline)")
    ap.add_argument("--fullrate", action="store_true",
                    help="full-rate de-dispersion of the synthesised series (2048-tap "
                         "overlap-save filter; a separate line, not the headline)")
    ap.add_argument("--lsmr", action="store_true",
                    help="PPF inversion by windowed LSMR instead of the FIR synthesis (a "
                         "separate line, not the headline; trigger on per-phase levels)")
    ap.add_argument("--gemm-config", type=int, default=-2,
                    help="fixed beamformer configuration index (-1: default; -2: autotune)")
    ap.add_argument("--chunk-frames", type=int, default=0,
                    help="beam rows for chunks of this many frames (multiple of 256; 0: the "
                         "whole block), with a first power-only beamformer pass")
    ap.add_argument("--graph", action="store_true",
                    help="replay each block's launches from a captured CUDA graph (on a side "
                         "stream; stage times are then not recorded)")
    ap.add_argument("--frames", type=int, default=0,
                    help="block length override for small profiling cases (not a bench line)")
    return ap.parse_args()


def bench_workload(args):
    w = synth.PRECISION
    if args.frames:
        import dataclasses
        w = dataclasses.replace(w, name=w.name.replace("65536fr", f"{args.frames}fr"),
                                block_len=args.frames)
    return w


def tiling(fpc):
    """Name of a synthesis tiling: frames per block, or the balanced tiling (0)."""
    return "balanced (one block per SM)" if fpc == 0 else fpc


def gemm_desc(precision, cfgs, index):
    """Readable name of beamformer configuration `index` (-1: the default)."""
    if index < 0:
        return "default"
    a, b = cfgs[index]
    return f"{a} beams per pass" if precision == "fp32" else f"input ring {a}, fp16 ring {b}"


def workload_config(w, precision):
    return {
        "workload": w.name.replace("fp16", precision),
        "stations": w.stations, "pols": w.pols, "subbands": w.subbands,
        "first_bin": w.first_bin, "beams": w.beams, "tec_trials": list(w.tec_trials),
        "block_frames": w.block_len, "input": w.dtype, "noise_sigma": w.noise_sigma,
        "beamformer": {"fp16": "tensor-core fp16 hi/lo, fp32 accumulate", "fp32": "fp32 fma",
                       "fp64-oracle": "fp64 direct station sum (CPU oracle)"}[precision],
        "synthesis": "fp64 radix-2 FFT + direct FIR (CPU oracle)" if precision == "fp64-oracle"
        else "fp32",
        "l2": "inputs larger than L2 (%.2f GB station block, %.1f GB beam intermediate)" % (
            w.input_bytes / 1e9, w.n_streams * w.subbands * w.block_len * 8 / 1e9),
        "block_seconds": w.block_len * M / FS_HZ,
    }


# ------------------------------------------------------------ clocks -------

from paper_1612_06592_gb300.clocks import ClockSampler  # noqa: E402


# ------------------------------------------------------------ inputs -------

def device_block(w, seed, device, contrib=None):
    """Seeded synthetic block on the device (Gaussian quantile table, rounded)."""
    return synth.device_noise_block(w, seed, device, contrib)


# ------------------------------------------------------------ CPU oracle ---

def oracle_sample(w, x_host_window, frames, chunk=2048):
    """Time the FP64 oracle on one stream (beam 0, trial 0, pol 0) over `frames`
    frames (in chunks of `chunk` frames with their 15 history frames).
    Returns seconds and the extrapolated seconds per block of the workload."""
    import oracle as O
    enu, dirs, tec = synth.make_geometry(w)
    nu = O.sky_frequencies(w.first_bin, w.subbands)
    wts = O.geometric_weights(nu, enu, dirs[:1])[:, 0, :]
    dd = O.dedispersion_weights(nu, tec, 0.5 * (nu[0] + nu[-1]))[:, 0]
    g = O.synthesis_filter()
    t0 = time.perf_counter()
    done = 0
    while done < frames:
        n = min(chunk, frames - done)
        lo = max(0, done - 15)
        sub = x_host_window[:, :, lo:done + n]
        u = O.stream_window(sub, wts, dd, 0, w.first_bin, g, done - lo, done - lo + n)
        env = np.abs(u)
        _ = int(np.count_nonzero(env > 1e30))
        done += n
    dt = time.perf_counter() - t0
    per_block = dt * w.n_streams * (w.block_len / frames)
    return dt, per_block


def cpu_baseline(w, x_dev, frames):
    xs = x_dev[:, :, :frames].cpu().numpy()
    dt, per_block = oracle_sample(w, xs, frames)
    block_s = w.block_len * M / FS_HZ
    return {"value": block_s / per_block, "unit": "x realtime", "cores": 1, "kind": "oracle",
            "sample": f"1 of {w.n_streams} streams x {frames} of {w.block_len} frames "
                      f"({dt:.1f} s, numpy FP64 single thread), scaled by streams x frames",
            "seconds_per_block_extrapolated": per_block}


# ------------------------------------------------------------ ncu traffic --

def code_digest(path):
    """Hash of a CUDA source with comments and whitespace removed, so that a
    recorded measurement stays attached to the code, not to its comments."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = re.sub(r"\s+", "", text)
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def recorded_traffic(kernel_file):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if it
    was taken on the current code of that kernel."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    src = os.path.join(ROOT, "paper_1612_06592_gb300", "csrc", kernel_file)
    try:
        rec = json.load(open(path))
        digest = code_digest(src)
        ent = rec.get(kernel_file)
        if ent and ent.get("source_sha256_16") == digest:
            return ent["bytes_per_full_launch"]
    except (OSError, ValueError, KeyError):
        pass
    return None


# ------------------------------------------------------------ ranks --------

def max_over_ranks(values, device=None):
    """Element-wise maximum over all ranks of a list of timings (the slowest
    rank sets the whole-job time); works with the nccl and gloo backends."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_rate(world, block_s, ms_step_max, sharded=False):
    """Realtime factor of the whole job: N replicas each processing one block
    per step, or (sharded) N ranks sharing the beams of one block per step."""
    return (1 if sharded else world) * block_s / (ms_step_max / 1e3)


# ------------------------------------------------------------ main ---------

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1612_06592_gb300 import build
    build()
    from paper_1612_06592_gb300 import lp

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = bench_workload(args)
    enu, dirs, tec = synth.make_geometry(w)
    sharded = world > 1 and args.shard == "beams"
    # beam sharding: every rank holds the same block (its own copy on its own
    # GPU) and runs its beams; replicas: every rank its own block
    x = device_block(w, 1000 if sharded else 1000 + rank, dev)
    e2e_stream = not args.no_e2e and not args.lsmr and not args.graph and not args.fullrate
    plan_kw = dict(input_dtype=w.dtype, precision=args.precision, first_bin=w.first_bin,
                   host_input=not args.no_e2e and not args.lsmr, stream_blocks=e2e_stream,
                   frames_per_cta=max(0, args.synth_frames), fine_dedisp=args.fine,
                   fullrate_dedisp=args.fullrate,
                   inversion="lsmr" if args.lsmr else "fir", chunk_frames=args.chunk_frames,
                   use_graph=args.graph)
    if args.graph:
        torch.cuda.set_stream(torch.cuda.Stream())   # graph capture needs a non-default stream
    shard = None
    if sharded:
        from paper_1612_06592_gb300.shard import BeamShard
        shard = BeamShard(w.stations, w.pols, w.subbands, w.beams, len(w.tec_trials),
                          w.block_len, rank=rank, world=world, **plan_kw)
        plan = shard.plan
        shard.lp_set_weights(enu, dirs)
    else:
        plan = lp.Plan(w.stations, w.pols, w.subbands, w.beams, len(w.tec_trials), w.block_len,
                       **plan_kw)
        plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    n_streams_local = plan.shape[3] * plan.shape[4] * plan.shape[1]
    stream = torch.cuda.current_stream()
    # untimed blocks pick the beamformer configuration and the synthesis tiling
    # (autotuners), then warm-up
    gemm_cfgs = plan.lp_plan_gemm_configs()
    if args.gemm_config >= -1:
        plan.lp_plan_set_gemm_config(args.gemm_config)
        gemm_best, gemm_ms = args.gemm_config, {}
    else:
        gemm_best, gemm_ms = plan.lp_plan_autotune_gemm(x)
    if args.synth_frames or args.lsmr:
        tuned_fpc, tune_ms = max(0, args.synth_frames), {}
    else:
        tuned_fpc, tune_ms = plan.lp_plan_autotune(x)
    plan.lp_profile_enable(not args.graph)
    for _ in range(args.warmup):
        plan.lp_process_block(x)
    torch.cuda.synchronize()
    plan.lp_profile_read()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.lp_process_block(x)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stages, nrec = plan.lp_profile_read()
    _, ntrig, _ = plan.lp_get_triggers()

    # end to end through the same API from pinned host memory, triggers back
    e2e = None
    if not args.no_e2e:
        xh = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        xh.copy_(x)
        for _ in range(2):
            plan.lp_process_block(xh)
            plan.lp_get_triggers()
        barrier()
        torch.cuda.synchronize()
        plan.lp_profile_read()
        t0 = time.perf_counter()
        d2h = 0

        def read(block):
            # streaming host blocks: block `block`'s triggers are read while the
            # next block's copy and kernels run (otherwise the last block's, after it)
            t, n, _ = (plan.lp_get_triggers_block(block) if e2e_stream
                       else plan.lp_get_triggers())
            if shard is not None:
                # this rank's triggers relabelled to global beams, merged on rank 0
                from paper_1612_06592_gb300.shard import gather_triggers, to_global
                gather_triggers(to_global(t, shard.b0, shard.tec_trials, shard.pols))
            return t

        for i in range(args.steps):
            plan.lp_process_block(xh)
            if not e2e_stream:
                d2h += 8 + 32 * len(read(plan.blocks - 1))
            elif i:
                d2h += 8 + 32 * len(read(plan.blocks - 2))
        if e2e_stream:
            d2h += 8 + 32 * len(read(plan.blocks - 1))
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        barrier()
        e2e_stages, n_e2e = plan.lp_profile_read()
        e2e = (t_e2e, d2h / args.steps, x.numel() * x.element_size())

    if world > 1:
        ms, t_max_e2e = max_over_ranks([ms, e2e[0] if e2e else 0.0], dev)
        if e2e:
            e2e = (t_max_e2e, e2e[1], e2e[2])
    if rank != 0:
        return None

    block_s = w.block_len * M / FS_HZ
    ms_step = ms / args.steps
    rtf = whole_job_rate(world, block_s, ms_step, sharded)
    blocks_per_step = 1 if sharded else world
    synth_ms = stages["synth"] / max(nrec, 1)
    bf_ms = stages["beamform"] / max(nrec, 1)
    samples = w.n_streams * w.block_len * M
    # the roofline is rank 0's own synthesis launch (its share of the beams)
    flop = n_streams_local * w.block_len * M * SYNTH_FLOP_PER_SAMPLE
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    alu_peak, alu_peak_mhz, alu_peak_note = fp32_peak()
    achieved = flop / (synth_ms / 1e3) / 1e12 if synth_ms > 0 else float("nan")
    traffic = recorded_traffic("k_ippf.cu")
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    in_bytes = x.numel() * x.element_size()
    beams_bytes = n_streams_local * w.subbands * w.block_len * 8
    bf_gbs = (in_bytes + beams_bytes) / (bf_ms / 1e3) / 1e9 if bf_ms > 0 else float("nan")
    line = {
        "metric": "realtime factor at 48 stations×488 subbands×50 beams",
        "value": rtf, "unit": "x realtime", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": "f16 tensor-core beamformer, f32" if args.precision == "fp16" else "f32",
        "data": "synthetic (seeded rounded-Gaussian int8 station noise)",
        "config": dict(workload_config(w, args.precision), synth_frames_per_cta=tiling(tuned_fpc),
                       parallelism=(f"beams sharded over {world} GPUs (ranks own contiguous "
                                    "beam ranges of one block; triggers merged on rank 0)"
                                    if sharded else f"{world} replica(s), one block each"),
                       autotune_ms={str(tiling(k)): round(v, 3) for k, v in tune_ms.items()},
                       gemm_config=gemm_desc(args.precision, gemm_cfgs, gemm_best),
                       gemm_autotune_ms={gemm_desc(args.precision, gemm_cfgs, gemm_cfgs.index(k)):
                                         round(v, 3) for k, v in gemm_ms.items()}),
        "samples_per_s": {"station_complex": w.pols * w.subbands * w.block_len * w.stations
                          * blocks_per_step / (ms_step / 1e3),
                          "output_200MHz": samples * blocks_per_step / (ms_step / 1e3)},
        "stage_ms": {k: v / max(nrec, 1) for k, v in stages.items()
                     if (k != "fine" or args.fine) and (k != "fullrate" or args.fullrate)},
        "roofline": {"bound": "alu", "kernel": "k_ippf (inverse FFT + synthesis FIR + trigger)",
                     "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak, "traffic": traffic,
                     "peak_note": alu_peak_note,
                     "flop_per_sample": SYNTH_FLOP_PER_SAMPLE,
                     "frac_at_sampled_clock": (achieved / (alu_peak * clk["sm_mhz"] / alu_peak_mhz))
                     if clk.get("sm_mhz") and alu_peak_mhz else None},
        "roofline_beamform": {"bound": "hbm", "achieved": bf_gbs, "peak": hbm_peak,
                              "unit": "GB/s", "frac": bf_gbs / hbm_peak,
                              "bytes": in_bytes + beams_bytes,
                              "traffic": recorded_traffic("k_beamform_tc.cu")
                              if args.precision == "fp16" else None,
                              "note": "input read + FP32 beam intermediate write",
                              "write4_peak": write4_bandwidth(),
                              "frac_of_write4": (bf_gbs / write4_bandwidth()
                                                 if write4_bandwidth() else None),
                              "write4_note": "streaming kernel reading each word once and "
                                             "writing it four times (profiles/hbm_mix.json)"},
        "gpu_launches": plan.lp_launches_per_block() * args.steps,
        "triggers_last_block": int(ntrig),
        "clocks": clk,
    }
    if e2e:
        t_e2e, d2h, h2d = e2e
        line["e2e"] = {"value": blocks_per_step * block_s / (t_e2e / args.steps), "unit": "x realtime",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "ms_per_step": t_e2e / args.steps * 1e3,
                       "path": ("lp_process_block(pinned host block, streaming: the next "
                                "block's host copy overlaps this block's kernels) + "
                                "lp_get_triggers_block of the previous block each step"
                                if e2e_stream else
                                "lp_process_block(pinned host block: copy per polarisation, "
                                "then the kernels) + lp_get_triggers each step"),
                       "stage_ms": {k: v / max(n_e2e, 1) for k, v in e2e_stages.items()}}
    if args.fine:
        fine_ms = stages["fine"] / max(nrec, 1)
        fine_bytes = 2 * beams_bytes                      # beam rows read + filtered rows written
        line["metric"] += ", fine de-dispersion on"
        line["config"]["workload"] += "-fine"
        line["config"]["fine_dedispersion"] = "17-tap channel-domain filter per (subband, trial)"
        line["roofline_fine"] = {"bound": "hbm", "kernel": "k_fine",
                                 "achieved": fine_bytes / (fine_ms / 1e3) / 1e9,
                                 "peak": hbm_peak, "unit": "GB/s",
                                 "frac": fine_bytes / (fine_ms / 1e3) / 1e9 / hbm_peak,
                                 "bytes": fine_bytes,
                                 "traffic": recorded_traffic("k_fine.cu")}
    if args.fullrate:
        fr_ms = stages["fullrate"] / max(nrec, 1)
        # per 8192-point segment (6144 outputs): forward and inverse transforms
        # (5 N log2 N each) and the product with the taps' spectrum (6 N)
        fr_flop = (2 * 5 * 8192 * 13 + 6 * 8192) / 6144 * samples
        fr_bytes = samples * 8 * 8192 / 6144               # series rows read (segments overlap)
        line["metric"] += ", full-rate de-dispersion on"
        line["config"]["workload"] += "-fullrate"
        line["config"]["fullrate_dedispersion"] = ("2048-tap streaming filter of the synthesised "
                                                   "series (8192-point overlap-save), whole STEC "
                                                   "phase at full rate")
        line["roofline_fullrate"] = {"bound": "alu", "kernel": "k_fullrate" + (
                                         " (stage time with the series transpose, the per-phase "
                                         "noise level and the trigger of the LSMR path)"
                                         if args.lsmr else ""),
                                     "achieved": fr_flop / (fr_ms / 1e3) / 1e12,
                                     "peak": alu_peak, "unit": "TFLOP/s",
                                     "frac": fr_flop / (fr_ms / 1e3) / 1e12 / alu_peak,
                                     "flop_per_sample": fr_flop / samples,
                                     "hbm_gbs": fr_bytes / (fr_ms / 1e3) / 1e9,
                                     "traffic": recorded_traffic("k_fullrate.cu")}
    if args.lsmr:
        # per window and LSMR step: A v and A^T u (272 x 16 complex x real taps,
        # 4 FLOP each), two norms and two scalings of 287-element vectors, the
        # h / hbar / x updates; plus the start (one norm, A^T u, one norm)
        rows, cols, taps, iters = 272, 287, 16, 25
        per_step = 2 * rows * taps * 4 + 2 * cols * 4 + 2 * cols * 2 + 3 * cols * 4
        per_window = iters * per_step + rows * taps * 4 + rows * 4 + cols * 4
        windows = w.n_streams * M * (w.block_len // 256)
        inv_ms = stages["synth"] / max(nrec, 1)
        ach = windows * per_window / (inv_ms / 1e3) / 1e12
        line["metric"] = line["metric"].replace("realtime factor", "realtime factor, LSMR PPF "
                                                "inversion (per-phase level and trigger),")
        line["config"]["workload"] += "-lsmr"
        line["config"]["inversion"] = ("windowed LSMR: 256-frame windows, 16 frames of "
                                       "overlap, 25 iterations, per stream and phase")
        line["roofline"] = {"bound": "alu", "kernel": "k_ippf (inverse DFT only) + k_lsmr (with k_lsmr_sigma + k_lsmr_trigger unless --fullrate)",
                            "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                            "frac": ach / alu_peak, "traffic": None,
                            "flop_per_window": per_window, "windows": windows,
                            "peak_note": line["roofline"]["peak_note"]}
        line.pop("e2e", None)
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w, x, min(args.cpu_sample_frames, w.block_len))
    if args.serve_blocks > 0 and not args.frames:
        plan.close()
        del x
        torch.cuda.empty_cache()
        from paper_1612_06592_gb300 import serve
        sargs = serve.build_parser().parse_args(["--blocks", str(args.serve_blocks),
                                                 "--precision", args.precision])
        line["serving"] = serve.run(sargs)
    return line


def run_stress(args):
    """200 beams x 8 STEC trials x 262144 frames (1.34 s blocks) with 200 pulses:
    chunked processing (the beam intermediate of a whole block would be 3.3 TB),
    realtime factor and trigger recall against the injected pulses."""
    import torch
    from paper_1612_06592_gb300 import build
    build()
    from paper_1612_06592_gb300 import lp
    w = synth.STRESS
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    enu, dirs, tec = synth.make_geometry(w)
    plist, contrib = synth.pulse_contributions(w, 0, enu, dirs)
    x = device_block(w, 5000, dev, contrib)     # pulses added before rounding
    chunk = 8192
    stream = torch.cuda.Stream()                  # graph mode needs a non-default stream
    plan = lp.Plan(w.stations, w.pols, w.subbands, w.beams, len(tec), w.block_len,
                   input_dtype="int8", precision="fp16", first_bin=w.first_bin,
                   chunk_frames=chunk, trigger_cap=1 << 22, use_graph=True, stream=stream)
    plan.lp_set_weights(enu, dirs, stream=stream)
    plan.lp_set_tec(tec, stream=stream)
    # beamformer configuration and synthesis tiling by the autotuners (timed on
    # the block's first chunk)
    gemm_cfgs = plan.lp_plan_gemm_configs()
    gemm_best, gemm_ms = plan.lp_plan_autotune_gemm(x, stream=stream)
    tuned_fpc, tune_ms = plan.lp_plan_autotune(x, stream=stream)
    for _ in range(max(1, args.warmup)):          # the first block captures the graph
        plan.lp_reset_stream(stream=stream)       # every timed block is block 0 of the stream
        plan.lp_process_block(x, stream=stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 3))
    ms_tot = 0.0
    for _ in range(steps):
        plan.lp_reset_stream(stream=stream)
        e0.record(stream)
        plan.lp_process_block(x, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_tot += e0.elapsed_time(e1)
    clk = clocks.stop()
    trig, n_trig, st = plan.lp_get_triggers()
    ms = ms_tot / steps
    block_s = w.block_len * M / FS_HZ
    # recall: a pulse counts when its beam has a trigger near the arrival time of
    # some trial; the de-dispersed pulse sits at n0 + A_trial / nu_ref^2 (A =
    # 40.308 m^3/s^2 * STEC / c, nu_ref the centre of the selected band)
    nu_lo = FS_HZ / 2 + w.first_bin * FS_HZ / M
    nu_hi = FS_HZ / 2 + (w.first_bin + w.subbands - 1) * FS_HZ / M
    nu_ref = 0.5 * (nu_lo + nu_hi)
    delay = 40.308 * np.asarray(tec) * 1e16 / 299792458.0 / nu_ref ** 2 * FS_HZ
    by_beam = {}
    for r in trig:
        by_beam.setdefault(int(r["beam"]), []).append((int(r["n"]), int(r["tec"])))
    found, snrs, used = [], [], set()
    for p in plist:
        hit = False
        for (n, t) in by_beam.get(p.beam, []):
            if abs(n - (p.n0 + delay[t])) <= 512:
                hit = True
                used.add((p.beam, n, t))
        found.append(hit)
        snrs.append(p.snr)
    found, snrs = np.array(found), np.array(snrs)
    bins = [(5, 10), (10, 15), (15, 20.01)]
    samples = w.n_streams * w.block_len * M
    chunk_tflops = (w.n_streams * chunk * M * SYNTH_FLOP_PER_SAMPLE /
                    (tune_ms[tuned_fpc] / 1e3) / 1e12)
    return {
        "workload": w.name, "metric": "realtime factor at 48x488x200 beams x 8 trials",
        "value": block_s / (ms / 1e3), "unit": "x realtime", "ms_per_block": ms,
        "block_seconds": block_s, "chunk_frames": chunk,
        "launches_per_block": plan.lp_launches_per_block(),
        "output_samples_per_s": samples / (ms / 1e3),
        "synth_tflops": samples * SYNTH_FLOP_PER_SAMPLE / (ms / 1e3) / 1e12,
        "pulses": len(plist), "recall": float(found.mean()),
        "recall_by_snr": {f"{a}-{int(b)}": float(found[(snrs >= a) & (snrs < b)].mean())
                          for a, b in bins},
        "synth_frames_per_cta": tiling(tuned_fpc),
        "autotune_ms_per_chunk": {str(tiling(k)): round(v, 3) for k, v in tune_ms.items()},
        "gemm_config": gemm_desc("fp16", gemm_cfgs, gemm_best),
        "gemm_autotune_ms_per_chunk": {gemm_desc("fp16", gemm_cfgs, gemm_cfgs.index(k)): round(v, 3)
                                       for k, v in gemm_ms.items()},
        "cuda_graph": True,
        "roofline": {"bound": "alu", "kernel": "k_ippf", "basis": "autotuner's CUDA-event time of the synthesis of one 8192-frame chunk",
                     "achieved": chunk_tflops, "peak": fp32_peak_tflops(), "unit": "TFLOP/s",
                     "frac": chunk_tflops / fp32_peak_tflops()},
        "triggers": int(n_trig), "trigger_status": int(st),
        "triggers_not_near_a_pulse": int(len(trig) - sum(
            1 for r in trig if (int(r["beam"]), int(r["n"]), int(r["tec"])) in used)),
        "clocks": clk, "data": "synthetic (device noise + host-built dispersed pulses)",
    }


def run_two_stage(args):
    """Two-stage beamforming at the precision configuration: the 48 stations in
    8 compact groups form 8 int16 preliminary beams toward the pointing centre
    (lp_prebeam), from which the 50 final beams, the synthesis and the triggers
    follow (an lp_plan with the group centres as its 8 stations; FP16 tensor-core
    form, int16 samples entering as two exact FP16 parts).  One step = both
    stages on one block."""
    import torch
    from paper_1612_06592_gb300 import build
    build()
    from paper_1612_06592_gb300 import lp
    w = bench_workload(args)
    G, scale = 8, 4.0
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    enu, dirs, tec = synth.make_geometry(w)
    x = device_block(w, 1000, dev)
    grp = synth.station_groups(enu, G)
    pb = lp.Prebeam(w.stations, w.pols, w.subbands, w.block_len, G, first_bin=w.first_bin,
                    input_dtype=w.dtype)
    pb.lp_prebeam_set_groups(grp, enu, np.tile(synth.pointing_enu(), (G, 1)))
    y = torch.empty((w.pols, w.subbands, w.block_len, G, 2), dtype=torch.int16, device=dev)
    plan = lp.Plan(G, w.pols, w.subbands, w.beams, len(tec), w.block_len, input_dtype="int16",
                   precision="fp16", first_bin=w.first_bin)
    plan.lp_set_weights(pb.lp_prebeam_group_centres(), dirs)
    plan.lp_set_tec(tec)
    stream = torch.cuda.current_stream()
    pb.lp_prebeam_run(x, y, scale)
    gemm_cfgs = plan.lp_plan_gemm_configs()
    gemm_best, gemm_ms = plan.lp_plan_autotune_gemm(y)
    tuned_fpc, tune_ms = plan.lp_plan_autotune(y)
    for _ in range(max(3, args.warmup)):
        pb.lp_prebeam_run(x, y, scale)
        plan.lp_process_block(y)
    torch.cuda.synchronize()
    pb.lp_prebeam_saturated()
    plan.lp_profile_enable(True)
    clocks = ClockSampler(0)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for a, b in ev:
        a.record(stream)
        pb.lp_prebeam_run(x, y, scale)
        b.record(stream)
        plan.lp_process_block(y)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_step = e0.elapsed_time(e1) / args.steps
    pre_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    stages, nrec = plan.lp_profile_read()
    n_sat = pb.lp_prebeam_saturated()
    block_s = w.block_len * M / FS_HZ
    in_bytes = x.numel() * x.element_size()
    out_bytes = y.numel() * y.element_size()
    hbm_peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    pre_gbs = (in_bytes + out_bytes) / (pre_ms / 1e3) / 1e9
    # the frame-pair kernel takes int8 input, a multiple of 8 stations and 4, 8 or 16 groups
    pre_kernel = ("k_prebeam_pairs" if w.dtype == "int8" and w.stations % 8 == 0
                  and G in (4, 8, 16) else "k_prebeam")
    return {
        "metric": "realtime factor, two-stage beamforming (48 stations in 8 groups) x 488 "
                  "subbands x 50 beams",
        "value": block_s / (ms_step / 1e3), "unit": "x realtime", "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16 tensor-core beamformer (int16 preliminary beams), f32", "data":
        "synthetic (seeded rounded-Gaussian int8 station noise)",
        "config": dict(workload_config(w, "fp16"), workload="two-stage-48st-8grp-488sb-50bm-"
                       f"{w.block_len}fr", groups=G, group_sizes=np.bincount(grp).tolist(),
                       preliminary_direction="pointing centre", transport="complex int16",
                       scale=scale, synth_frames_per_cta=tiling(tuned_fpc),
                       gemm_config=gemm_desc("fp16", gemm_cfgs, gemm_best),
                       gemm_autotune_ms={gemm_desc("fp16", gemm_cfgs, gemm_cfgs.index(k)):
                                         round(v, 3) for k, v in gemm_ms.items()}),
        "stage_ms": dict({"prebeam": pre_ms}, **{k: v / max(nrec, 1) for k, v in stages.items()
                                                  if k not in ("h2d", "fine")}),
        "roofline_prebeam": {"bound": "hbm", "kernel": pre_kernel, "achieved": pre_gbs,
                             "peak": hbm_peak, "unit": "GB/s", "frac": pre_gbs / hbm_peak,
                             "bytes": in_bytes + out_bytes,
                             "note": "station block read + int16 preliminary beams written"},
        "saturated_codes_per_block": n_sat / args.steps,
        "gpu_launches": args.steps * (1 + plan.lp_launches_per_block()),
        "clocks": clk,
    }


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = synth.PRECISION
    frames = 2048
    rng = np.random.default_rng(7)
    table = synth.gaussian_table(w.noise_sigma, w.dtype)
    xs = table[rng.integers(0, 65536, size=(w.pols, w.subbands, frames, w.stations, 2))]
    for _ in range(args.warmup):
        oracle_sample(w, xs, frames)
    t0 = time.perf_counter()
    per = []
    for _ in range(args.steps):
        per.append(oracle_sample(w, xs, frames)[1])
    dt = time.perf_counter() - t0
    block_s = w.block_len * M / FS_HZ
    per_block = float(np.mean(per))
    v = block_s / per_block
    return {
        "impl": "reference", "metric": "realtime factor at 48 stations×488 subbands×50 beams",
        "value": v, "unit": "x realtime", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_block * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, "fp64-oracle"),
        "cpu_baseline": {"value": v, "unit": "x realtime", "cores": 1, "kind": "oracle",
                         "sample": f"per step 1 of {w.n_streams} streams x {frames} frames, "
                                   "scaled by streams x frames"},
        "e2e": {"value": v, "unit": "x realtime", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": dt,
    }


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.workload == "stress":
        line = run_stress(args) if rank == 0 else None
    elif args.workload == "two-stage":
        line = run_two_stage(args) if rank == 0 else None
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        line = run_ours(args, rank, world, local_rank)
        if (line is not None and world == 1 and args.stress_blocks > 0 and not args.frames
                and not args.fine and not args.lsmr and args.precision == "fp16"):
            import copy
            import torch
            torch.cuda.empty_cache()
            sargs = copy.copy(args)
            sargs.steps, sargs.warmup = args.stress_blocks, 1
            line["stress"] = run_stress(sargs)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
