"""Measure the FP32 FMA peak of the current GPU and record it.

    python -m paper_1612_06592_gb300.microbench.peaks [--out profiles/fp32_peak.json]

Times scalar FFMA and packed FFMA2 chains on every SM (fma_peak.cu) with CUDA
events, the grid a multiple of the SM count, while ``nvidia-smi`` samples the
SM clock; records the best of several timed launches per form, the median SM
clock under load, the rate per SM and clock (FLOP / (SM * cycle)) and whether
FFMA2 raises the lane rate.  The pipeline's ALU roofline fractions divide by
the larger of the two measured rates.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def _lib():
    from paper_1612_06592_gb300.build import MB_LIB, build
    build()
    lib = ctypes.CDLL(MB_LIB)
    lib.mb_fma_flop.restype = ctypes.c_double
    lib.mb_fma_flop.argtypes = [ctypes.c_int] * 4
    lib.mb_fma_run.restype = ctypes.c_int
    lib.mb_fma_run.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p,
                                                    ctypes.POINTER(ctypes.c_double)]
    return lib


def measure(iters: int = 65536, reps: int = 5, rounds: int = 3, blocks_per_sm: int = 8,
            threads: int = 256) -> dict:
    import torch
    from paper_1612_06592_gb300.clocks import ClockSampler
    lib = _lib()
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    blocks = sms * blocks_per_sm
    out = torch.empty(blocks * threads, dtype=torch.float32, device="cuda")
    res = {}
    for variant, name in ((0, "ffma"), (1, "ffma2")):
        flop = lib.mb_fma_flop(variant, blocks, threads, iters)
        clocks = ClockSampler(dev)
        clocks.start()
        time.sleep(0.3)
        best = None
        times = []
        for _ in range(rounds):
            ms = ctypes.c_double(0.0)
            rc = lib.mb_fma_run(variant, blocks, threads, iters, reps, out.data_ptr(),
                                ctypes.byref(ms))
            if rc != 0:
                raise RuntimeError(f"mb_fma_run({name}) failed with cudaError {rc}")
            times.append(ms.value)
            best = ms.value if best is None else min(best, ms.value)
        clk = clocks.stop()
        tflops = flop / (best / 1e3) / 1e12
        mhz = clk.get("sm_mhz")
        res[name] = {
            "tflops": tflops,
            "ms_per_launch_best": best, "ms_per_launch_all": times,
            "flop_per_launch": flop,
            "flop_per_sm_per_cycle": (tflops * 1e12 / (sms * mhz * 1e6)) if mhz else None,
            "clocks": clk,
        }
    best_name = max(res, key=lambda k: res[k]["tflops"])
    ratio = res["ffma2"]["tflops"] / res["ffma"]["tflops"]
    return {
        "what": "FP32 fused multiply-add peak, all SMs, CUDA events",
        "gpu": props.name, "sms": sms, "grid": f"{blocks} blocks x {threads} threads "
        f"({blocks_per_sm} per SM), 8 independent chains per thread",
        "forms": res,
        "peak_tflops": res[best_name]["tflops"],
        "peak_form": best_name,
        "ffma2_over_ffma": ratio,
        "reading": ("FFMA2 doubles the lane rate" if ratio > 1.5 else
                    "FFMA2 issues half the instructions at the same lane rate"),
        "command": "python -m paper_1612_06592_gb300.microbench.peaks",
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "profiles", "fp32_peak.json"))
    ap.add_argument("--iters", type=int, default=65536)
    args = ap.parse_args()
    rec = measure(iters=args.iters)
    with open(args.out, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps({k: rec[k] for k in ("peak_tflops", "peak_form", "ffma2_over_ffma",
                                          "reading")}))


if __name__ == "__main__":
    main()
