"""Measure streaming HBM bandwidth at the beamformer's read/write mix and record it.

    python -m paper_1612_06592_gb300.microbench.hbm [--out profiles/hbm_mix.json]

Times hbm_mix.cu with CUDA events for fan = 1 (a copy: every word read once and
written once) and fan = 4 (read once, written four times: the tensor-core
beamformer's 6.14 GB read to 25.6 GB written at 48 x 488 x 50), 6 GB of input
in both cases (far larger than L2), while ``nvidia-smi`` samples the SM clock.
The pipeline's HBM fractions keep dividing by the driver's measured copy
bandwidth; this record says how far a kernel that writes four times what it
reads can get at all.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def measure(in_gb: float = 6.0, reps: int = 5, blocks_per_sm: int = 4) -> dict:
    import torch
    from paper_1612_06592_gb300.build import MB_LIB, build
    from paper_1612_06592_gb300.clocks import ClockSampler
    build()
    lib = ctypes.CDLL(MB_LIB)
    lib.mb_mix_run.restype = ctypes.c_int
    lib.mb_mix_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    n = int(in_gb * 1e9) // 16
    src = torch.ones(n * 4, dtype=torch.float32, device="cuda")
    res = {}
    for fan in (1, 4):
        dst = torch.empty(n * 4 * fan, dtype=torch.float32, device="cuda")
        clocks = ClockSampler(dev)
        clocks.start()
        time.sleep(0.3)
        ms = ctypes.c_double(0.0)
        rc = lib.mb_mix_run(src.data_ptr(), dst.data_ptr(), n, fan,
                            props.multi_processor_count * blocks_per_sm, reps, ctypes.byref(ms))
        clk = clocks.stop()
        if rc != 0:
            raise RuntimeError(f"mb_mix_run(fan={fan}) failed with cudaError {rc}")
        moved = 16.0 * n * (1 + fan)
        res[f"fan{fan}"] = {"bytes_per_launch": moved, "ms_per_launch": ms.value,
                            "gbs": moved / (ms.value / 1e3) / 1e9, "clocks": clk}
        del dst
        torch.cuda.empty_cache()
    return {
        "what": "streaming HBM bandwidth, each 16-byte word read once and written fan times",
        "gpu": props.name, "input_gb": 16.0 * n / 1e9,
        "grid": f"{props.multi_processor_count * blocks_per_sm} blocks x 512 threads",
        "forms": res,
        "write4_over_copy": res["fan4"]["gbs"] / res["fan1"]["gbs"],
        "command": "python -m paper_1612_06592_gb300.microbench.hbm",
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "profiles", "hbm_mix.json"))
    args = ap.parse_args()
    rec = measure()
    with open(args.out, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps({k: (v["gbs"] if isinstance(v, dict) and "gbs" in v else v)
                      for k, v in rec["forms"].items()}))


if __name__ == "__main__":
    main()
