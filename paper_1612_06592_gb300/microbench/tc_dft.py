"""Time the tensor-core lower bound of the two inverse-DFT stages (tc_dft_bound.cu).

    python -m paper_1612_06592_gb300.microbench.tc_dft [--out profiles/tc_dft_bound.json]

For each shape (0: the DFT's 576 MMAs of N = 64 per 128-frame tile; 1: the same
FLOP as 144 MMAs of N = 256) it records the MMA rate of all SMs and the time
the two stages would take, on the tensor cores alone, for the 48 x 488 x 50
block (100 streams x 65536 frames = 51200 tiles), next to the measured bf16
peak.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
TILES_PER_BLOCK = 100 * 65536 // 128


def measure(tiles: int = 2048, reps: int = 5) -> dict:
    import torch
    from paper_1612_06592_gb300.build import MB_LIB, build
    from paper_1612_06592_gb300.clocks import ClockSampler
    build()
    lib = ctypes.CDLL(MB_LIB)
    lib.mb_tc_dft_run.restype = ctypes.c_int
    lib.mb_tc_dft_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_double)]
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    out = {}
    for shape in (0, 1):
        n_mma = lib.mb_tc_dft_mmas_per_tile(shape)
        n = lib.mb_tc_dft_n(shape)
        clocks = ClockSampler(dev)
        clocks.start()
        ms = ctypes.c_double(0.0)
        rc = lib.mb_tc_dft_run(shape, tiles, reps, err.data_ptr(), ctypes.byref(ms))
        clk = clocks.stop()
        if rc != 0:
            raise RuntimeError(f"mb_tc_dft_run({shape}) failed with cudaError {rc}")
        if int(err.item()):
            raise RuntimeError("a bounded wait gave up")
        mmas = sms * tiles * n_mma
        flop = mmas * 2.0 * 128 * n * 16
        tflops = flop / (ms.value / 1e3) / 1e12
        out["dft_n64" if shape == 0 else "same_flop_n256"] = {
            "mma_shape": f"M128 N{n} K16 kind::f16, both operands in shared memory",
            "mmas_per_tile": n_mma, "ms_per_launch": ms.value, "tiles_per_sm": tiles,
            "tflops": tflops,
            "ms_per_48x488x50_block": ms.value * TILES_PER_BLOCK / (sms * tiles),
            "clocks": clk,
        }
    bf16 = peaks.get("bf16_tflops")
    for v in out.values():
        v["frac_of_measured_bf16"] = v["tflops"] / bf16 if bf16 else None
    return {"what": "tensor-core lower bound of the two 32-point inverse-DFT stages "
                    "(MMAs only: no loads, conversions, twiddles, transposes or epilogue)",
            "tiles_per_block": TILES_PER_BLOCK, "shapes": out, "bf16_tflops_measured": bf16,
            "command": "python -m paper_1612_06592_gb300.microbench.tc_dft"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "profiles", "tc_dft_bound.json"))
    args = ap.parse_args()
    rec = measure()
    with open(args.out, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps({k: (round(v["ms_per_48x488x50_block"], 3), round(v["tflops"], 1))
                      for k, v in rec["shapes"].items()}))


if __name__ == "__main__":
    main()
