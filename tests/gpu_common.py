"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded inputs, and compare.

Tolerances (derived from the arithmetic, stated once here):
  * FP32 form: beams carry FP32 weights (~6e-8) and FP32 sums over <= 64
    stations; the 1024-point FFT adds ~log2(1024) roundings of ~6e-8 and the
    16-tap FIR a few more: relative RMS errors of ~1e-6 are expected, the
    tests allow TOL_TS_FP32 = 2e-5 on the time series and beams.
  * FP16 tensor-core form: weights as FP16 hi + lo (~2^-22 relative), int8
    samples exact, FP32 accumulation: ~1e-6 as well; the pipeline's stated
    target is 1e-4, the tests allow TOL_TS_FP16 = 1e-4.
  * Triggers: both lists must agree except for samples whose oracle envelope
    lies within TAU * theta of the threshold (TAU = 1e-5 FP32, 1e-4 FP16).
"""

from __future__ import annotations

import numpy as np

import oracle as O
import synth

TOL_TS_FP32 = 2e-5
TOL_TS_FP16 = 1e-4
TAU_FP32 = 1e-5
TAU_FP16 = 1e-4


def rel_rms(got, ref):
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.sqrt(np.mean(np.abs(got - ref) ** 2) / np.mean(np.abs(ref) ** 2)))


def make_plan(lp, S, P, K, B, Tr, F, first_bin, dtype, precision="fp32", **kw):
    return lp.Plan(S, P, K, B, Tr, F, input_dtype=dtype, precision=precision,
                   first_bin=first_bin, **kw)


def gpu_blocks(lp, plan, blocks, enu, dirs, tec, want_ts=True):
    """Run blocks through the plan; per block: dict(y [J,F*M], beams, trig, sigma)."""
    import torch
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    S, P, K, B, Tr, F = plan.shape
    outs = []
    for xb in blocks:
        xd = torch.from_numpy(np.ascontiguousarray(xb)).cuda()
        plan.lp_process_block(xd)
        trig, n, st = plan.lp_get_triggers()
        o = {"trig": trig, "n_trig": n, "status": st, "sigma": plan.lp_get_sigma()}
        if want_ts:
            ys, bms = [], []
            for b in range(B):
                for t in range(Tr):
                    for p in range(P):
                        ys.append(plan.lp_get_timeseries(b, t, p))
                        bms.append(plan.lp_get_beams(b, t, p))
            o["y"] = np.stack(ys)
            o["beams"] = np.stack(bms)          # [J, K, F]
        outs.append(o)
        del xd
    return outs


def oracle_blocks(S, P, K, B, Tr, F, first_bin, blocks, enu, dirs, tec, k_sigma=6.0):
    pipe = O.Pipeline(S, P, K, B, Tr, F, first_bin, enu, dirs, np.asarray(tec), k_sigma=k_sigma)
    return pipe, [pipe.process_block(xb) for xb in blocks]


def trigger_set(trig_rows):
    return {(int(r["stream"]), int(r["n"])) for r in trig_rows}


def compare_triggers(gpu_trig, ora, P, Tr, tau):
    """Symmetric difference of trigger sets, each element inside the band."""
    ora_set = set()
    for (n, b, t, p, e, s) in ora["triggers"]:
        ora_set.add(((b * Tr + t) * P + p, n))
    g = trigger_set(gpu_trig)
    diff = g ^ ora_set
    bad = []
    for (j, n) in diff:
        i = n - ora["n_first"]
        env = ora["env"][j, i]
        th = ora["theta"][j]
        if abs(env - th) > tau * th:
            bad.append((j, n, env, th))
    return len(g), len(ora_set), len(diff), bad


def random_case(seed, S, P, K, B, Tr, F, first_bin, dtype="int16", nblocks=1, amp=40):
    rng = np.random.default_rng(seed)
    info = np.iinfo(dtype)
    lo, hi = max(info.min, -amp), min(info.max, amp)
    blocks = [rng.integers(lo, hi + 1, size=(P, K, F, S, 2)).astype(dtype) for _ in range(nblocks)]
    enu = synth.station_positions(S, seed)
    dirs = synth.hex_beam_directions(B) if B > 1 else synth.pointing_enu()[None]
    tec = np.linspace(3.0, 30.0, Tr)
    return blocks, enu, dirs, tec
