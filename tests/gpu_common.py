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
  * Per sample (assert_samples_close), on top of the relative RMS: every sample
    must satisfy |y - y_ref| <= C * eps * (sigma_y + env_local), eps = 2^-24,
    sigma_y the stream's noise level and env_local the largest oracle envelope
    within 16 frames of the sample (the FIR reaches 15 frames back and a
    frame's inverse FFT mixes all its bins, so the rounding error of a sample
    scales with the magnitudes in that window, not with the sample itself).
    C: an output sample collects about S products and S roundings in its beams
    (S <= 64), 2 log2(1024) = 20 in the inverse FFT and 16 in the FIR, so its
    error is near Gaussian with a standard deviation of at most
    sqrt(64 + 20 + 16) = 10 eps in those units; the largest of up to 1e8
    samples stays below 6.5 standard deviations, 65 eps.  C_FP32 = 128 keeps a
    factor two.  The FP16 form's weights carry 2^-22 (4 eps) from the hi/lo
    split on each of the S products: sqrt(16 * 64 + 36) = 33 eps, times 6.5 =
    213; C_FP16 = 512.  One sample off by 1e-3 sigma_y already fails both.
"""

from __future__ import annotations

import numpy as np

import oracle as O
import synth

TOL_TS_FP32 = 2e-5
TOL_TS_FP16 = 1e-4
TAU_FP32 = 1e-5
TAU_FP16 = 1e-4
EPS32 = 2.0 ** -24
C_FP32 = 128.0
C_FP16 = 512.0


REL_FP32 = C_FP32 * EPS32
REL_FP16 = C_FP16 * EPS32


def assert_samples_close(got, ref, env, sigma, rel, what="y"):
    """Per-sample bound |got - ref| <= rel * (sigma + env_local) on streams of
    whole frames (rel = C * eps, REL_FP32 or REL_FP16): got, ref, env [J, N] (or
    [N]) with N a multiple of 1024, sigma [J] (or scalar).  env_local = max of
    env over the sample's frame and the 16 frames on either side."""
    from scipy.ndimage import maximum_filter1d
    got = np.atleast_2d(np.asarray(got, dtype=np.float64))
    ref = np.atleast_2d(np.asarray(ref, dtype=np.float64))
    env = np.atleast_2d(np.asarray(env, dtype=np.float64))
    sig = np.broadcast_to(np.atleast_1d(np.asarray(sigma, dtype=np.float64)), (got.shape[0],))
    J, N = got.shape
    assert ref.shape == got.shape == env.shape and N % 1024 == 0, (got.shape, ref.shape, env.shape)
    fr = env.reshape(J, N // 1024, 1024).max(axis=2)
    loc = maximum_filter1d(fr, size=33, axis=1, mode="nearest")
    bound = rel * (sig[:, None] + np.repeat(loc, 1024, axis=1))
    err = np.abs(got - ref)
    ratio = err / bound
    worst = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    assert ratio[worst] <= 1.0, (
        f"{what}: sample {worst} off by {err[worst]:.3e} > bound {bound[worst]:.3e} "
        f"(ref {ref[worst]:.4e}, sigma {sig[worst[0]]:.4e})")
    return float(ratio[worst])


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
