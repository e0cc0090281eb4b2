"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Element-by-element comparisons on seeded inputs at sizes the oracle finishes
in seconds (several tiles and ragged tails), plus the tiny workload with its
injected pulse in full.  Tolerances are derived in tests/gpu_common.py.
"""

import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import (REL_FP16, REL_FP32, TAU_FP16, TAU_FP32, TOL_TS_FP16, TOL_TS_FP32,
                        assert_samples_close, compare_triggers, gpu_blocks, make_plan,
                        oracle_blocks, random_case, rel_rms)

pytestmark = pytest.mark.gpu


CASES = [
    # S, P, K, B, Tr, F, first_bin, dtype, nblocks
    (2, 1, 1, 1, 1, 16, 1, "int16", 2),          # minimum sizes, bin 1 (next to DC)
    (3, 2, 5, 2, 2, 64, 220, "int8", 2),
    (6, 2, 16, 1, 1, 200, 154, "int16", 2),       # ragged frame tiles (200 = 128 + 72)
    (5, 2, 37, 3, 1, 136, 474, "int8", 1),        # band reaching bin 510
    (7, 1, 64, 5, 3, 96, 100, "int16", 3),        # 3 blocks: history and running sigma
    (48, 2, 8, 34, 1, 72, 300, "int8", 1),        # 48 stations, 34 beams (two weight chunks)
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "S%d_P%d_K%d_B%d_T%d_F%d_b%d_%s_x%d" % c)
def test_fp32_path_matches_oracle(cuda_lib, case):
    S, P, K, B, Tr, F, fb, dtype, nb = case
    blocks, enu, dirs, tec = random_case(11, S, P, K, B, Tr, F, fb, dtype, nb)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, dtype, store_timeseries=True,
                     frames_per_cta=64 if F >= 64 else 8)
    g = gpu_blocks(cuda_lib, plan, blocks, enu, dirs, tec)
    pipe, o = oracle_blocks(S, P, K, B, Tr, F, fb, blocks, enu, dirs, tec)
    for gb, ob in zip(g, o):
        # beams: oracle [J, F, K], GPU [J, K, F]
        assert rel_rms(gb["beams"], ob["beams"].transpose(0, 2, 1)) < TOL_TS_FP32
        assert rel_rms(gb["y"], ob["y"]) < TOL_TS_FP32
        assert_samples_close(gb["y"], ob["y"], ob["env"], ob["sigma"], REL_FP32)
        np.testing.assert_allclose(gb["sigma"], ob["sigma"], rtol=1e-5)
        ng, no, nd, bad = compare_triggers(gb["trig"], ob, P, Tr, TAU_FP32)
        assert not bad, bad[:5]


FP16_CASES = [
    # S, P, K, B, Tr, F, first_bin, nblocks, dtype: tensor-core beamformer
    (4, 2, 8, 3, 1, 256, 200, 2, "int8"),
    (48, 2, 12, 50, 1, 600, 100, 2, "int8"),      # 50 beams, ragged 256-frame tile
    (8, 1, 5, 70, 2, 2104, 300, 1, "int8"),       # two beam tiles, two 2048-frame chunks
    (64, 2, 3, 64, 1, 72, 12, 1, "int8"),         # 64 stations (K = 128), exactly one tile
    (12, 1, 2, 1, 3, 40, 450, 2, "int8"),         # one beam, three trials, tiny block
    (8, 2, 10, 50, 1, 600, 150, 2, "int16"),      # int16 (full range): two B images
    (36, 1, 4, 70, 2, 2104, 300, 1, "int16"),     # int16, two beam tiles, K = 72 (padded 80)
]


@pytest.mark.parametrize("case", FP16_CASES, ids=lambda c: "S%d_P%d_K%d_B%d_T%d_F%d_b%d_x%d_%s" % c)
def test_fp16_tensor_core_path_matches_oracle(cuda_lib, case):
    S, P, K, B, Tr, F, fb, nb, dtype = case
    amp = 127 if dtype == "int8" else 32767
    blocks, enu, dirs, tec = random_case(31, S, P, K, B, Tr, F, fb, dtype, nb, amp=amp)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, dtype, precision="fp16",
                     store_timeseries=True, frames_per_cta=64 if F >= 64 else 8, k_sigma=4.0)
    g = gpu_blocks(cuda_lib, plan, blocks, enu, dirs, tec)
    _, o = oracle_blocks(S, P, K, B, Tr, F, fb, blocks, enu, dirs, tec, k_sigma=4.0)
    for gb, ob in zip(g, o):
        eb = rel_rms(gb["beams"], ob["beams"].transpose(0, 2, 1))
        ey = rel_rms(gb["y"], ob["y"])
        # hi/lo FP16 weights keep the beams near FP32 accuracy
        assert eb < 1e-5, eb
        assert ey < TOL_TS_FP16 and ey < 1e-5, ey
        assert_samples_close(gb["y"], ob["y"], ob["env"], ob["sigma"], REL_FP16)
        np.testing.assert_allclose(gb["sigma"], ob["sigma"], rtol=1e-5)
        ng, no, nd, bad = compare_triggers(gb["trig"], ob, P, Tr, TAU_FP16)
        assert not bad, bad[:5]


def test_fp16_and_fp32_forms_agree(cuda_lib):
    S, P, K, B, Tr, F, fb = 16, 2, 20, 9, 2, 512, 250
    blocks, enu, dirs, tec = random_case(32, S, P, K, B, Tr, F, fb, "int8", 1, amp=100)
    ys = []
    for prec in ("fp32", "fp16"):
        plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision=prec,
                         store_timeseries=True)
        ys.append(gpu_blocks(cuda_lib, plan, blocks, enu, dirs, tec)[0]["y"])
    assert rel_rms(ys[1], ys[0]) < 2e-6


def test_many_triggers_compaction(cuda_lib):
    """Low threshold: thousands of triggers, compared one by one."""
    S, P, K, B, Tr, F, fb = 4, 2, 24, 2, 2, 128, 200
    blocks, enu, dirs, tec = random_case(5, S, P, K, B, Tr, F, fb, "int16", 2)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int16", k_sigma=2.5, store_timeseries=True,
                     frames_per_cta=32)
    g = gpu_blocks(cuda_lib, plan, blocks, enu, dirs, tec)
    _, o = oracle_blocks(S, P, K, B, Tr, F, fb, blocks, enu, dirs, tec, k_sigma=2.5)
    for gb, ob in zip(g, o):
        ng, no, nd, bad = compare_triggers(gb["trig"], ob, P, Tr, TAU_FP32)
        assert no > 1000 and not bad and nd <= 2
        # the records carry the envelope and sigma of the sample
        env = ob["env"][gb["trig"]["stream"], gb["trig"]["n"] - ob["n_first"]]
        np.testing.assert_allclose(gb["trig"]["env"], env, rtol=1e-5)
        # sorted by (beam, tec, pol, n)
        keys = list(zip(gb["trig"]["beam"], gb["trig"]["tec"], gb["trig"]["pol"], gb["trig"]["n"]))
        assert keys == sorted(keys)


def test_trigger_overflow_reports_and_keeps_first(cuda_lib):
    S, P, K, B, Tr, F, fb = 3, 1, 8, 1, 1, 64, 300
    blocks, enu, dirs, tec = random_case(6, S, P, K, B, Tr, F, fb, "int16", 1)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int16", k_sigma=1.0, trigger_cap=100)
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    import torch
    plan.lp_process_block(torch.from_numpy(blocks[0]).cuda())
    trig, n, st = plan.lp_get_triggers(cap=50)
    assert st == cuda_lib.LP_ERR_OVERFLOW and n > 100 and len(trig) == 50


def test_tiny_workload_with_pulse(cuda_lib):
    """6 stations, 16 subbands at 130 MHz, int16 sigma 8, one pulse at TEC 10, SNR 10."""
    w = synth.TINY
    enu, dirs, tec = synth.make_geometry(w)
    blocks = [synth.make_block(w, b, enu, dirs)[0] for b in range(2)]
    pulses = synth.make_block(w, 0, enu, dirs)[1]
    plan = make_plan(cuda_lib, w.stations, w.pols, w.subbands, w.beams, len(w.tec_trials),
                     w.block_len, w.first_bin, w.dtype, store_timeseries=True)
    g = gpu_blocks(cuda_lib, plan, blocks, enu, dirs, tec)
    _, o = oracle_blocks(w.stations, w.pols, w.subbands, w.beams, len(w.tec_trials),
                         w.block_len, w.first_bin, blocks, enu, dirs, tec)
    for gb, ob in zip(g, o):
        assert rel_rms(gb["y"], ob["y"]) < TOL_TS_FP32
        assert_samples_close(gb["y"], ob["y"], ob["env"], ob["sigma"], REL_FP32)
        ng, no, nd, bad = compare_triggers(gb["trig"], ob, w.pols, 1, TAU_FP32)
        assert not bad
    # the injected pulse triggers near its de-dispersed arrival time
    nu = O.sky_frequencies(w.first_bin, w.subbands)
    nu_ref = 0.5 * (nu[0] + nu[-1])
    t_exp = pulses[0].n0 + O.dispersion_coefficient_hz(w.tec_trials[0]) / nu_ref ** 2 * O.FS_HZ
    ns = g[0]["trig"]["n"]
    assert len(ns) > 0 and np.min(np.abs(ns - t_exp)) < 200


@pytest.mark.parametrize("precision,pinned", [("fp32", False), ("fp16", True), ("fp32", True)])
def test_host_input_equals_device_input(cuda_lib, precision, pinned):
    """A host block (copied one polarisation at a time, the copy of pol 1
    overlapping the work on pol 0) gives exactly the device block's results:
    every stream's time series, the noise levels and the triggers of every
    block, over several blocks (history and running sigma carried)."""
    S, P, K, B, Tr, F, fb = 8, 2, 12, 2, 2, 96, 250
    blocks, enu, dirs, tec = random_case(8, S, P, K, B, Tr, F, fb, "int8", 3)
    import torch
    res = []
    for host in (False, True):
        plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision=precision,
                         store_timeseries=True, host_input=True, k_sigma=3.0)
        plan.lp_set_weights(enu, dirs)
        plan.lp_set_tec(tec)
        out = []
        for xb in blocks:
            if host:
                x = torch.from_numpy(xb).pin_memory() if pinned else xb
            else:
                x = torch.from_numpy(xb).cuda()
            plan.lp_process_block(x)
            ys = [plan.lp_get_timeseries(b, t, pol)
                  for b in range(B) for t in range(Tr) for pol in range(P)]
            out.append((np.stack(ys), plan.lp_get_sigma().copy(), plan.lp_get_triggers()[0]))
        res.append(out)
    for (ya, sa, ta), (yb, sb, tb) in zip(*res):
        np.testing.assert_array_equal(ya, yb)
        np.testing.assert_array_equal(sa, sb)
        np.testing.assert_array_equal(ta, tb)


def test_deterministic_reruns(cuda_lib):
    S, P, K, B, Tr, F, fb = 8, 2, 40, 3, 2, 256, 120
    blocks, enu, dirs, tec = random_case(9, S, P, K, B, Tr, F, fb, "int8", 1)
    outs = []
    for _ in range(2):
        plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", store_timeseries=True,
                         k_sigma=3.0)
        outs.append(gpu_blocks(cuda_lib, plan, blocks, enu, dirs, tec)[0])
    np.testing.assert_array_equal(outs[0]["y"], outs[1]["y"])
    np.testing.assert_array_equal(outs[0]["sigma"], outs[1]["sigma"])
    np.testing.assert_array_equal(outs[0]["trig"], outs[1]["trig"])


def test_reset_stream_restarts_history(cuda_lib):
    S, P, K, B, Tr, F, fb = 3, 1, 6, 1, 1, 64, 330
    blocks, enu, dirs, tec = random_case(12, S, P, K, B, Tr, F, fb, "int16", 2)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int16", store_timeseries=True)
    a = gpu_blocks(cuda_lib, plan, blocks[:1], enu, dirs, tec)[0]["y"]
    gpu_blocks(cuda_lib, plan, blocks[1:], enu, dirs, tec)
    plan.lp_reset_stream()
    b = gpu_blocks(cuda_lib, plan, blocks[:1], enu, dirs, tec)[0]["y"]
    np.testing.assert_array_equal(a, b)


def test_bad_arguments_on_device(cuda_lib):
    import torch
    S, P, K, B, Tr, F, fb = 3, 1, 6, 2, 1, 64, 330
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int16")
    x = torch.zeros((P, K, F, S, 2), dtype=torch.int16, device="cuda")
    with pytest.raises(cuda_lib.LPError):          # weights not set yet
        plan.lp_process_block(x)
    with pytest.raises(cuda_lib.LPError):          # not unit vectors
        plan.lp_set_weights(np.zeros((S, 3)), np.ones((B, 3)))
    plan.lp_set_weights(np.zeros((S, 3)), synth.hex_beam_directions(2))
    plan.lp_set_tec([5.0])
    with pytest.raises(cuda_lib.LPError):          # host pointer without host_input
        plan.lp_process_block(np.zeros((P, K, F, S, 2), dtype=np.int16))
    plan.lp_process_block(x)
    trig, n, st = plan.lp_get_triggers()
    assert n == 0 and st == cuda_lib.LP_OK


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_balanced_tiling_equals_fixed_runs(cuda_lib, precision):
    """The balanced synthesis tiling (one block per SM walking an equal range of
    the streams' frames; here 10 streams x 1000 frames in ranges of 72 frames,
    so ranges cross stream boundaries) gives the time series, noise levels and
    triggers of fixed 64-frame runs bit for bit, over two blocks."""
    import torch
    S, P, K, B, Tr, F, fb = 8, 2, 20, 5, 1, 1000, 140
    blocks, enu, dirs, tec = random_case(71, S, P, K, B, Tr, F, fb, "int8", 2, amp=60)
    plans = [make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision=precision,
                       store_timeseries=True, k_sigma=3.5, frames_per_cta=fpc)
             for fpc in (0, 64)]
    for p in plans:
        p.lp_set_weights(enu, dirs)
        p.lp_set_tec(tec)
    for xb in blocks:
        xd = torch.from_numpy(xb).cuda()
        res = []
        for p in plans:
            p.lp_process_block(xd)
            ys = np.stack([p.lp_get_timeseries(b, 0, pol) for b in range(B) for pol in range(P)])
            res.append((ys, p.lp_get_sigma().copy(), p.lp_get_triggers()[0]))
        (ya, sa, ta), (yb, sb, tb) = res
        np.testing.assert_array_equal(ya, yb)
        np.testing.assert_array_equal(sa, sb)
        np.testing.assert_array_equal(ta, tb)
        assert len(ta) > 0
