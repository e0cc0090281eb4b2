"""The no-allocation entry point, lp_process_block_noalloc.

It serves callers that cannot call cudaMalloc -- a host process that forbids
device allocation once it runs, or a plug-in whose framework owns the device
heap and hands it only the buffers it planned -- so they cannot bind a plan
workspace: its scratch is a static device array inside the library.

The tests call it through the C ABI and check:
  * two calls in a row on different blocks, each against the FP64 oracle
    (time series, noise level, the unsorted trigger set) and against the plan
    path (lp_process_block with a bound workspace);
  * a larger shape followed by a smaller one (the second call must not see the
    first one's scratch), once with the optional sigma2 and trigger_count
    outputs left NULL;
  * the refusals of arguments that are not device memory of the current device
    or not aligned, and of shapes too large for the static scratch, none of
    which launches anything.
The file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""

import ctypes

import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import (REL_FP32, TAU_FP32, TOL_TS_FP32, assert_samples_close, compare_triggers,
                        random_case, rel_rms)

pytestmark = pytest.mark.gpu

TRIG_BYTES = 32


def _plan_path(lp, x, shape, fb, enu, dirs, tec, k_sigma):
    import torch
    S, P, K, B, Tr, F = shape
    plan = lp.Plan(S, P, K, B, Tr, F, input_dtype="int16", precision="fp32", first_bin=fb,
                   store_timeseries=True, k_sigma=k_sigma)
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    plan.lp_process_block(torch.from_numpy(x).cuda())
    y = np.stack([plan.lp_get_timeseries(b, t, p) for b in range(B) for t in range(Tr)
                  for p in range(P)])
    sig = plan.lp_get_sigma()
    trig, n, _ = plan.lp_get_triggers()
    plan.close()
    return y, sig, {(int(r["stream"]), int(r["n"])) for r in trig}


def _config(lp, fb, k_sigma):
    cfg = lp.config_default()
    cfg.input_dtype = lp.LP_INPUT_INT16
    cfg.first_bin = fb
    cfg.k_sigma = k_sigma
    return cfg


def _call(lp, shape, cfg, enu, dirs, tec, x_ptr, y_ptr, s2_ptr, trig_ptr, cap, cnt_ptr):
    import torch
    S, P, K, B, Tr, F = shape
    enu = np.ascontiguousarray(enu, dtype=np.float64)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64)
    tec = np.ascontiguousarray(tec, dtype=np.float64)
    err = ctypes.create_string_buffer(256)
    st = lp._lib.lp_process_block_noalloc(
        S, P, K, B, Tr, F, ctypes.byref(cfg), enu.ctypes.data, dirs.ctypes.data,
        tec.ctypes.data, x_ptr, y_ptr, s2_ptr, trig_ptr, cap, cnt_ptr,
        torch.cuda.current_stream().cuda_stream, err, 256)
    return st, err.value


def _noalloc(lp, x, shape, fb, enu, dirs, tec, k_sigma, cap=8192, outputs=True):
    """One call; returns y [J, F*M], sigma [J] (None without the output), the
    trigger set {(stream, n)} read from the device records."""
    import torch
    S, P, K, B, Tr, F = shape
    J = B * Tr * P
    xd = torch.from_numpy(x).cuda()
    y = torch.empty((J, F * 1024), dtype=torch.float32, device="cuda")
    s2 = torch.empty(J, dtype=torch.float64, device="cuda") if outputs else None
    # records pre-filled with n = -1: without a counter, the written ones are
    # those with n >= 0 (a first block never emits n < 0)
    trig = torch.full((cap * TRIG_BYTES,), 0xFF, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda") if outputs else None
    st, msg = _call(lp, shape, _config(lp, fb, k_sigma), enu, dirs, tec, xd.data_ptr(),
                    y.data_ptr(), s2.data_ptr() if outputs else None, trig.data_ptr(), cap,
                    cnt.data_ptr() if outputs else None)
    assert st == lp.LP_OK, msg
    torch.cuda.synchronize()
    recs = np.frombuffer(trig.cpu().numpy().tobytes(), dtype=lp.TRIGGER_DTYPE)
    written = recs[recs["n"] >= 0]
    if outputs:
        assert int(cnt.item()) <= cap, "the case must keep every trigger"
        assert int(cnt.item()) == len(written)
    trig_set = {(int(r["stream"]), int(r["n"])) for r in written}
    sig = np.sqrt(s2.cpu().numpy()) if outputs else None
    return y.cpu().numpy(), sig, trig_set, written


def _check_against_oracle(y, sig, written, x, shape, fb, enu, dirs, tec, k_sigma):
    S, P, K, B, Tr, F = shape
    ref = O.Pipeline(S, P, K, B, Tr, F, fb, enu, dirs, np.asarray(tec),
                     k_sigma=k_sigma).process_block(x)
    assert rel_rms(y, ref["y"]) < TOL_TS_FP32
    assert_samples_close(y, ref["y"], ref["env"], ref["sigma"], REL_FP32)
    if sig is not None:
        np.testing.assert_allclose(sig, ref["sigma"], rtol=1e-5)
    ng, no, nd, bad = compare_triggers(written, ref, P, Tr, TAU_FP32)
    assert not bad, bad[:5]
    return no


def test_noalloc_matches_oracle_and_plan_path_twice(cuda_lib):
    lp = cuda_lib
    shape = (6, 2, 16, 2, 2, 512)
    fb = 154
    k_sigma = 4.0
    blocks_a, enu, dirs, tec = random_case(21, *shape, fb, "int16", 1)
    blocks_b, _, _, _ = random_case(22, *shape, fb, "int16", 1)
    for x in (blocks_a[0], blocks_b[0]):         # two calls in a row, different data
        y, s, t_set, written = _noalloc(lp, x, shape, fb, enu, dirs, tec, k_sigma)
        assert _check_against_oracle(y, s, written, x, shape, fb, enu, dirs, tec, k_sigma) > 0
        y_ref, s_ref, t_ref = _plan_path(lp, x, shape, fb, enu, dirs, tec, k_sigma)
        assert rel_rms(y, y_ref) < TOL_TS_FP32
        np.testing.assert_allclose(s, s_ref, rtol=1e-6)
        assert t_set == t_ref


def test_noalloc_larger_then_smaller_shape_and_null_outputs(cuda_lib):
    """Four beams, then one beam with fewer frames: the second call's beam rows,
    noise partials and counters must not carry the first call's.  The second
    call leaves sigma2 and trigger_count NULL (they then live in the scratch)."""
    lp = cuda_lib
    fb, k_sigma = 200, 4.0
    big = (5, 2, 24, 4, 2, 768)
    small = (5, 1, 24, 1, 1, 256)
    xb, enu, dirs4, tec2 = random_case(41, *big, fb, "int16", 1)
    xs, _, _, _ = random_case(42, *small, fb, "int16", 1)
    dirs1 = dirs4[:1]
    tec1 = tec2[:1]
    for (shape, x, dirs, tec, outputs) in ((big, xb[0], dirs4, tec2, True),
                                           (small, xs[0], dirs1, tec1, False),
                                           (small, xs[0], dirs1, tec1, True)):
        y, s, t_set, written = _noalloc(lp, x, shape, fb, enu, dirs, tec, k_sigma,
                                        outputs=outputs)
        assert _check_against_oracle(y, s, written, x, shape, fb, enu, dirs, tec, k_sigma) > 0
        y_ref, s_ref, t_ref = _plan_path(lp, x, shape, fb, enu, dirs, tec, k_sigma)
        assert rel_rms(y, y_ref) < TOL_TS_FP32
        assert t_set == t_ref


def test_noalloc_refuses_bad_pointers_without_launching(cuda_lib):
    import torch
    lp = cuda_lib
    shape = (4, 1, 8, 1, 1, 64)
    S, P, K, B, Tr, F = shape
    fb = 300
    cfg = _config(lp, fb, 3.0)
    blocks, enu, dirs, tec = random_case(43, *shape, fb, "int16", 1)
    xd = torch.from_numpy(blocks[0]).cuda()
    y = torch.empty((1, F * 1024), dtype=torch.float32, device="cuda")
    trig = torch.empty(64 * TRIG_BYTES, dtype=torch.uint8, device="cuda")
    host_y = np.zeros(F * 1024, dtype=np.float32)
    pinned = torch.empty(F * 1024, dtype=torch.float32, pin_memory=True)
    cases = [
        ("y in pageable host memory", dict(y_ptr=host_y.ctypes.data)),
        ("y in pinned host memory", dict(y_ptr=pinned.data_ptr())),
        ("x not aligned to a complex int16 sample", dict(x_ptr=xd.data_ptr() + 2)),
        ("y not aligned", dict(y_ptr=y.data_ptr() + 2)),
        ("triggers not aligned", dict(trig_ptr=trig.data_ptr() + 4)),
        ("triggers in host memory", dict(trig_ptr=host_y.ctypes.data)),
    ]
    for what, override in cases:
        args = dict(x_ptr=xd.data_ptr(), y_ptr=y.data_ptr(), s2_ptr=None,
                    trig_ptr=trig.data_ptr(), cap=64, cnt_ptr=None)
        args.update(override)
        y.fill_(-7.0)
        torch.cuda.synchronize()
        st, msg = _call(lp, shape, cfg, enu, dirs, tec, **args)
        assert st == lp.LP_ERR_ARG, (what, st, msg)
        assert msg, what
        torch.cuda.synchronize()
        assert bool((y == -7.0).all()), what             # nothing ran


def test_noalloc_refuses_shapes_beyond_its_scratch(cuda_lib):
    lp = cuda_lib
    w = synth.PRECISION
    cfg = lp.config_default()
    cfg.first_bin = w.first_bin
    err = ctypes.create_string_buffer(256)
    dummy = np.zeros(3 * w.beams, dtype=np.float64)
    dummy[2::3] = 1.0                               # unit vectors
    st = lp._lib.lp_process_block_noalloc(
        w.stations, w.pols, w.subbands, w.beams, 1, w.block_len, ctypes.byref(cfg),
        dummy.ctypes.data, dummy.ctypes.data, dummy.ctypes.data, 16, 16, None, None, 0, None,
        None, err, 256)
    assert st == lp.LP_ERR_ARG
    assert b"static buffer" in err.value
