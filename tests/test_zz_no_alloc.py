"""The no-allocation entry point, lp_process_block_noalloc.

It serves callers that cannot call cudaMalloc (a host that owns the device
heap, or code that must not allocate once running or while capturing a
stream): its scratch is a static device array inside the library.  This test
calls it through the C ABI twice in a row on different blocks and checks each
result against the ordinary plan path (lp_process_block with a bound
workspace) within the FP32 tolerance of the parity tests, and that a shape too
large for the static scratch is refused.  The file is collected last so that a
run stopping at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

import synth
from gpu_common import TOL_TS_FP32, random_case, rel_rms

pytestmark = pytest.mark.gpu


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
    _, n, _ = plan.lp_get_triggers()
    plan.close()
    return y, sig, n


def _noalloc(lp, x, shape, fb, enu, dirs, tec, k_sigma, cap=4096):
    import torch
    S, P, K, B, Tr, F = shape
    J = B * Tr * P
    cfg = lp.config_default()
    cfg.input_dtype = lp.LP_INPUT_INT16
    cfg.first_bin = fb
    cfg.k_sigma = k_sigma
    xd = torch.from_numpy(x).cuda()
    y = torch.empty((J, F * 1024), dtype=torch.float32, device="cuda")
    s2 = torch.empty(J, dtype=torch.float64, device="cuda")
    trig = torch.empty(cap * 32, dtype=torch.uint8, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    enu = np.ascontiguousarray(enu, dtype=np.float64)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64)
    tec = np.ascontiguousarray(tec, dtype=np.float64)
    err = ctypes.create_string_buffer(256)
    st = lp._lib.lp_process_block_noalloc(
        S, P, K, B, Tr, F, ctypes.byref(cfg), enu.ctypes.data, dirs.ctypes.data,
        tec.ctypes.data, xd.data_ptr(), y.data_ptr(), s2.data_ptr(), trig.data_ptr(), cap,
        cnt.data_ptr(), torch.cuda.current_stream().cuda_stream, err, 256)
    assert st == lp.LP_OK, err.value
    torch.cuda.synchronize()
    return y.cpu().numpy(), np.sqrt(s2.cpu().numpy()), int(cnt.item())


def test_noalloc_matches_plan_path_twice(cuda_lib):
    lp = cuda_lib
    shape = (6, 2, 16, 2, 2, 512)
    fb = 154
    k_sigma = 3.0
    blocks_a, enu, dirs, tec = random_case(21, *shape, fb, "int16", 1)
    blocks_b, _, _, _ = random_case(22, *shape, fb, "int16", 1)
    for x in (blocks_a[0], blocks_b[0]):         # two calls in a row, different data
        y_ref, s_ref, n_ref = _plan_path(lp, x, shape, fb, enu, dirs, tec, k_sigma)
        y, s, n = _noalloc(lp, x, shape, fb, enu, dirs, tec, k_sigma)
        assert rel_rms(y, y_ref) < TOL_TS_FP32
        np.testing.assert_allclose(s, s_ref, rtol=1e-6)
        assert n == n_ref and n > 0


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
