"""Fine-resolution (channel-domain) de-dispersion on the GPU against the FP64
oracle, and its equality across the host-input and captured-graph paths.

The time series with the filter on is compared with the oracle's Pipeline
run with ``fine_dedispersion=True`` (same tolerances as the plain path: the
filter adds 17 FP32 complex products per bin-frame); the beams read back are
the rows before the filter and are not compared here.
"""

import numpy as np
import pytest

import oracle as O
from gpu_common import (REL_FP16, REL_FP32, TAU_FP16, TAU_FP32, TOL_TS_FP16, TOL_TS_FP32,
                        assert_samples_close, compare_triggers, gpu_blocks, make_plan,
                        random_case, rel_rms)

pytestmark = pytest.mark.gpu

FINE_CASES = [
    # S, P, K, B, Tr, F, first_bin, dtype, precision, nblocks
    (6, 2, 24, 2, 2, 1544, 12, "int16", "fp32", 2),    # two filter tiles, the second ragged
    (8, 2, 40, 3, 2, 256, 150, "int8", "fp16", 3),     # three blocks: filter history carried
    (3, 1, 7, 1, 3, 16, 480, "int16", "fp32", 2),      # shortest block (16 frames)
]


@pytest.mark.parametrize("case", FINE_CASES,
                         ids=lambda c: "S%d_P%d_K%d_B%d_T%d_F%d_b%d_%s_%s_x%d" % c)
def test_fine_dedispersion_matches_oracle(cuda_lib, case):
    S, P, K, B, Tr, F, fb, dtype, prec, nb = case
    blocks, enu, dirs, tec = random_case(31, S, P, K, B, Tr, F, fb, dtype, nb)
    tec = np.linspace(6.0, 38.0, Tr)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, dtype, precision=prec,
                     store_timeseries=True, k_sigma=3.5, fine_dedisp=True)
    assert plan.lp_launches_per_block() == 5
    g = gpu_blocks(cuda_lib, plan, blocks, enu, dirs, tec)
    pipe = O.Pipeline(S, P, K, B, Tr, F, fb, enu, dirs, tec, k_sigma=3.5,
                      fine_dedispersion=True)
    tol, tau = (TOL_TS_FP16, TAU_FP16) if prec == "fp16" else (TOL_TS_FP32, TAU_FP32)
    # the filter adds 17 complex products per bin-frame: sqrt(17) of the bound's
    # 10-eps budget more, inside its factor of two
    rel = REL_FP16 if prec == "fp16" else REL_FP32
    n_oracle = 0
    for gb, xb in zip(g, blocks):
        ob = pipe.process_block(xb)
        assert rel_rms(gb["y"], ob["y"]) < tol
        assert_samples_close(gb["y"], ob["y"], ob["env"], ob["sigma"], rel)
        np.testing.assert_allclose(gb["sigma"], ob["sigma"], rtol=1e-5)
        ng, no, nd, bad = compare_triggers(gb["trig"], ob, P, Tr, tau)
        assert not bad, bad[:5]
        n_oracle += no
    # (a 16-frame first block emits one frame, which the 8-frame delay leaves empty)
    assert n_oracle > 0


def test_fine_host_input_and_graph_equal_device_input(cuda_lib):
    """The filter launched per polarisation (host blocks) and replayed from a
    captured graph gives the device block's results bit for bit."""
    import torch
    S, P, K, B, Tr, F, fb = 8, 2, 12, 2, 2, 96, 250
    blocks, enu, dirs, tec = random_case(32, S, P, K, B, Tr, F, fb, "int8", 3)
    res = []
    for mode in ("device", "host", "graph"):
        stream = torch.cuda.Stream()
        plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision="fp16",
                         store_timeseries=True, host_input=mode == "host", k_sigma=3.0,
                         fine_dedisp=True, use_graph=mode == "graph", stream=stream)
        plan.lp_set_weights(enu, dirs, stream=stream)
        plan.lp_set_tec(tec, stream=stream)
        xd = torch.empty((P, K, F, S, 2), dtype=torch.int8, device="cuda")
        out = []
        for xb in blocks:
            if mode == "host":
                plan.lp_process_block(torch.from_numpy(xb).pin_memory(), stream=stream)
            else:
                with torch.cuda.stream(stream):
                    xd.copy_(torch.from_numpy(xb))
                plan.lp_process_block(xd, stream=stream)
            ys = [plan.lp_get_timeseries(b, t, pol)
                  for b in range(B) for t in range(Tr) for pol in range(P)]
            out.append((np.stack(ys), plan.lp_get_sigma().copy(), plan.lp_get_triggers()[0]))
        res.append(out)
    for other in res[1:]:
        for (ya, sa, ta), (yb, sb, tb) in zip(res[0], other):
            np.testing.assert_array_equal(ya, yb)
            np.testing.assert_array_equal(sa, sb)
            np.testing.assert_array_equal(ta, tb)


def test_fine_dedispersion_limits(cuda_lib):
    S, P, K, B, Tr, F, fb = 4, 1, 488, 1, 1, 64, 12
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", fine_dedisp=True)
    with pytest.raises(cuda_lib.LPError):
        plan.lp_set_tec(np.array([400.0]))            # subband delays beyond 4 frames
    plan.lp_set_tec(np.array([40.0]))
    with pytest.raises(cuda_lib.LPError):
        make_plan(cuda_lib, 8, 1, 4, 1, 1, 4096, 100, "int8", precision="fp16",
                  chunk_frames=2048, fine_dedisp=True)
