"""Full-rate de-dispersion on the GPU (Sec. 3, third paragraph, at full
resolution) against the FP64 oracle's streaming filter, and its equality
across the host-input and captured-graph paths.

The time series and triggers of the filtered series are compared with the
oracle's Pipeline run with ``fullrate_dedispersion=True``.  Tolerance of the
per-sample bound (see gpu_common): a filtered sample mixes 2048 synthesised
samples with taps of unit total power, so their errors (10 eps of the local
magnitude, near Gaussian) carry over at the same size; the two 8192-point
transforms add 2 log2(8192) = 26 roundings of the segment's magnitudes and the
FP32 spectrum of the taps one more: sqrt(100 + 26 + 1) = 11.3 eps, times 6.5
for the largest of 1e8 samples = 73 eps.  C = 256 keeps a factor three; the
relative RMS tolerances are the plain path's.
"""

import numpy as np
import pytest

import oracle as O
from gpu_common import (EPS32, TAU_FP16, TAU_FP32, TOL_TS_FP16, TOL_TS_FP32,
                        assert_samples_close, compare_triggers, gpu_blocks, make_plan,
                        random_case, rel_rms)

pytestmark = pytest.mark.gpu

REL_FULLRATE = 256.0 * EPS32
REL_FULLRATE_FP16 = 1024.0 * EPS32     # the FP16 form's 33 eps in place of 10, same margin

FULLRATE_CASES = [
    # S, P, K, B, Tr, F, first_bin, dtype, precision, nblocks, tec
    (6, 2, 24, 2, 2, 40, 12, "int16", "fp32", 3, (10.0, 40.0)),   # ragged last segment
    (8, 2, 40, 3, 1, 24, 150, "int8", "fp16", 2, (25.0,)),        # segments fill the block
    (4, 1, 300, 1, 1, 16, 100, "int8", "fp16", 3, (33.0,)),       # shortest block, wide band
]


@pytest.mark.parametrize("case", FULLRATE_CASES,
                         ids=lambda c: "S%d_P%d_K%d_B%d_T%d_F%d_b%d_%s_%s_x%d" % c[:10])
def test_fullrate_dedispersion_matches_oracle(cuda_lib, case):
    S, P, K, B, Tr, F, fb, dtype, prec, nb, tec = case
    blocks, enu, dirs, _ = random_case(41, S, P, K, B, Tr, F, fb, dtype, nb)
    tec = np.asarray(tec)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, dtype, precision=prec,
                     store_timeseries=True, k_sigma=3.5, fullrate_dedisp=True)
    assert plan.lp_launches_per_block() == 6
    g = gpu_blocks(cuda_lib, plan, blocks, enu, dirs, tec)
    pipe = O.Pipeline(S, P, K, B, Tr, F, fb, enu, dirs, tec, k_sigma=3.5,
                      fullrate_dedispersion=True)
    tol, tau = (TOL_TS_FP16, TAU_FP16) if prec == "fp16" else (TOL_TS_FP32, TAU_FP32)
    rel = REL_FULLRATE_FP16 if prec == "fp16" else REL_FULLRATE
    n_oracle = 0
    for gb, xb in zip(g, blocks):
        ob = pipe.process_block(xb)
        assert rel_rms(gb["y"], ob["y"]) < tol
        assert_samples_close(gb["y"], ob["y"], ob["env"], ob["sigma"], rel)
        np.testing.assert_allclose(gb["sigma"], ob["sigma"], rtol=1e-5)
        ng, no, nd, bad = compare_triggers(gb["trig"], ob, P, Tr, tau)
        assert not bad, bad[:5]
        assert gb["status"] == 0
        n_oracle += no
    assert n_oracle > 0


def test_fullrate_at_zero_tec_is_the_plain_path_delayed(cuda_lib):
    """STEC 0: the taps are the unit impulse at 1024 samples, so the filtered
    series is the plain path's one frame later (up to the transforms'
    rounding), over two blocks with the history carried."""
    S, P, K, B, Tr, F, fb = 8, 1, 30, 2, 1, 32, 200
    blocks, enu, dirs, _ = random_case(42, S, P, K, B, Tr, F, fb, "int8", 2)
    tec = np.array([0.0])
    full = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision="fp16",
                     store_timeseries=True, fullrate_dedisp=True)
    plain = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision="fp16",
                      store_timeseries=True)
    gf = gpu_blocks(cuda_lib, full, blocks, enu, dirs, tec)
    gp = gpu_blocks(cuda_lib, plain, blocks, enu, dirs, tec)
    yf = np.concatenate([o["y"] for o in gf], axis=1)
    yp = np.concatenate([o["y"] for o in gp], axis=1)
    d = O.FULLRATE_DELAY
    assert rel_rms(yf[:, d:], yp[:, :-d]) < 2e-6
    assert np.abs(yf[:, :d]).max() <= 1e-5 * np.abs(yp).max()
    for a, b in zip(gf, gp):
        np.testing.assert_array_equal(a["sigma"], b["sigma"])


def test_fullrate_host_input_and_graph_equal_device_input(cuda_lib):
    """The full-rate plan fed from pinned host blocks and replayed from a
    captured graph gives the device block's results bit for bit."""
    import torch
    S, P, K, B, Tr, F, fb = 8, 2, 12, 2, 2, 48, 250
    blocks, enu, dirs, _ = random_case(43, S, P, K, B, Tr, F, fb, "int8", 3)
    tec = np.array([12.0, 31.0])
    res = []
    for mode in ("device", "host", "graph"):
        stream = torch.cuda.Stream()
        plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision="fp16",
                         store_timeseries=True, host_input=mode == "host", k_sigma=3.0,
                         fullrate_dedisp=True, use_graph=mode == "graph", stream=stream)
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


def test_fullrate_limits(cuda_lib):
    S, P, K, B, Tr, F, fb = 4, 1, 488, 1, 1, 64, 12
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", fullrate_dedisp=True)
    with pytest.raises(cuda_lib.LPError):
        plan.lp_set_tec(np.array([80.0]))           # group delay beyond 768 samples
    plan.lp_set_tec(np.array([40.0]))
    for kw in ({"fine_dedisp": True}, {"stream_blocks": True, "host_input": True}):
        with pytest.raises(cuda_lib.LPError):
            make_plan(cuda_lib, 8, 1, 4, 1, 1, 4096, 100, "int8", fullrate_dedisp=True, **kw)
    with pytest.raises(cuda_lib.LPError):
        make_plan(cuda_lib, 8, 1, 4, 1, 1, 4096, 100, "int8", precision="fp16",
                  chunk_frames=2048, fullrate_dedisp=True)


def test_lsmr_then_fullrate_matches_oracle(cuda_lib):
    """The paper's order: the LSMR inversion, then the full-rate filter of the
    recovered series (both histories carried over two blocks), then the LSMR
    path's per-phase noise level (running) and trigger on the filtered series,
    against the oracle composing lsmr_invert, fullrate_filter,
    lsmr_noise_power and update_sigma2.  Tolerances: the LSMR path's own
    (1e-5, its iterate's FP32 error dominating the filter's), per-sample
    factor 8 as there."""
    import torch
    S, P, K, B, Tr, F, fb, ks = 8, 1, 12, 2, 1, 512, 200, 3.5
    blocks, enu, dirs, _ = random_case(55, S, P, K, B, Tr, F, fb, "int8", 2, amp=60)
    tec = np.array([30.0])
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", inversion="lsmr",
                     fullrate_dedisp=True, k_sigma=ks)
    assert plan.lp_launches_per_block() == 8
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    nu = O.sky_frequencies(fb, K)
    nu_ref = 0.5 * (nu[0] + nu[-1])
    w = O.geometric_weights(nu, enu, dirs)
    taps = O.fullrate_taps(tec, nu_ref)
    h = O.prototype_filter()
    J = B * Tr * P
    lsmr_hist = np.zeros((J, O.LSMR_OVERLAP, K), dtype=complex)
    fr_hist = np.zeros((J, O.FULLRATE_TAPS - 1), dtype=complex)
    s2 = None
    tol = 1e-5
    n_oracle = 0
    for bi, xb in enumerate(blocks):
        plan.lp_process_block(torch.from_numpy(xb).cuda())
        bm = O.beamform(xb[..., 0].astype(np.float64) + 1j * xb[..., 1], w, np.ones((K, Tr)))
        vs = np.zeros((J, F, O.M), dtype=complex)
        for b in range(B):
            j = b * Tr * P
            lext = np.concatenate([lsmr_hist[j], bm[b, 0, 0].T])
            x = O.lsmr_invert(lext, fb, h).reshape(-1)
            lsmr_hist[j] = lext[-O.LSMR_OVERLAP:]
            uext = np.concatenate([fr_hist[j], x])
            vs[j] = O.fullrate_filter(uext, taps[0]).reshape(F, O.M)
            fr_hist[j] = uext[-(O.FULLRATE_TAPS - 1):]
        pw = np.stack([O.lsmr_noise_power(vs[j]) for j in range(J)])
        s2 = O.update_sigma2(s2, pw, 0.25, bi == 0)
        sig = np.sqrt(s2)
        got = np.stack([plan.lp_get_timeseries(b, 0, 0) for b in range(B)])
        want = vs.real.reshape(J, -1)
        assert rel_rms(got, want) < tol
        assert_samples_close(got, want, np.abs(vs).reshape(J, -1),
                             np.sqrt(np.mean(sig ** 2, axis=1)), 8 * tol)
        np.testing.assert_allclose(plan.lp_get_lsmr_sigma(), sig, rtol=10 * tol)
        n = ((bi * F + np.arange(F) - O.LSMR_OVERLAP)[:, None] * O.M + np.arange(O.M)[None, :])
        want_trig = set()
        for j in range(J):
            hit = (np.abs(vs[j]) > ks * sig[j][None, :]) & (n >= 0)
            want_trig |= {(j, int(v)) for v in n[hit]}
        g_trig, _, st = plan.lp_get_triggers()
        assert st == 0
        got_trig = {(int(r["stream"]), int(r["n"])) for r in g_trig}
        first = int(n[0, 0])
        for (j, nn) in got_trig ^ want_trig:
            i, p = divmod(nn - first, O.M)
            th = ks * sig[j, p]
            assert abs(abs(vs[j, i, p]) - th) <= 10 * tol * th, (j, nn)
        n_oracle += len(want_trig)
    assert n_oracle > 0


def test_lsmr_then_fullrate_host_input_and_graph_equal_device_input(cuda_lib):
    """The paper's chain (LSMR, then the full-rate filter, whose series rows
    k_lsmr writes directly) fed from pinned host blocks and replayed from a
    captured graph gives the device block's results bit for bit, over two
    blocks and two trials."""
    import torch
    S, P, K, B, Tr, F, fb = 8, 2, 12, 1, 2, 256, 200
    blocks, enu, dirs, _ = random_case(44, S, P, K, B, Tr, F, fb, "int8", 2, amp=60)
    tec = np.array([12.0, 31.0])
    res = []
    for mode in ("device", "host", "graph"):
        stream = torch.cuda.Stream()
        plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision="fp16",
                         inversion="lsmr", host_input=mode == "host", k_sigma=3.0,
                         fullrate_dedisp=True, use_graph=mode == "graph", stream=stream)
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
            out.append((np.stack(ys), plan.lp_get_lsmr_sigma().copy(), plan.lp_get_triggers()[0]))
        res.append(out)
    assert any(len(t) for _, _, t in res[0])
    for other in res[1:]:
        for (ya, sa, ta), (yb, sb, tb) in zip(res[0], other):
            np.testing.assert_array_equal(ya, yb)
            np.testing.assert_array_equal(sa, sb)
            np.testing.assert_array_equal(ta, tb)
