"""Parity at the full sizes of the benchmarked workloads.

* Full band: 24 stations x 244 subbands x 65536 frames (int16, 20 dispersed
  pulses), one beam, FP32 form: the whole block, both polarisations, element
  by element against the oracle, plus the trigger lists.
* Precision: 48 stations x 488 subbands x 50 beams x 65536 frames (int8),
  FP16 tensor-core form in the launch configuration bench.py times: beams at
  sampled frames of sampled streams, the time series on sampled windows the
  oracle computes one by one for all 100 streams, each stream's sigma from
  the whole block, and the trigger lists on those windows.
* Stress shape: 48 stations x 488 subbands x 200 beams x 8 trials, chunked
  beam rows replayed from a captured graph, sampled windows of eight streams.
* Precision block with full-rate de-dispersion: sampled windows of six
  streams of the filtered series and their triggers.
"""

import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import (REL_FP16, REL_FP32, TAU_FP16, TAU_FP32, TOL_TS_FP32,
                        assert_samples_close, rel_rms)

pytestmark = pytest.mark.gpu


def _noise_block(w, block=0):
    x = np.empty((w.pols, w.subbands, w.block_len, w.stations, 2), dtype=w.dtype)
    for pol in range(w.pols):
        for k in range(w.subbands):
            x[pol, k] = synth.noise_slab(w.seed, block, pol, k, w.block_len, w.stations,
                                         w.noise_sigma, w.dtype)
    return x


def test_fullband_block_matches_oracle(cuda_lib):
    import torch
    w = synth.FULLBAND
    enu, dirs, tec = synth.make_geometry(w)
    x, pulses = synth.make_block(w, 0, enu, dirs)
    plan = cuda_lib.Plan(w.stations, w.pols, w.subbands, w.beams, len(tec), w.block_len,
                         input_dtype=w.dtype, precision="fp32", first_bin=w.first_bin,
                         store_timeseries=True)
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    plan.lp_process_block(torch.from_numpy(x).cuda())
    trig, n, st = plan.lp_get_triggers()
    pipe = O.Pipeline(w.stations, w.pols, w.subbands, w.beams, len(tec), w.block_len,
                      w.first_bin, enu, dirs, tec)
    ref = pipe.process_block(x)
    for p in range(w.pols):
        y = plan.lp_get_timeseries(0, 0, p)
        assert rel_rms(y, ref["y"][p]) < TOL_TS_FP32
        assert_samples_close(y, ref["y"][p], ref["env"][p], ref["sigma"][p], REL_FP32)
    np.testing.assert_allclose(plan.lp_get_sigma(), ref["sigma"], rtol=1e-5)
    got = {(int(r["stream"]), int(r["n"])) for r in trig}
    want = {(p, nn) for (nn, b, t, p, e, s) in ref["triggers"]}
    for (j, nn) in got ^ want:
        env = ref["env"][j, nn - ref["n_first"]]
        assert abs(env - ref["theta"][j]) <= TAU_FP32 * ref["theta"][j]
    # the 20 injected pulses (SNR 4..20 at TEC 5..30, one trial at 17.5 TECU)
    # produce triggers; the strongest near-trial ones must be found
    assert len(want) > 0


def _noise_level(x, wts, dd_t, g, pol, F):
    """sigma_y of every beam of one polarisation and trial from the whole block
    (the Parseval estimate of block 0): |beam|^2 summed over frames is
    w^T R w* with the station covariance R[k] = sum_m x_m x_m^H."""
    K, S = x.shape[1], x.shape[3]
    power = np.zeros(wts.shape[1])
    for k in range(K):
        xc = x[pol, k, :, :, 0].astype(np.float64) + 1j * x[pol, k, :, :, 1]
        R = xc.T @ xc.conj()                                  # [S, S]
        wk = wts[k]                                           # [B, S]
        power += np.real(np.einsum("bs,st,bt->b", wk, R, wk.conj())) * abs(dd_t[k]) ** 2
    g2 = float(np.sum(g ** 2))
    return np.sqrt(2.0 * g2 / 1024.0 ** 3 * power / F)


def _window_checks(y, x, wts_b, dd_t, pol, fb, g, windows, sigma, theta, got_n, rel, tau):
    """One stream on sampled windows against the oracle's own computation of
    each window: relative RMS, the per-sample bound and the trigger set."""
    for (m0, m1) in windows:
        u = O.stream_window(x, wts_b, dd_t, pol, fb, g, m0, m1)
        yw = y[m0 * 1024:m1 * 1024]
        assert rel_rms(yw, u.real.reshape(-1)) < 1e-5
        assert_samples_close(yw, u.real.reshape(-1), np.abs(u).reshape(-1), sigma, rel)
        env = np.abs(u).reshape(-1)
        n_first = (m0 - 15) * 1024
        n_ref, _ = O.find_triggers(env, theta, n_first)
        g_win = {nn for nn in got_n if n_first <= nn < n_first + env.size}
        for nn in g_win ^ set(n_ref.tolist()):
            assert abs(env[nn - n_first] - theta) <= tau * theta


def test_precision_block_sampled_parity(cuda_lib):
    """The benchmarked launch configuration (FP16 form, whole 65536-frame block):
    beams of three streams at sampled frames, and for every one of the 100
    streams the time series and the triggers on three sampled windows (start,
    middle, end of the block) against the oracle, with each stream's noise
    level from the whole block."""
    import torch
    w = synth.PRECISION
    enu, dirs, tec = synth.make_geometry(w)
    x = _noise_block(w)
    k_sigma = 4.5
    plan = cuda_lib.Plan(w.stations, w.pols, w.subbands, w.beams, len(tec), w.block_len,
                         input_dtype="int8", precision="fp16", first_bin=w.first_bin,
                         store_timeseries=True, k_sigma=k_sigma)
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    xd = torch.from_numpy(x).cuda()
    plan.lp_process_block(xd)
    trig, n, st = plan.lp_get_triggers()
    assert st == cuda_lib.LP_OK
    del xd
    nu = O.sky_frequencies(w.first_bin, w.subbands)
    wts = O.geometric_weights(nu, enu, dirs)
    dd = O.dedispersion_weights(nu, tec, 0.5 * (nu[0] + nu[-1]))
    g = O.synthesis_filter()
    F = w.block_len
    windows = [(0, 48), (31000, 31064), (F - 40, F)]
    for (b, pol) in [(0, 0), (23, 1), (49, 0)]:
        beams = plan.lp_get_beams(b, 0, pol)               # [K, F]
        for (m0, m1) in windows:
            xc = x[pol, :, m0:m1, :, 0].astype(np.float64) + 1j * x[pol, :, m0:m1, :, 1]
            bref = np.einsum("ks,kns->kn", wts[:, b, :], xc) * dd[:, 0][:, None]
            assert rel_rms(beams[:, m0:m1], bref) < 1e-5
    sig_gpu = plan.lp_get_sigma()
    by_stream = {}
    for r in trig:
        by_stream.setdefault(int(r["stream"]), set()).add(int(r["n"]))
    for pol in range(w.pols):
        sigma = _noise_level(x, wts, dd[:, 0], g, pol, F)   # [B]
        for b in range(w.beams):
            j = (b * len(tec)) * w.pols + pol
            assert abs(sig_gpu[j] / sigma[b] - 1) < 1e-5, (b, pol)
            y = plan.lp_get_timeseries(b, 0, pol)
            _window_checks(y, x, wts[:, b, :], dd[:, 0], pol, w.first_bin, g, windows, sigma[b],
                           k_sigma * sigma[b], by_stream.get(j, set()), REL_FP16, TAU_FP16)


def test_stress_shape_chunked_graph_sampled_parity(cuda_lib):
    """The stress configuration's shape (48 stations x 488 subbands, 200 beams x 8
    STEC trials x 2 pols = 3200 streams) in the launch configuration its bench
    uses -- chunked beam rows (here 2048 of 4096 frames) replayed from a captured
    CUDA graph -- on a seeded noise block: a replay equals the capturing run bit
    for bit, and sampled windows of eight streams (trials 0 and 7, beams at both
    ends of the grid, windows at the start, across the chunk boundary and at the
    end) match the oracle, with their triggers."""
    import torch
    w = synth.STRESS
    F, chunk, k_sigma = 4096, 2048, 5.0
    enu, dirs, tec = synth.make_geometry(w)
    x = np.empty((w.pols, w.subbands, F, w.stations, 2), dtype=w.dtype)
    for pol in range(w.pols):
        for k in range(w.subbands):
            x[pol, k] = synth.noise_slab(w.seed, 0, pol, k, F, w.stations, w.noise_sigma,
                                         w.dtype)
    stream = torch.cuda.Stream()
    plan = cuda_lib.Plan(w.stations, w.pols, w.subbands, w.beams, len(tec), F,
                         input_dtype="int8", precision="fp16", first_bin=w.first_bin,
                         chunk_frames=chunk, use_graph=True, store_timeseries=True,
                         k_sigma=k_sigma, trigger_cap=1 << 22, stream=stream)
    plan.lp_set_weights(enu, dirs, stream=stream)
    plan.lp_set_tec(tec, stream=stream)
    assert plan.lp_launches_per_block() == 2 + 3 * (F // chunk)
    xd = torch.empty(x.shape, dtype=torch.int8, device="cuda")
    with torch.cuda.stream(stream):
        xd.copy_(torch.from_numpy(x))
    picks = [(0, 0, 0), (0, 7, 1), (199, 0, 1), (199, 7, 0), (77, 3, 0), (120, 5, 1),
             (13, 7, 0), (186, 1, 1)]
    runs = []
    for rep in range(2):                     # capture + launch, then a replay
        plan.lp_reset_stream(stream=stream)
        plan.lp_process_block(xd, stream=stream)
        trig, n, st = plan.lp_get_triggers()
        assert st == cuda_lib.LP_OK
        ys = {(b, t, p): plan.lp_get_timeseries(b, t, p) for (b, t, p) in picks}
        runs.append((trig, plan.lp_get_sigma().copy(), ys))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    for key in picks:
        np.testing.assert_array_equal(runs[0][2][key], runs[1][2][key])
    trig, sig_gpu, ys = runs[1]
    del xd
    nu = O.sky_frequencies(w.first_bin, w.subbands)
    wts = O.geometric_weights(nu, enu, dirs)
    dd = O.dedispersion_weights(nu, np.asarray(tec), 0.5 * (nu[0] + nu[-1]))
    g = O.synthesis_filter()
    windows = [(0, 40), (chunk - 20, chunk + 20), (F - 40, F)]
    by_stream = {}
    for r in trig:
        by_stream.setdefault(int(r["stream"]), set()).add(int(r["n"]))
    for (b, t, pol) in picks:
        j = (b * len(tec) + t) * w.pols + pol
        sigma = _noise_level(x, wts[:, b:b + 1, :], dd[:, t], g, pol, F)[0]
        assert abs(sig_gpu[j] / sigma - 1) < 1e-5, (b, t, pol)
        _window_checks(ys[(b, t, pol)], x, wts[:, b, :], dd[:, t], pol, w.first_bin, g, windows,
                       sigma, k_sigma * sigma, by_stream.get(j, set()), REL_FP16, TAU_FP16)


def test_precision_block_fullrate_sampled_parity(cuda_lib):
    """The benchmarked block (48 x 488 x 50, 65536 frames, FP16 form) with
    full-rate de-dispersion: for six streams the filtered series and its
    triggers on sampled windows (start, middle, end) against the oracle, which
    synthesises each window's series from two frames earlier (the filter's
    2047 samples of reach) with stream_window and filters it with
    fullrate_filter; each stream's noise level from the whole block."""
    import torch
    w = synth.PRECISION
    enu, dirs, tec = synth.make_geometry(w)
    x = _noise_block(w)
    k_sigma = 4.5
    plan = cuda_lib.Plan(w.stations, w.pols, w.subbands, w.beams, len(tec), w.block_len,
                         input_dtype="int8", precision="fp16", first_bin=w.first_bin,
                         store_timeseries=True, k_sigma=k_sigma, fullrate_dedisp=True)
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    xd = torch.from_numpy(x).cuda()
    plan.lp_process_block(xd)
    trig, n, st = plan.lp_get_triggers()
    assert st == cuda_lib.LP_OK
    del xd
    nu = O.sky_frequencies(w.first_bin, w.subbands)
    nu_ref = 0.5 * (nu[0] + nu[-1])
    wts = O.geometric_weights(nu, enu, dirs)
    ones = np.ones(w.subbands, dtype=complex)                 # no per-subband phase
    g = O.synthesis_filter()
    h = O.fullrate_taps(tec, nu_ref)[0]
    F, L = w.block_len, O.FULLRATE_TAPS
    windows = [(0, 24), (40000, 40024), (F - 24, F)]
    sig_gpu = plan.lp_get_sigma()
    by_stream = {}
    for r in trig:
        by_stream.setdefault(int(r["stream"]), set()).add(int(r["n"]))
    for (b, pol) in [(0, 0), (11, 1), (24, 0), (37, 1), (48, 1), (49, 0)]:
        j = (b * len(tec)) * w.pols + pol
        sigma = _noise_level(x, wts[:, b:b + 1, :], ones, g, pol, F)[0]
        assert abs(sig_gpu[j] / sigma - 1) < 1e-5, (b, pol)
        theta = k_sigma * sigma
        y = plan.lp_get_timeseries(b, 0, pol)
        for (m0, m1) in windows:
            # the window's series and the 2047 samples before it (zero before the start)
            lo = max(0, m0 - 2)
            u = O.stream_window(x, wts[:, b, :], ones, pol, w.first_bin, g, lo, m1).reshape(-1)
            uext = (np.concatenate([np.zeros(L - 1), u]) if m0 == 0
                    else u[(m0 - lo) * 1024 - (L - 1):])
            v = O.fullrate_filter(uext, h)
            assert v.size == (m1 - m0) * 1024
            yw = y[m0 * 1024:m1 * 1024]
            assert rel_rms(yw, v.real) < 1e-5
            assert_samples_close(yw, v.real, np.abs(v), sigma, 2 * REL_FP16)
            env = np.abs(v)
            n_first = (m0 - 15) * 1024
            n_ref, _ = O.find_triggers(env, theta, n_first)
            g_win = {nn for nn in by_stream.get(j, set()) if n_first <= nn < n_first + env.size}
            for nn in g_win ^ set(n_ref.tolist()):
                assert abs(env[nn - n_first] - theta) <= TAU_FP16 * theta
