"""PPF inversion by windowed LSMR on the GPU against the FP64 oracle.

The oracle beamforms and de-disperses each stream (the same definitions as
the plain path), carries the last 16 frames of the previous block, and
inverts each block with ``lsmr_invert``.  Tolerance: in the kernel the
vectors and scalars are FP32; 25 LSMR steps on these window systems move the
FP32 iterate ~1e-7 (relative) from the FP64 one, the inverse FFT adds ~1e-6:
TOL_LSMR = 1e-5 for the FP32 beamformer, the FP16 form's own 1e-4 above it.
"""

import numpy as np
import pytest

import oracle as O
from gpu_common import TOL_TS_FP16, assert_samples_close, make_plan, random_case, rel_rms

pytestmark = pytest.mark.gpu

TOL_LSMR = 1e-5
# per sample: the error of the FP32 iterate is spread like the RMS one, so the
# largest of the <= 1e7 samples of a case stays below 6.5 times the RMS bound;
# with the noise level and the local envelope as the scale, 8 * tol
SAMPLE_FACTOR = 8.0


def _oracle_series(blocks, enu, dirs, tec, fb, P, K, B, Tr, F, k_sigma=6.0, alpha=0.25):
    """Per block: the LSMR series per stream [J, F, M], its per-phase noise
    levels [J, M] (running update) and the set of triggers {(j, n)}."""
    nu = O.sky_frequencies(fb, K)
    w = O.geometric_weights(nu, enu, dirs)
    d = O.dedispersion_weights(nu, tec, 0.5 * (nu[0] + nu[-1]))
    h = O.prototype_filter()
    J = B * Tr * P
    hist = np.zeros((J, O.LSMR_OVERLAP, K), dtype=complex)
    s2 = None
    out = []
    for bi, xb in enumerate(blocks):
        xc = xb[..., 0].astype(np.float64) + 1j * xb[..., 1]
        bm = O.beamform(xc, w, d)                                # [B, Tr, P, K, F]
        xs = np.zeros((J, F, O.M), dtype=complex)
        for b in range(B):
            for t in range(Tr):
                for p in range(P):
                    j = (b * Tr + t) * P + p
                    fr = np.concatenate([hist[j], bm[b, t, p].T])
                    xs[j] = O.lsmr_invert(fr, fb, h)
                    hist[j] = fr[-O.LSMR_OVERLAP:]
        pw = np.stack([O.lsmr_noise_power(xs[j]) for j in range(J)])
        s2 = O.update_sigma2(s2, pw, alpha, bi == 0)
        sig = np.sqrt(s2)
        n = ((bi * F + np.arange(F) - O.LSMR_OVERLAP)[:, None] * O.M + np.arange(O.M)[None, :])
        trig = set()
        for j in range(J):
            hit = (np.abs(xs[j]) > k_sigma * sig[j][None, :]) & (n >= 0)
            trig |= {(j, int(v)) for v in n[hit]}
        out.append((xs, sig, trig, n))
    return out


def _check_lsmr_triggers(gpu_trig, xs, sig, trig, n, k_sigma, tau):
    """Triggers equal except samples within tau of their per-phase threshold."""
    got = {(int(r["stream"]), int(r["n"])) for r in gpu_trig}
    first = int(n[0, 0])
    for (j, nn) in got ^ trig:
        i, p = divmod(nn - first, O.M)
        th = k_sigma * sig[j, p]
        assert abs(abs(xs[j, i, p]) - th) <= tau * th, (j, nn)
    return len(got), len(trig)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_lsmr_inversion_matches_oracle(cuda_lib, precision):
    """Two blocks of two windows each (history across the block boundary): the
    series, the per-phase noise levels (running update) and the triggers."""
    S, P, K, B, Tr, F, fb, ks = 8, 1, 12, 2, 1, 512, 200, 3.5
    blocks, enu, dirs, tec = random_case(51, S, P, K, B, Tr, F, fb, "int8", 2, amp=60)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision=precision,
                     inversion="lsmr", k_sigma=ks)
    assert plan.lp_launches_per_block() == 6
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    want = _oracle_series(blocks, enu, dirs, tec, fb, P, K, B, Tr, F, k_sigma=ks)
    import torch
    tol = TOL_LSMR if precision == "fp32" else TOL_TS_FP16
    for xb, (xs, sig, trig, n) in zip(blocks, want):
        plan.lp_process_block(torch.from_numpy(xb).cuda())
        got = np.stack([plan.lp_get_timeseries(b, 0, 0) for b in range(B)])
        assert rel_rms(got, xs.real.reshape(B, -1)) < tol
        sig_j = np.sqrt(np.mean(sig ** 2, axis=1))
        assert_samples_close(got, xs.real.reshape(B, -1), np.abs(xs).reshape(B, -1), sig_j,
                             SAMPLE_FACTOR * tol)
        np.testing.assert_allclose(plan.lp_get_lsmr_sigma(), sig, rtol=10 * tol)
        np.testing.assert_allclose(plan.lp_get_sigma(), np.sqrt(np.mean(sig ** 2, axis=1)),
                                   rtol=10 * tol)
        g_trig, n_total, st = plan.lp_get_triggers()
        ng, no = _check_lsmr_triggers(g_trig, xs, sig, trig, n, ks, 10 * tol)
        assert no > 0


def test_lsmr_iterations_and_limits(cuda_lib):
    """A different iteration count follows the oracle too; the block length must
    be a multiple of the window."""
    S, P, K, B, Tr, F, fb = 4, 1, 6, 1, 1, 256, 300
    blocks, enu, dirs, tec = random_case(52, S, P, K, B, Tr, F, fb, "int16", 1, amp=300)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int16", inversion="lsmr", lsmr_iters=7)
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    import torch
    plan.lp_process_block(torch.from_numpy(blocks[0]).cuda())
    nu = O.sky_frequencies(fb, K)
    xc = blocks[0][..., 0].astype(np.float64) + 1j * blocks[0][..., 1]
    bm = O.beamform(xc, O.geometric_weights(nu, enu, dirs),
                    O.dedispersion_weights(nu, tec, 0.5 * (nu[0] + nu[-1])))
    fr = np.concatenate([np.zeros((O.LSMR_OVERLAP, K)), bm[0, 0, 0].T])
    want = O.lsmr_invert(fr, fb, O.prototype_filter(), iters=7).real.reshape(-1)
    assert rel_rms(plan.lp_get_timeseries(0, 0, 0), want) < TOL_LSMR
    with pytest.raises(cuda_lib.LPError):
        make_plan(cuda_lib, S, P, K, B, Tr, 384, fb, "int16", inversion="lsmr")


def test_lsmr_host_input_and_graph_equal_device_input(cuda_lib):
    """A host block (copied whole, then inverted) and a graph replay give the
    device block's series bit for bit, over blocks with carried history."""
    import torch
    S, P, K, B, Tr, F, fb = 4, 2, 8, 1, 1, 256, 150
    blocks, enu, dirs, tec = random_case(53, S, P, K, B, Tr, F, fb, "int8", 2, amp=50)
    res = []
    for mode in ("device", "host", "graph"):
        stream = torch.cuda.Stream()
        plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", inversion="lsmr",
                         host_input=mode == "host", use_graph=mode == "graph", stream=stream)
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
            out.append(np.stack([plan.lp_get_timeseries(0, 0, p) for p in range(P)]))
        res.append(out)
    for other in res[1:]:
        for a, b in zip(res[0], other):
            np.testing.assert_array_equal(a, b)


def test_fine_dedispersion_then_lsmr_matches_oracle(cuda_lib):
    """The channel-domain filter feeds the LSMR inversion (both histories carried)."""
    S, P, K, B, Tr, F, fb = 6, 1, 16, 1, 2, 256, 60
    blocks, enu, dirs, tec = random_case(54, S, P, K, B, Tr, F, fb, "int16", 2, amp=200)
    tec = np.array([9.0, 31.0])
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int16", inversion="lsmr",
                     fine_dedisp=True)
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    nu = O.sky_frequencies(fb, K)
    nu_ref = 0.5 * (nu[0] + nu[-1])
    w = O.geometric_weights(nu, enu, dirs)
    d = O.dedispersion_weights(nu, tec, nu_ref)
    r = O.fine_dedispersion_taps(nu, tec, nu_ref)
    h = O.prototype_filter()
    fine_hist = np.zeros((Tr, O.FINE_TAPS - 1, K), dtype=complex)
    lsmr_hist = np.zeros((Tr, O.LSMR_OVERLAP, K), dtype=complex)
    import torch
    for xb in blocks:
        plan.lp_process_block(torch.from_numpy(xb).cuda())
        bm = O.beamform(xb[..., 0].astype(np.float64) + 1j * xb[..., 1], w, d)
        for t in range(Tr):
            fext = np.concatenate([fine_hist[t], bm[0, t, 0].T])
            fr = O.fine_dedisperse(fext, r[:, t])
            fine_hist[t] = fext[-(O.FINE_TAPS - 1):]
            lext = np.concatenate([lsmr_hist[t], fr])
            want = O.lsmr_invert(lext, fb, h).real.reshape(-1)
            lsmr_hist[t] = lext[-O.LSMR_OVERLAP:]
            assert rel_rms(plan.lp_get_timeseries(0, t, 0), want) < TOL_LSMR
