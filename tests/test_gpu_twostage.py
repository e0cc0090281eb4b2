"""Two-stage beamforming on the GPU against the FP64 oracle.

Stage 1 (preliminary beams of station groups, int16 transport) is compared
code for code: the kernel sums in FP32 and the oracle in FP64, so a code may
differ by one where scale * value lies within the FP32 summation error of a
rounding boundary (a half-integer); every other code must be equal.  The
whole chain (stage 1, then the ordinary pipeline with the group centres as
stations) is compared on time series and triggers, each side running its own
stage 1.
"""

import numpy as np
import pytest

import oracle as O
import synth
from gpu_common import TAU_FP32, TOL_TS_FP32, compare_triggers, gpu_blocks, make_plan, \
    oracle_blocks, rel_rms

pytestmark = pytest.mark.gpu


def _oracle_codes(x, enu, grp, gdir, first_bin, scale):
    """Oracle int16 codes, scale * value (FP64, [..., 2]) and a bound on the
    FP32 error of the kernel's scale * value: (n_g + 2) 2^-23 scale sum |x|."""
    P, K, F, S, _ = x.shape
    nu = O.sky_frequencies(first_bin, K)
    pbv = O.prebeam(x[..., 0].astype(np.float64) + 1j * x[..., 1],
                    O.prebeam_weights(nu, enu, grp, gdir))
    G = gdir.shape[0]
    absx = np.abs(x.astype(np.float64)).sum(axis=-1)              # |re| + |im|, [P,K,F,S]
    bound = np.zeros(pbv.shape)
    for g in range(G):
        m = grp == g
        bound[..., g] = (m.sum() + 2) * 2.0 ** -23 * scale * absx[..., m].sum(axis=-1)
    v = np.stack([pbv.real, pbv.imag], axis=-1) * scale
    return O.transport_int16(pbv, scale), v, np.stack([bound, bound], axis=-1) + 1e-6


def _check_codes(got, want, v, window):
    """Codes equal except by one next to a half-integer of scale * value."""
    diff = got.astype(np.int64) - want
    assert np.abs(diff).max(initial=0) <= 1
    near = np.abs(np.abs(v - np.floor(v)) - 0.5) < window
    assert np.all(near[diff != 0])
    assert np.count_nonzero(diff) <= 1e-3 * diff.size + 2
    return np.count_nonzero(diff)


@pytest.mark.parametrize("dtype,amp,scale,S,G,F", [
    ("int8", 128, 2.0, 20, 5, 700), ("int16", 3000, 4.0, 20, 5, 700), ("int8", 128, 2.0, 21, 5, 700),
    ("int8", 128, 2.0, 24, 8, 701), ("int8", 128, 64.0, 16, 4, 700), ("int8", 128, 2.0, 48, 16, 512)])
def test_prebeam_matches_oracle(cuda_lib, dtype, amp, scale, S, G, F):
    """20 stations, 5 groups: 16-byte chunk reads; 21 (int8): slabs not 16-byte
    aligned, sample-by-sample reads.  int8 with S a multiple of 8 and 4, 8 or 16
    groups: the frame-pair kernel (701 frames: a last pair with one frame;
    scale 64: saturating codes)."""
    import torch
    P, K, fb = 2, 6, 130                               # 700 frames: two tiles + a ragged one
    rng = np.random.default_rng(61)
    info = np.iinfo(dtype)
    x = rng.integers(max(info.min, -amp), min(info.max, amp) + 1,
                     size=(P, K, F, S, 2)).astype(dtype)
    enu = synth.station_positions(S, 62)
    grp = synth.station_groups(enu, G)
    spare = int(np.flatnonzero(grp == np.argmax(np.bincount(grp)))[0])
    grp[spare] = -1                                    # one unused station
    gdir = synth.hex_beam_directions(G, spacing_deg=0.4)
    pb = cuda_lib.Prebeam(S, P, K, F, G, first_bin=fb, input_dtype=dtype)
    pb.lp_prebeam_set_groups(grp, enu, gdir)
    np.testing.assert_allclose(pb.lp_prebeam_group_centres(), O.group_centres(enu, grp, G),
                               rtol=0, atol=1e-9)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty((P, K, F, G, 2), dtype=torch.int16, device="cuda")
    pb.lp_prebeam_run(xd, yd, scale)
    got = yd.cpu().numpy()
    want, v, window = _oracle_codes(x, enu, grp, gdir, fb, scale)
    _check_codes(got, want, v, window)
    n_sat = pb.lp_prebeam_saturated()
    sat_oracle = int(np.count_nonzero(np.abs(np.rint(v)) > O.INT16_MAX))
    near_edge = int(np.count_nonzero(np.abs(np.abs(v) - (O.INT16_MAX + 0.5)) < window))
    assert abs(n_sat - sat_oracle) <= near_edge
    if dtype == "int16" or scale > 8:
        assert sat_oracle > 0                          # the case does saturate
    assert pb.lp_prebeam_saturated() == 0              # the count resets


@pytest.mark.parametrize("G", [6, 8])
def test_two_stage_chain_matches_oracle(cuda_lib, G):
    """Station block -> preliminary beams (GPU) -> final beams, synthesis and
    triggers (GPU, stations = groups at their centres), against the oracle
    doing the same two stages in FP64 (8 groups: the frame-pair stage 1)."""
    import torch
    S, P, K, F, fb = 24, 2, 10, 1024, 200
    B, Tr, scale, nblocks = 3, 2, 4.0, 2
    rng = np.random.default_rng(63)
    blocks = [rng.integers(-20, 21, size=(P, K, F, S, 2)).astype(np.int8) for _ in range(nblocks)]
    enu = synth.station_positions(S, 64)
    grp = synth.station_groups(enu, G)
    gdir = np.tile(synth.pointing_enu(), (G, 1))
    dirs = synth.hex_beam_directions(B)
    tec = np.array([4.0, 25.0])

    pb = cuda_lib.Prebeam(S, P, K, F, G, first_bin=fb, input_dtype="int8")
    pb.lp_prebeam_set_groups(grp, enu, gdir)
    stage1 = []
    for xb in blocks:
        yd = torch.empty((P, K, F, G, 2), dtype=torch.int16, device="cuda")
        pb.lp_prebeam_run(torch.from_numpy(xb).cuda(), yd, scale)
        stage1.append(yd.cpu().numpy())
    assert pb.lp_prebeam_saturated() == 0
    plan = make_plan(cuda_lib, G, P, K, B, Tr, F, fb, "int16", store_timeseries=True,
                     k_sigma=4.5)
    gout = gpu_blocks(cuda_lib, plan, stage1, pb.lp_prebeam_group_centres(), dirs, tec)

    cen = O.group_centres(enu, grp, G)
    codes = [_oracle_codes(xb, enu, grp, gdir, fb, scale)[0] for xb in blocks]
    _, oout = oracle_blocks(G, P, K, B, Tr, F, fb, codes, cen, dirs, tec, k_sigma=4.5)
    for g_, o_, c_gpu, c_ora in zip(gout, oout, stage1, codes):
        # the chain is linear in the stage-1 codes, so codes that the two sides
        # rounded differently (by one, next to a half-integer) add at most
        # ||delta c|| / ||c|| = sqrt(n_mismatch) / ||c|| of relative error
        n_mis = int(np.count_nonzero(c_gpu != c_ora))
        assert n_mis <= 1e-4 * c_ora.size + 2
        tie = np.sqrt(n_mis) / np.linalg.norm(c_ora.astype(np.float64))
        assert rel_rms(g_["y"], o_["y"]) < TOL_TS_FP32 + 3 * tie
        n_g, n_o, n_diff, bad = compare_triggers(g_["trig"], o_, P, Tr, TAU_FP32)
        assert n_o > 0 and not bad


def test_prebeam_full_size_sampled(cuda_lib):
    """The benchmarked stage-1 launch (48 stations in 8 groups, 488 subbands,
    a whole 65536-frame block, int8; the frame-pair kernel): every subband and
    group at three sampled frame windows (start, middle, end) against the
    oracle, code for code; the noise block cannot saturate at scale 4."""
    import torch
    w = synth.PRECISION
    G, scale = 8, 4.0
    enu, _, _ = synth.make_geometry(w)
    x = np.empty((w.pols, w.subbands, w.block_len, w.stations, 2), dtype=w.dtype)
    for pol in range(w.pols):
        for k in range(w.subbands):
            x[pol, k] = synth.noise_slab(w.seed, 0, pol, k, w.block_len, w.stations,
                                         w.noise_sigma, w.dtype)
    grp = synth.station_groups(enu, G)
    gdir = np.tile(synth.pointing_enu(), (G, 1))
    pb = cuda_lib.Prebeam(w.stations, w.pols, w.subbands, w.block_len, G,
                          first_bin=w.first_bin, input_dtype=w.dtype)
    pb.lp_prebeam_set_groups(grp, enu, gdir)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty((w.pols, w.subbands, w.block_len, G, 2), dtype=torch.int16, device="cuda")
    pb.lp_prebeam_run(xd, yd, scale)
    del xd
    assert pb.lp_prebeam_saturated() == 0
    F = w.block_len
    for (m0, m1) in [(0, 64), (31000, 31064), (F - 64, F)]:
        got = yd[:, :, m0:m1].cpu().numpy()
        want, v, window = _oracle_codes(x[:, :, m0:m1], enu, grp, gdir, w.first_bin, scale)
        _check_codes(got, want, v, window)
