"""Plan groups (lp_group): several sessions' blocks in four shared launches.

Plans of different beams, STEC trials and subband ranges of one station block
run as one group; every plan's time series, noise level and triggers equal,
bit for bit, those of the same plan processed alone, over several blocks
(history and running noise level carried), and a group makes four launches per
block whatever its size.
"""

import numpy as np
import pytest

import synth
from gpu_common import make_plan

pytestmark = pytest.mark.gpu


def _plans(lp, S, F, n_sub, fb0, enu, grid, shapes, stream=None):
    out = []
    for (beams, k0, nsub, tec) in shapes:
        p = make_plan(lp, S, 2, nsub, len(beams), len(tec), F, fb0 + k0, "int8",
                      precision="fp16", store_timeseries=True, k_sigma=3.5, stream=stream)
        p.lp_set_weights(enu, grid[beams], stream=stream)
        p.lp_set_tec(np.asarray(tec), stream=stream)
        out.append(p)
    return out


def _outputs(p):
    S, P, K, B, Tr, F = p.shape
    ys = np.stack([p.lp_get_timeseries(b, t, q) for b in range(B) for t in range(Tr)
                   for q in range(P)])
    return ys, p.lp_get_sigma().copy(), p.lp_get_triggers()[0]


def test_group_equals_plans_alone(cuda_lib):
    import torch
    lp = cuda_lib
    S, F, n_sub, fb0 = 8, 520, 40, 150
    grid = synth.hex_beam_directions(7)
    enu = synth.station_positions(S, 9)
    rng = np.random.default_rng(71)
    blocks = [rng.integers(-90, 91, size=(2, n_sub, F, S, 2)).astype(np.int8) for _ in range(3)]
    shapes = [(np.array([0, 2, 5]), 3, 20, [8.0]),
              (np.array([1]), 0, 40, [5.0, 12.0, 30.0]),
              (np.array([0, 1, 2, 3, 4, 5, 6]), 10, 24, [20.0, 35.0]),
              (np.array([6, 4]), 33, 7, [15.0])]
    stream = torch.cuda.Stream()
    grouped = _plans(lp, S, F, n_sub, fb0, enu, grid, shapes, stream)
    alone = _plans(lp, S, F, n_sub, fb0, enu, grid, shapes, stream)
    grp = lp.Group(grouped)
    assert grp.lp_group_launches_per_block() == 4
    xd = torch.empty((2, n_sub, F, S, 2), dtype=torch.int8, device="cuda")
    pol_stride = n_sub * F * S
    n_trig = 0
    for xb in blocks:
        with torch.cuda.stream(stream):
            xd.copy_(torch.from_numpy(xb))
        grp.lp_group_process_block(xd, n_sub, fb0, stream=stream)
        for (beams, k0, nsub, tec), pa in zip(shapes, alone):
            off = k0 * F * S * 2
            pa.lp_process_block_strided(xd.view(-1)[off:], pol_stride, stream=stream)
        for pg, pa in zip(grouped, alone):
            (yg, sg, tg), (ya, sa, ta) = _outputs(pg), _outputs(pa)
            np.testing.assert_array_equal(yg, ya)
            np.testing.assert_array_equal(sg, sa)
            np.testing.assert_array_equal(tg, ta)
            n_trig += len(tg)
    assert n_trig > 100
    grp.close()


def test_group_per_polarisation_equals_whole_block(cuda_lib):
    """A block run one polarisation at a time (pol 0, then pol 1) gives every
    plan's series, noise level and triggers of the whole-block call, bit for
    bit, over three blocks; polarisations out of order, out of range, or a
    whole-block call between them are refused."""
    import torch
    lp = cuda_lib
    S, F, n_sub, fb0 = 8, 264, 30, 140
    grid = synth.hex_beam_directions(5)
    enu = synth.station_positions(S, 4)
    rng = np.random.default_rng(72)
    blocks = [rng.integers(-90, 91, size=(2, n_sub, F, S, 2)).astype(np.int8) for _ in range(3)]
    shapes = [(np.array([0, 3]), 2, 18, [9.0]), (np.array([1, 2, 4]), 0, 30, [6.0, 25.0])]
    stream = torch.cuda.Stream()
    whole = lp.Group(_plans(lp, S, F, n_sub, fb0, enu, grid, shapes, stream))
    split = lp.Group(_plans(lp, S, F, n_sub, fb0, enu, grid, shapes, stream))
    xd = torch.empty((2, n_sub, F, S, 2), dtype=torch.int8, device="cuda")
    with pytest.raises(lp.LPError):
        split.lp_group_process_block_pol(xd, n_sub, fb0, 1, stream=stream)   # pol 0 first
    with pytest.raises(lp.LPError):
        split.lp_group_process_block_pol(xd, n_sub, fb0, 2, stream=stream)   # no pol 2
    n_trig = 0
    for i, xb in enumerate(blocks):
        with torch.cuda.stream(stream):
            xd.copy_(torch.from_numpy(xb))
        whole.lp_group_process_block(xd, n_sub, fb0, stream=stream)
        split.lp_group_process_block_pol(xd, n_sub, fb0, 0, stream=stream)
        if i == 0:
            with pytest.raises(lp.LPError):      # the block's pol 1 is still due
                split.lp_group_process_block(xd, n_sub, fb0, stream=stream)
        split.lp_group_process_block_pol(xd, n_sub, fb0, 1, stream=stream)
        for pw, ps in zip(whole.plans, split.plans):
            (yw, sw, tw), (ys, ss, ts) = _outputs(pw), _outputs(ps)
            np.testing.assert_array_equal(yw, ys)
            np.testing.assert_array_equal(sw, ss)
            np.testing.assert_array_equal(tw, ts)
            n_trig += len(tw)
    assert n_trig > 50
    whole.close()
    split.close()


def test_group_refuses_plans_it_cannot_fuse(cuda_lib):
    lp = cuda_lib
    S, F, fb = 8, 256, 150
    a = make_plan(lp, S, 2, 10, 2, 1, F, fb, "int8", precision="fp16")
    b32 = make_plan(lp, S, 2, 10, 2, 1, F, fb, "int8", precision="fp32")
    other_F = make_plan(lp, S, 2, 10, 2, 1, 2 * F, fb, "int8", precision="fp16")
    enu = synth.station_positions(S, 2)
    for p in (a, b32, other_F):
        p.lp_set_weights(enu, synth.hex_beam_directions(2))
        p.lp_set_tec(np.array([10.0]))
    for bad in ([a, b32], [a, other_F], [a, a]):
        with pytest.raises(lp.LPError):
            lp.Group(bad)
    g = lp.Group([a])
    import torch
    x = torch.zeros((2, 10, F, S, 2), dtype=torch.int8, device="cuda")
    with pytest.raises(lp.LPError):           # the plan's bins lie outside the block's
        g.lp_group_process_block(x, 10, fb + 1)
