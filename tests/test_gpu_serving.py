"""Strided block views, captured-graph mode and the continuous-batching loop.

The serving test runs several sessions of different shapes alone and then
all together on their own CUDA streams against one resident station block:
every session's triggers and noise level must be identical (the kernels are
deterministic, so the mix can change nothing).  A small HBM budget checks that
admission waits for memory to free up.
"""

import numpy as np
import pytest

import synth
from gpu_common import TOL_TS_FP32, gpu_blocks, make_plan, random_case, rel_rms

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_strided_view_equals_contiguous_block(cuda_lib, precision):
    import torch
    S, P, Kfull, F, fb0 = 8, 2, 30, 96, 100
    k0, K, B, Tr = 7, 12, 3, 2
    blocks, enu, dirs, tec = random_case(41, S, P, Kfull, B, Tr, F, fb0, "int8", 2, amp=100)
    ys = []
    for view in (False, True):
        plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb0 + k0, "int8", precision=precision,
                         store_timeseries=True, k_sigma=3.0)
        plan.lp_set_weights(enu, dirs)
        plan.lp_set_tec(tec)
        out = []
        for xb in blocks:
            if view:
                full = torch.from_numpy(np.ascontiguousarray(xb)).cuda()
                flat = full.view(-1)
                off = k0 * F * S * 2
                plan.lp_process_block_strided(flat[off:], Kfull * F * S)
            else:
                sub = np.ascontiguousarray(xb[:, k0:k0 + K])
                plan.lp_process_block(torch.from_numpy(sub).cuda())
            out.append((plan.lp_get_timeseries(2, 1, 1), plan.lp_get_triggers()[0]))
        ys.append(out)
    for (ya, ta), (yb, tb) in zip(*ys):
        np.testing.assert_array_equal(ya, yb)
        np.testing.assert_array_equal(ta, tb)


def test_graph_mode_equals_direct_launches(cuda_lib):
    import torch
    S, P, K, B, Tr, F, fb = 8, 2, 20, 4, 2, 128, 210
    blocks, enu, dirs, tec = random_case(42, S, P, K, B, Tr, F, fb, "int8", 3, amp=100)
    res = []
    for graph in (False, True):
        stream = torch.cuda.Stream()
        plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision="fp16",
                         store_timeseries=True, k_sigma=3.0, use_graph=graph, stream=stream)
        plan.lp_set_weights(enu, dirs, stream=stream)
        plan.lp_set_tec(tec, stream=stream)
        xd = torch.empty((P, K, F, S, 2), dtype=torch.int8, device="cuda")
        out = []
        for xb in blocks:              # same device address every block: one capture
            with torch.cuda.stream(stream):
                xd.copy_(torch.from_numpy(xb))
            plan.lp_process_block(xd, stream=stream)
            out.append((plan.lp_get_timeseries(3, 1, 0), plan.lp_get_triggers()[0],
                        plan.lp_get_sigma()))
        res.append(out)
    for a, b in zip(*res):
        for u, v in zip(a, b):
            np.testing.assert_array_equal(u, v)


def _serve(lp, reqs, budget, enu, grid, blocks, F, n_sub, fb0, S=8, batch=True):
    import torch
    from paper_1612_06592_gb300.serve import Server
    srv = Server(S, 2, n_sub, fb0, F, enu, grid, budget, precision="fp16", k_sigma=3.5,
                 batch=batch)
    hosts = [torch.from_numpy(np.ascontiguousarray(b).reshape(-1)).pin_memory() for b in blocks]
    got = {r.rid: [] for r in reqs}
    admitted_at = {}
    for bi, h in enumerate(hosts):
        for r in reqs:
            if r.arrival == bi:
                srv.submit(r)
        srv.retire()
        for rid in srv.admit():
            admitted_at[rid] = bi
        out = srv.run_block(h)
        for rid, (trig, n) in out.items():
            got[rid].append((bi, trig.copy(), srv.active[rid].plan.lp_get_sigma().copy()))
    return got, admitted_at


def test_serving_results_identical_alone_and_in_the_mix(cuda_lib):
    from paper_1612_06592_gb300.serve import Request
    S, F, n_sub, fb0 = 8, 256, 40, 150
    grid = synth.hex_beam_directions(6)
    enu = synth.station_positions(S, 3)
    rng = np.random.default_rng(43)
    blocks = [rng.integers(-90, 91, size=(2, n_sub, F, S, 2)).astype(np.int8) for _ in range(4)]
    reqs = [Request(0, np.array([0, 2, 5]), 3, 20, np.array([8.0]), 0, 4),
            Request(1, np.array([1]), 0, 40, np.array([5.0, 12.0, 30.0]), 0, 3),
            Request(2, np.array([0, 1, 2, 3, 4, 5]), 10, 24, np.array([20.0, 35.0]), 1, 3)]
    mixed, _ = _serve(cuda_lib, reqs, 1e12, enu, grid, blocks, F, n_sub, fb0)
    for r in reqs:
        alone, _ = _serve(cuda_lib, [r], 1e12, enu, grid, blocks, F, n_sub, fb0)
        assert len(alone[r.rid]) == len(mixed[r.rid]) == r.blocks
        for (ba, ta, sa), (bm, tm, sm) in zip(alone[r.rid], mixed[r.rid]):
            assert ba == bm
            np.testing.assert_array_equal(ta, tm)
            np.testing.assert_array_equal(sa, sm)


def test_batched_serving_equals_unbatched_and_launches_do_not_grow(cuda_lib):
    """The batched server (all sessions in four shared launches per polarisation
    of a block) gives each request exactly the results of the unbatched one (each
    session its own launches on its own stream); its launch count per block stays
    8 while the unbatched count grows with the sessions."""
    from paper_1612_06592_gb300.serve import Request, Server
    S, F, n_sub, fb0 = 8, 256, 40, 150
    grid = synth.hex_beam_directions(6)
    enu = synth.station_positions(S, 3)
    rng = np.random.default_rng(45)
    blocks = [rng.integers(-90, 91, size=(2, n_sub, F, S, 2)).astype(np.int8) for _ in range(4)]
    reqs = [Request(0, np.array([0, 2, 5]), 3, 20, np.array([8.0]), 0, 4),
            Request(1, np.array([1]), 0, 40, np.array([5.0, 12.0, 30.0]), 0, 3),
            Request(2, np.array([0, 1, 2, 3, 4, 5]), 10, 24, np.array([20.0, 35.0]), 1, 3),
            Request(3, np.array([4]), 16, 24, np.array([9.0]), 1, 2)]
    batched, _ = _serve(cuda_lib, reqs, 1e12, enu, grid, blocks, F, n_sub, fb0, batch=True)
    single, _ = _serve(cuda_lib, reqs, 1e12, enu, grid, blocks, F, n_sub, fb0, batch=False)
    for r in reqs:
        assert len(batched[r.rid]) == len(single[r.rid]) == r.blocks
        for (ba, ta, sa), (bs, ts, ss) in zip(batched[r.rid], single[r.rid]):
            assert ba == bs
            np.testing.assert_array_equal(ta, ts)
            np.testing.assert_array_equal(sa, ss)
    srv = Server(S, 2, n_sub, fb0, F, enu, grid, 1e12, precision="fp16", k_sigma=3.5)
    import torch
    h = torch.from_numpy(np.ascontiguousarray(blocks[0]).reshape(-1)).pin_memory()
    for n in (1, 3, 6):
        while len(srv.active) < n:
            k = len(srv.active)
            srv.submit(Request(100 + k, np.array([k % 6]), 0, 20, np.array([10.0]), 0, 10))
            srv.admit()
        srv.run_block(h)
    assert srv.launches == [8, 8, 8]


def test_serving_calibration_fits_the_timed_blocks(cuda_lib):
    from paper_1612_06592_gb300.serve import Server
    S, F, n_sub, fb0 = 8, 8192, 488, 12
    grid = synth.hex_beam_directions(40)
    enu = synth.station_positions(S, 3)
    srv = Server(S, 2, n_sub, fb0, F, enu, grid, 1e12, precision="fp16")
    m = srv.calibrate()
    assert m.measured and m.c_stream >= 0 and m.c_row >= 0 and m.c_in >= 0
    assert len(srv.calibration) == 7 and all(c["ms"] > 0 for c in srv.calibration)
    # the fitted model reproduces the combined block within a factor of two
    comb = srv.calibration[-1]
    pred = m.fixed(F) + sum(m.session(P, K, B, Tr, F) for P, K, B, Tr in comb["sessions"])
    assert 0.5 < pred / comb["ms"] < 2.0


def test_serving_admission_waits_for_memory(cuda_lib):
    from paper_1612_06592_gb300.serve import Request, workspace_bytes
    S, F, n_sub, fb0 = 8, 128, 30, 150
    grid = synth.hex_beam_directions(4)
    enu = synth.station_positions(S, 5)
    rng = np.random.default_rng(44)
    blocks = [rng.integers(-90, 91, size=(2, n_sub, F, S, 2)).astype(np.int8) for _ in range(5)]
    reqs = [Request(0, np.array([0, 1, 2, 3]), 0, 30, np.array([10.0]), 0, 2),
            Request(1, np.array([0, 1, 2, 3]), 0, 30, np.array([10.0]), 0, 2),
            Request(2, np.array([0] * 1), 0, 30, np.array([10.0] * 1), 0, 1)]
    one = workspace_bytes(S, 2, 30, 4, 1, F, fb0, "fp16")
    got, admitted_at = _serve(cuda_lib, reqs, int(one * 1.5), enu, grid, blocks, F, n_sub, fb0)
    # only one big session fits: the second waits until the first has finished
    assert admitted_at[0] == 0 and admitted_at[1] == 2
    assert len(got[0]) == 2 and len(got[1]) == 2
    # the small one is queued behind request 1 (arrival order) and runs after it
    assert admitted_at[2] >= 2


@pytest.mark.parametrize("graph", [False, True])
def test_chunked_block_equals_whole_block(cuda_lib, graph):
    """Frame chunks inside a block (beam rows sized for one chunk, noise level
    from a first power-only pass), launched directly or from a captured graph,
    give exactly the unchunked results."""
    import torch
    S, P, K, B, Tr, F, fb = 8, 2, 12, 5, 2, 8192, 140
    blocks, enu, dirs, tec = random_case(45, S, P, K, B, Tr, F, fb, "int8", 2, amp=100)
    res = []
    for chunk in (0, 2048, 512, 256):
        stream = torch.cuda.Stream()
        plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision="fp16",
                         store_timeseries=True, k_sigma=3.5, chunk_frames=chunk,
                         use_graph=graph and chunk > 0, stream=stream)
        plan.lp_set_weights(enu, dirs, stream=stream)
        plan.lp_set_tec(tec, stream=stream)
        xd = torch.empty((P, K, F, S, 2), dtype=torch.int8, device="cuda")
        out = []
        for xb in blocks:              # same device address every block: one capture
            with torch.cuda.stream(stream):
                xd.copy_(torch.from_numpy(xb))
            plan.lp_process_block(xd, stream=stream)
            out.append((plan.lp_get_timeseries(4, 1, 1), plan.lp_get_timeseries(0, 0, 0),
                        plan.lp_get_triggers()[0], plan.lp_get_sigma()))
        if chunk:
            with pytest.raises(cuda_lib.LPError):
                plan.lp_get_beams(0, 0, 0)       # only one chunk of rows is kept
            assert plan.lp_launches_per_block() == 2 + 3 * (F // chunk)
        res.append(out)
    for other in res[1:]:
        for a, b in zip(res[0], other):
            for u, v in zip(a, b):
                np.testing.assert_array_equal(u, v)


def test_autotune_keeps_results(cuda_lib):
    import torch
    S, P, K, B, Tr, F, fb = 8, 2, 16, 6, 1, 4096, 200
    blocks, enu, dirs, tec = random_case(46, S, P, K, B, Tr, F, fb, "int8", 2, amp=100)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision="fp16",
                     store_timeseries=True, k_sigma=3.5)
    ref = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision="fp16",
                    store_timeseries=True, k_sigma=3.5)
    for p in (plan, ref):
        p.lp_set_weights(enu, dirs)
        p.lp_set_tec(tec)
    for i, xb in enumerate(blocks):
        xd = torch.from_numpy(xb).cuda()
        ref.lp_process_block(xd)
        if i == 0:                     # the tuned block's outputs are a normal block's
            best, ms = plan.lp_plan_autotune(xd)
            assert best in ms and len(ms) >= 5 and all(v > 0 for v in ms.values())
        else:
            plan.lp_process_block(xd)
        np.testing.assert_array_equal(plan.lp_get_timeseries(5, 0, 1), ref.lp_get_timeseries(5, 0, 1))
        np.testing.assert_array_equal(plan.lp_get_triggers()[0], ref.lp_get_triggers()[0])
        np.testing.assert_array_equal(plan.lp_get_sigma(), ref.lp_get_sigma())


@pytest.mark.parametrize("precision,chunk", [("fp32", 0), ("fp16", 0), ("fp16", 2048)])
def test_gemm_configs_bit_identical(cuda_lib, precision, chunk):
    """Every beamformer configuration the GEMM autotuner may pick (ring depths of
    the tensor-core form, beams per pass of the FP32 form) gives the same beams,
    noise level, time series and triggers bit for bit; so does a block processed
    by the autotuner itself."""
    import torch
    S, P, K, B, Tr, F, fb = 24, 2, 12, 37, 2, 4096, 230
    blocks, enu, dirs, tec = random_case(47, S, P, K, B, Tr, F, fb, "int8", 2, amp=60)
    plan = make_plan(cuda_lib, S, P, K, B, Tr, F, fb, "int8", precision=precision,
                     store_timeseries=True, k_sigma=5.0, chunk_frames=chunk)
    plan.lp_set_weights(enu, dirs)
    plan.lp_set_tec(tec)
    cfgs = plan.lp_plan_gemm_configs()
    if precision == "fp32":
        assert cfgs == [(8, 0), (16, 0), (4, 0)]
    else:
        assert len(cfgs) >= 2 and all(1 <= a <= 3 and 1 <= b <= 2 for a, b in cfgs)
    xds = [torch.from_numpy(xb).cuda() for xb in blocks]

    def run(index, tune=False):
        plan.lp_reset_stream()
        if not tune:
            plan.lp_plan_set_gemm_config(index)
        out = []
        for i, xd in enumerate(xds):
            if tune and i == 0:
                best, ms = plan.lp_plan_autotune_gemm(xd)
                assert 0 <= best < len(cfgs) and cfgs[best] in ms
                assert len(ms) == len(cfgs) and all(v > 0 for v in ms.values())
            else:
                plan.lp_process_block(xd)
            trig, n_trig, st = plan.lp_get_triggers()
            assert st == 0 and 0 < n_trig == len(trig)   # the whole list (no overflow)
            out.append((plan.lp_get_beams(36, 1, 1) if not chunk else None,
                        plan.lp_get_timeseries(36, 1, 1), plan.lp_get_timeseries(3, 0, 0),
                        plan.lp_get_sigma(), trig))
        return out

    ref = run(-1)
    for i in list(range(len(cfgs))) + ["tune"]:
        got = run(-1, tune=True) if i == "tune" else run(i)
        for a, b in zip(ref, got):
            for u, v in zip(a, b):
                if u is not None:
                    np.testing.assert_array_equal(u, v)
    with pytest.raises(Exception):
        plan.lp_plan_set_gemm_config(len(cfgs))
