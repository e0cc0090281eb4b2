"""Beam sharding (Sec. 4: every node receives all station data, the beams are
divided among the nodes) on the CPU: the partition, the relabelling of a
shard's triggers to global indices, the merge, and a world-size-2 gloo run in
which each rank evaluates the FP64 oracle on its own beams of one block; the
gathered, merged list must equal the single-rank list of all beams.
"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1612_06592_gb300.shard import beam_range, merge_triggers, to_global


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_beam_range_partitions_every_beam_once():
    for B in (1, 2, 7, 50, 200):
        for world in range(1, min(B, 9) + 1):
            ranges = [beam_range(B, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == B
            for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
                assert a1 == b0                       # contiguous, disjoint
            sizes = [b1 - b0 for b0, b1 in ranges]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        beam_range(3, 4, 0)                          # a rank without a beam
    with pytest.raises(ValueError):
        beam_range(8, 2, 2)


def _records(rows):
    from paper_1612_06592_gb300.lp import TRIGGER_DTYPE
    return np.array(rows, dtype=TRIGGER_DTYPE)


def test_to_global_and_merge_order():
    Tr, P = 3, 2
    # shard beams 4..5: local beam 1, trial 2, pol 1 -> global beam 5, stream (5*3+2)*2+1
    loc = _records([(900, 1, 2, 1, (1 * Tr + 2) * P + 1, 9.0, 1.0),
                    (100, 0, 0, 0, 0, 8.0, 1.0)])
    g = to_global(loc, 4, Tr, P)
    assert list(g["beam"]) == [5, 4]
    assert list(g["stream"]) == [(5 * Tr + 2) * P + 1, (4 * Tr + 0) * P + 0]
    assert list(loc["beam"]) == [1, 0]               # the input is not modified
    other = _records([(50, 0, 1, 0, 2, 7.0, 1.0), (40, 0, 1, 0, 2, 7.5, 1.0)])
    m = merge_triggers([g, None, other])
    keys = list(zip(m["beam"], m["tec"], m["pol"], m["n"]))
    assert keys == sorted(keys) and len(m) == 4
    assert len(merge_triggers([])) == 0


def _oracle_records(res, b0, Tr, P):
    rows = [(n, b, t, p, (b * Tr + t) * P + p, e, s) for (n, b, t, p, e, s) in res["triggers"]]
    return to_global(_records(rows), b0, Tr, P)


CASE = dict(S=5, P=2, K=12, B=5, Tr=2, F=64, fb=180, k_sigma=3.0)


def _case_inputs():
    import synth
    c = CASE
    rng = np.random.default_rng(77)
    x = rng.integers(-40, 41, size=(c["P"], c["K"], c["F"], c["S"], 2)).astype(np.int16)
    enu = synth.station_positions(c["S"], 3)
    dirs = synth.hex_beam_directions(c["B"])
    tec = np.array([6.0, 25.0])
    return x, enu, dirs, tec


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import oracle as O
    from paper_1612_06592_gb300.shard import gather_sigma, gather_triggers
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = CASE
    x, enu, dirs, tec = _case_inputs()
    b0, b1 = beam_range(c["B"], world, rank)
    pipe = O.Pipeline(c["S"], c["P"], c["K"], b1 - b0, c["Tr"], c["F"], c["fb"], enu,
                      dirs[b0:b1], tec, k_sigma=c["k_sigma"])
    res = pipe.process_block(x)
    merged = gather_triggers(_oracle_records(res, b0, c["Tr"], c["P"]))
    sig = gather_sigma(res["sigma"])
    if rank == 0:
        out["merged"] = merged.tobytes()
        out["sigma"] = sig.tobytes()
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_oracle_gloo_two_ranks_equals_single_rank():
    import oracle as O
    from paper_1612_06592_gb300.lp import TRIGGER_DTYPE
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    c = CASE
    x, enu, dirs, tec = _case_inputs()
    full = O.Pipeline(c["S"], c["P"], c["K"], c["B"], c["Tr"], c["F"], c["fb"], enu, dirs, tec,
                      k_sigma=c["k_sigma"]).process_block(x)
    want = merge_triggers([_oracle_records(full, 0, c["Tr"], c["P"])])
    got = np.frombuffer(out["merged"], dtype=TRIGGER_DTYPE)
    assert len(want) > 50
    key = ("n", "beam", "tec", "pol", "stream")
    assert [tuple(r[k] for k in key) for r in got] == [tuple(r[k] for k in key) for r in want]
    np.testing.assert_allclose(got["env"], want["env"], rtol=1e-12)
    np.testing.assert_allclose(np.frombuffer(out["sigma"], dtype=np.float64), full["sigma"],
                               rtol=1e-12)
