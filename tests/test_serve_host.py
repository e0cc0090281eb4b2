"""Host logic of the serving loop, on the CPU: request generation and the
admission policy (FIFO; wait for memory; refuse what can never fit in memory
or in time; wait for a time slot; set-ups that would run into the next block
wait for the next gap; retire frees memory and cost; the cost correction
follows measured block times).  Plans and CUDA streams are replaced
by fakes; workspace sizes come from the library's host-only query."""

from collections import deque

import numpy as np
import pytest


@pytest.fixture(scope="module")
def serve():
    from paper_1612_06592_gb300 import build
    build()
    from paper_1612_06592_gb300 import serve as sv
    return sv


class _FakePlan:
    made = []

    def __init__(self, *a, **kw):
        _FakePlan.made.append((a, kw))

    def lp_set_weights(self, *a, **kw):
        pass

    def lp_set_tec(self, *a, **kw):
        pass

    def close(self):
        pass


class _FakeStream:
    def synchronize(self):
        pass


class _FakeTorch:
    class cuda:
        @staticmethod
        def Stream(device=None):
            return _FakeStream()


def _server(serve, monkeypatch, budget, time_budget_ms=None):
    monkeypatch.setattr(serve.lp, "Plan", _FakePlan)
    srv = object.__new__(serve.Server)
    srv.torch = _FakeTorch
    srv.S, srv.P, srv.n_sub, srv.fb0, srv.F = 48, 2, 488, 12, 65536
    srv.enu = np.zeros((48, 3))
    srv.grid = np.tile([0.0, 0.0, 1.0], (50, 1))
    srv.budget = int(budget)
    srv.precision = "fp16"
    srv.k_sigma = 6.0
    srv.use_graph = False
    srv.device = None
    srv.pending = deque()
    srv.active = {}
    srv.used = 0
    srv.ws_of = {}
    srv.log = []
    srv.time_budget_ms = time_budget_ms
    srv.cost_corr = serve.INITIAL_CORRECTION
    srv.cost_used = 0.0
    srv.copy_ms = 0.0
    srv.model = serve.PRIOR
    srv.batch = False
    srv.stream = None
    srv.groups, srv.group_key, srv.launches = [], None, []
    srv.setup_ms, srv.deferred = [], 0
    return srv


def _req(serve, rid, nb, nsub, ntr, blocks=2):
    return serve.Request(rid, np.arange(nb), 0, nsub, np.linspace(5, 30, ntr), 0, blocks)


def test_requests_are_seeded_and_within_bounds(serve):
    a = serve.make_requests(3, 200)
    b = serve.make_requests(3, 200)
    assert [(r.rid, r.k0, r.nsub, tuple(r.beams), tuple(r.tec)) for r in a] == \
           [(r.rid, r.k0, r.nsub, tuple(r.beams), tuple(r.tec)) for r in b]
    assert len(a) > 20 and [r.rid for r in a] == list(range(len(a)))
    for r in a:
        assert 1 <= len(r.beams) <= 50 and len(set(r.beams)) == len(r.beams)
        assert np.all(np.diff(r.beams) > 0) and r.beams.max() < 50
        assert 122 <= r.nsub <= 488 and 0 <= r.k0 and r.k0 + r.nsub <= 488
        assert 1 <= len(r.tec) <= 4 and np.all((r.tec >= 5) & (r.tec <= 40))
        assert 4 <= r.blocks <= 64
    assert all(x.arrival <= y.arrival for x, y in zip(a, a[1:]))


def test_workspace_query_and_cost_model(serve):
    small = serve.workspace_bytes(48, 2, 122, 1, 1, 65536, 12)
    big = serve.workspace_bytes(48, 2, 488, 50, 4, 65536, 12)
    assert big > 50 * small / 2
    # beam rows dominate: streams x subbands x (F + 16) complex floats
    assert big >= 50 * 4 * 2 * 488 * (65536 + 16) * 8
    c1 = serve.session_cost_ms(2, 488, 50, 1, 65536)
    assert c1 > 0
    assert abs(serve.session_cost_ms(2, 488, 50, 1, 32768) - c1 / 2) < 1e-12
    assert serve.session_cost_ms(2, 488, 50, 2, 65536) > c1


def test_admission_waits_for_memory_in_arrival_order(serve, monkeypatch):
    probe = _server(serve, monkeypatch, 1 << 62)
    r0, r1, r2 = _req(serve, 0, 30, 300, 2), _req(serve, 1, 40, 400, 2), _req(serve, 2, 1, 122, 1)
    w0, w1, w2 = probe._ws(r0), probe._ws(r1), probe._ws(r2)
    srv = _server(serve, monkeypatch, w0 + w1 - 1)
    for r in (r0, r1, r2):
        srv.submit(r)
    assert srv.admit() == [0]                 # r1 does not fit next to r0 ...
    assert [r.rid for r in srv.pending] == [1, 2]   # ... and r2 waits behind it (FIFO)
    assert srv.used == w0
    srv.active[0].blocks_done = r0.blocks
    assert srv.retire() == [0] and srv.used == 0 and srv.cost_used == 0.0
    assert srv.admit() == [1, 2] and srv.used == w1 + w2


def test_admission_refuses_what_can_never_fit(serve, monkeypatch):
    probe = _server(serve, monkeypatch, 1 << 62)
    big, small = _req(serve, 0, 50, 488, 4), _req(serve, 1, 2, 122, 1)
    srv = _server(serve, monkeypatch, probe._ws(big) - 1)
    srv.submit(big)
    srv.submit(small)
    assert srv.admit() == [1]
    assert srv.log == [("refused", 0, probe._ws(big))]
    # in time: a request whose own predicted time exceeds the budget
    srv = _server(serve, monkeypatch, 1 << 62, time_budget_ms=1.0)
    srv.submit(_req(serve, 5, 50, 488, 4))
    assert srv.admit() == [] and srv.log[0][:2] == ("refused", 5)


def test_admission_waits_for_a_time_slot_and_learns_the_cost(serve, monkeypatch):
    r0, r1 = _req(serve, 0, 20, 488, 2), _req(serve, 1, 20, 488, 2)
    c = serve.session_cost_ms(2, 488, 20, 2, 65536)
    # room for one session's predicted time (with the initial correction), not two
    srv = _server(serve, monkeypatch, 1 << 62, time_budget_ms=1.5 * c * serve.INITIAL_CORRECTION)
    srv.submit(r0)
    srv.submit(r1)
    assert srv.admit() == [0] and [r.rid for r in srv.pending] == [1]
    # measured blocks much faster than predicted: the correction falls, r1 fits
    for _ in range(20):
        srv.observe(0.5 * c)
    assert srv.cost_corr < 0.75 * serve.INITIAL_CORRECTION
    assert srv.admit() == [1]


def test_cost_model_fit_recovers_the_coefficients(serve):
    """The start-up calibration fits T = c0 + c_in * slab-tiles + c_row * rows +
    c_stream * streams by non-negative least squares: exact data from the
    calibration shapes give back the coefficients, at any block length."""
    truth = serve.CostModel(1.5, 2.0e-3, 4.0e-5, 0.21)
    shapes = [(1, 122, 1), (8, 488, 2), (16, 244, 1), (40, 488, 1), (2, 488, 4), (24, 160, 3)]
    combos = [[s] for s in shapes] + [shapes]
    for F in (65536, 16384):
        samples = [(F, [(2, K, B, Tr) for (B, K, Tr) in c],
                    truth.fixed(F) + sum(truth.session(2, K, B, Tr, F) for (B, K, Tr) in c))
                   for c in combos]
        m = serve.CostModel.fit(samples)
        assert m.measured
        np.testing.assert_allclose([m.c0, m.c_in, m.c_row, m.c_stream],
                                   [1.5, 2.0e-3, 4.0e-5, 0.21], rtol=1e-6)


def test_cost_used_is_recomputed_without_residue(serve, monkeypatch):
    srv = _server(serve, monkeypatch, 1 << 62)
    reqs = [_req(serve, i, 3 + i, 150 + 10 * i, 1 + i % 3, blocks=1) for i in range(5)]
    for r in reqs:
        srv.submit(r)
    srv.admit()
    for s in srv.active.values():
        s.blocks_done = 1
    srv.retire()
    assert srv.cost_used == 0.0 and not srv.active
    cc = srv.cost_corr
    srv.observe(50.0)                      # no session: the correction stays
    assert srv.cost_corr == cc


def test_setup_waits_for_a_gap_long_enough(serve, monkeypatch):
    """A set-up that, at the longest recent set-up time, would end after the
    next block's arrival waits (FIFO kept); with time enough it is admitted and
    its set-up time recorded."""
    import time
    r0, r1 = _req(serve, 0, 4, 122, 1), _req(serve, 1, 4, 122, 1)
    srv = _server(serve, monkeypatch, 1 << 50)
    srv.setup_ms = [40.0, 90.0, 60.0]            # longest recent: 90 ms
    srv.submit(r0)
    srv.submit(r1)
    assert srv.admit(until=time.perf_counter() + 0.05) == []
    assert srv.deferred == 1 and len(srv.pending) == 2
    assert srv.admit(until=time.perf_counter() + 10.0) == [0, 1]
    assert len(srv.setup_ms) == 5 and all(t >= 0.0 for t in srv.setup_ms[3:])
    r2 = _req(serve, 2, 4, 122, 1)
    srv.submit(r2)
    assert srv.admit() == [2]                    # no arrival clock: no limit
