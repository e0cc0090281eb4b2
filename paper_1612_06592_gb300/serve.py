"""Streaming request loop: continuous batching of pipeline sessions on one GPU.

A station stream (48 stations x 2 pols x 488 subbands, complex int8) delivers
one block of 65536 frames every 0.336 s.  Requests subscribe to it with their
own shape: a subset of the 50 beams, a contiguous range of 122..488 subbands,
1..4 STEC trials, for a number of blocks.  Each admitted request is a session:
one plan of the C ABI with its own workspace (synthesis history and running
noise level stay on the device between blocks).

Per block: the block is copied once from pinned host memory into a device
buffer shared by all sessions.  Batched (the default, FP16 form): the active
sessions' plans form a group (lp_group) and each polarisation of the block
runs as four launches -- one beamformer over every session's beams and
subbands, one noise level, one synthesis over every session's streams, one
history shift -- however many sessions there are, as soon as its slab is on
the device (the other slab's copy runs under them); each session reads its
own subband range of the buffer.  Unbatched (FP32 form, or batch=False): every session launches its
own pipeline on its own CUDA stream and sessions overlap on the device.  Each
session's triggers come back to the host.  Requests that arrive wait in a
queue and are admitted at a block boundary as soon as their workspace fits in
the HBM budget next to the sessions already running and their predicted
device time fits the time budget; finished sessions free theirs.  Admission
and retirement run between blocks, after a block's triggers are back: a
request that arrived by then is set up (plan, workspace, tables) there and
joins from the next block.  Set-ups are timed, and one that would not end,
at the longest recently measured, before the next block arrives waits for the
next gap, so that no block waits for another session's set-up.  The cost model
of the prediction is measured at start-up (``Server.calibrate``).

Latency of a block = time from its arrival (the realtime clock of the stream)
to the moment the last session's triggers for it are on the host.  All compute
runs in the kernels of liblp.so; this module only schedules.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import lp

FS_HZ = 200e6
M = 1024


@dataclass
class Request:
    rid: int
    beams: np.ndarray          # indices into the beam grid
    k0: int                    # first subband (offset into the stream's subbands)
    nsub: int
    tec: np.ndarray            # STEC trials (TECU)
    arrival: int               # block at which it arrives
    blocks: int                # how many blocks it stays


@dataclass
class Session:
    req: Request
    plan: object
    stream: object
    done: object = None
    blocks_done: int = 0
    triggers: list = field(default_factory=list)


def workspace_bytes(S, P, K, B, Tr, F, first_bin, precision="fp16"):
    """Device workspace a session of this shape needs (host-only query)."""
    h = ctypes.c_void_p()
    st = lp._lib.lp_plan_create(ctypes.byref(h), S, P, K, B, Tr, F)
    if st != lp.LP_OK:
        raise lp.LPError(st, "lp_plan_create")
    try:
        c = lp.config_default()
        c.first_bin = first_bin
        c.precision = lp.LP_PREC_FP16 if precision == "fp16" else lp.LP_PREC_FP32
        st = lp._lib.lp_plan_configure(h, ctypes.byref(c))
        if st != lp.LP_OK:
            raise lp.LPError(st, lp._lib.lp_last_error(h).decode())
        n = ctypes.c_size_t()
        lp._lib.lp_plan_workspace_bytes(h, ctypes.byref(n))
        return n.value
    finally:
        lp._lib.lp_plan_destroy(h)


def make_requests(seed, n_blocks, n_beams_grid=50, n_sub=488, rate=0.25, min_sub=122,
                  max_trials=4, dur=(4, 64), max_beams=50):
    """Seeded request arrivals: about `rate` per block, uneven shapes."""
    rng = np.random.default_rng(seed)
    reqs = []
    rid = 0
    for b in range(n_blocks):
        for _ in range(rng.poisson(rate) if b else max(1, rng.poisson(4 * rate))):
            nb = int(rng.integers(1, min(max_beams, n_beams_grid) + 1))
            nsub = int(rng.integers(min_sub, n_sub + 1))
            k0 = int(rng.integers(0, n_sub - nsub + 1))
            ntr = int(rng.integers(1, max_trials + 1))
            reqs.append(Request(rid, np.sort(rng.choice(n_beams_grid, nb, replace=False)), k0,
                                nsub, np.sort(rng.uniform(5.0, 40.0, ntr)), b,
                                int(rng.integers(dur[0], dur[1] + 1))))
            rid += 1
    return reqs


class CostModel:
    """Device time of a block of sessions, ms:
        T = (F / 65536) * (c0 + sum_s (c_in * P K_s ceil(B_s / 64)
                                        + c_row * J_s K_s + c_stream * J_s)),
    J_s = B_s Tr_s P the session's streams.  The beamformer reads the session's
    P K_s subband slabs once per 64-beam tile of the tensor-core GEMM and writes
    J_s K_s beam rows; the synthesis costs the same per stream whatever its
    subband count (the inverse DFT is always 1024 points).  The coefficients are
    measured at start-up by Server.calibrate (non-negative least squares over
    timed blocks); until then (and in host-only tests) a prior holds, from one
    GB300 measurement of a whole-band 50-beam session: c_in 1e-3, c_row 4.5e-5,
    c_stream 0.22 ms."""

    def __init__(self, c0=0.0, c_in=1.0e-3, c_row=4.5e-5, c_stream=0.22, measured=False):
        self.c0, self.c_in, self.c_row, self.c_stream = c0, c_in, c_row, c_stream
        self.measured = measured

    @staticmethod
    def features(P, K, B, Tr):
        J = B * Tr * P
        return np.array([P * K * ((B + 63) // 64), J * K, J], dtype=np.float64)

    def session(self, P, K, B, Tr, F):
        f = self.features(P, K, B, Tr)
        return F / 65536.0 * float(np.dot([self.c_in, self.c_row, self.c_stream], f))

    def fixed(self, F):
        return F / 65536.0 * self.c0

    @classmethod
    def fit(cls, samples):
        """Non-negative least squares over samples [(F, [(P, K, B, Tr), ...], ms), ...]."""
        from scipy.optimize import nnls
        rows, y = [], []
        for F, sessions, ms in samples:
            sc = F / 65536.0
            f = sum((cls.features(*x) for x in sessions), np.zeros(3))
            rows.append(sc * np.concatenate([[1.0], f]))
            y.append(ms)
        coef, _ = nnls(np.array(rows), np.array(y, dtype=np.float64))
        return cls(*(float(v) for v in coef), measured=True)

    def as_dict(self):
        return {"c0_ms": self.c0, "ms_per_slab_beam_tile": self.c_in,
                "ms_per_stream_subband_row": self.c_row, "ms_per_stream": self.c_stream,
                "measured": self.measured}


PRIOR = CostModel()
# admission multiplies the modelled time by a correction learned from the
# measured block times, starting from this margin above the calibrated model
INITIAL_CORRECTION = 1.25


def session_cost_ms(P, K, B, Tr, F, model: CostModel = PRIOR):
    return model.session(P, K, B, Tr, F)


class Server:
    """Continuous-batching loop over one station stream.

    A request is admitted when both its workspace fits in the HBM budget and
    the predicted device time of all sessions per block fits in the time
    budget (a fraction of the block period), so that blocks keep up with the
    realtime stream.
    """

    def __init__(self, stations, pols, n_sub, first_bin, block_len, station_enu, beam_grid,
                 hbm_budget_bytes, precision="fp16", k_sigma=6.0, use_graph=False, device=0,
                 time_budget_ms=None, batch=True):
        import torch
        self.torch = torch
        self.S, self.P, self.n_sub, self.fb0, self.F = stations, pols, n_sub, first_bin, block_len
        self.enu = np.asarray(station_enu, dtype=np.float64)
        self.grid = np.asarray(beam_grid, dtype=np.float64)
        self.budget = int(hbm_budget_bytes)
        self.precision = precision
        self.k_sigma = k_sigma
        self.use_graph = use_graph
        self.device = torch.device("cuda", device)
        self.pending = deque()
        self.active: dict[int, Session] = {}
        self.used = 0
        self.ws_of = {}
        self.log = []
        nbytes = pols * n_sub * block_len * stations * 2
        self.block_dev = torch.empty(nbytes, dtype=torch.int8, device=self.device)
        self.copy_stream = torch.cuda.Stream(device=self.device)
        self.time_budget_ms = time_budget_ms
        self.cost_corr = INITIAL_CORRECTION   # measured / modelled session time
        self.cost_used = 0.0
        self.copy_ms = 0.0                    # measured ingest time of a block
        self.model = PRIOR
        # batched: every session's plan joins one group per block (FP16 form)
        self.batch = bool(batch) and precision == "fp16"
        self.stream = torch.cuda.Stream(device=self.device)   # the batched launches
        self.groups = []
        self.group_key = None
        self.launches = []                    # kernel launches per block
        self.calibration = []
        self.setup_ms = []                    # measured set-up time of each admission
        self.deferred = 0                     # admissions put off to a later gap

    def _setup_estimate(self):
        """Set-up time to plan for: the longest of the recent set-ups (0 before
        the first)."""
        return max(self.setup_ms[-8:]) if self.setup_ms else 0.0

    # -- admission ---------------------------------------------------------
    def submit(self, req: Request):
        self.pending.append(req)

    def _ws(self, req):
        key = (len(req.beams), req.nsub, len(req.tec))
        if key not in self.ws_of:
            self.ws_of[key] = workspace_bytes(self.S, self.P, req.nsub, len(req.beams),
                                              len(req.tec), self.F, self.fb0 + req.k0,
                                              self.precision)
        return self.ws_of[key]

    def _cost(self, req):
        return self.model.session(self.P, req.nsub, len(req.beams), len(req.tec), self.F)

    def _fixed(self):
        return self.model.fixed(self.F)

    def _active_cost(self):
        """Modelled time of the active sessions (recomputed, so that admitting and
        retiring never leave a rounding residue)."""
        return sum(self._cost(s.req) for s in self.active.values())

    def admit(self, until=None):
        """Admit queued requests, in arrival order, while memory and time fit.
        until: perf_counter time by which set-up must be done (the next block's
        arrival); a request whose set-up, at the longest recently measured, would
        run past it waits for the next gap between blocks."""
        admitted = []
        while self.pending:
            req = self.pending[0]
            need = self._ws(req)
            cost = self._cost(req)
            too_slow = (self.time_budget_ms is not None
                        and self.copy_ms + (self._fixed() + cost) * self.cost_corr
                        > self.time_budget_ms)
            if need > self.budget or too_slow:
                self.pending.popleft()          # can never fit: refuse
                self.log.append(("refused", req.rid, need))
                continue
            if self.used + need > self.budget:
                break                           # wait for memory to free up
            if (self.time_budget_ms is not None and self.active and
                    self.copy_ms + (self._fixed() + self.cost_used + cost) * self.cost_corr
                    > self.time_budget_ms):
                break                           # wait for a time slot
            if until is not None and time.perf_counter() + self._setup_estimate() * 1e-3 > until:
                self.deferred += 1
                break                           # no time before the next block
            t_set = time.perf_counter()
            self.pending.popleft()
            stream = self.stream if self.batch else self.torch.cuda.Stream(device=self.device)
            plan = lp.Plan(self.S, self.P, req.nsub, len(req.beams), len(req.tec), self.F,
                           input_dtype="int8", precision=self.precision,
                           first_bin=self.fb0 + req.k0, k_sigma=self.k_sigma,
                           use_graph=self.use_graph and not self.batch, stream=stream)
            plan.lp_set_weights(self.enu, self.grid[req.beams], stream=stream)
            plan.lp_set_tec(req.tec, stream=stream)
            stream.synchronize()                # the tables are built before the next block
            self.setup_ms.append((time.perf_counter() - t_set) * 1e3)
            self.active[req.rid] = Session(req, plan, stream)
            self.used += need
            self.cost_used = self._active_cost()
            admitted.append(req.rid)
        return admitted

    def retire(self):
        gone = [rid for rid, s in self.active.items() if s.blocks_done >= s.req.blocks]
        if gone:
            self._drop_groups()
        for rid in gone:
            s = self.active.pop(rid)
            s.plan.close()
            self.used -= self._ws(s.req)
        self.cost_used = self._active_cost()
        return gone

    # -- one block -----------------------------------------------------------
    def run_block(self, host_block=None):
        """Launch every active session on the resident block; returns when all
        triggers are on the host.  host_block: pinned uint8/int8 tensor to copy
        in first (the block's arrival), or None if the buffer is already filled."""
        torch = self.torch
        # one event per polarisation slab: batched launches start on a slab as
        # soon as it is on the device (the next slab's copy runs under them)
        pol_ready = [torch.cuda.Event(enable_timing=True) for _ in range(self.P)]
        ready = pol_ready[-1]
        start = torch.cuda.Event(enable_timing=True)
        if host_block is not None:
            hb = host_block.view(torch.int8)
            n = self.block_dev.numel() // self.P
            with torch.cuda.stream(self.copy_stream):
                start.record(self.copy_stream)
                for pol in range(self.P):
                    self.block_dev[pol * n:(pol + 1) * n].copy_(hb[pol * n:(pol + 1) * n],
                                                                non_blocking=True)
                    pol_ready[pol].record(self.copy_stream)
        else:
            start.record(torch.cuda.current_stream(self.device))
            for ev in pol_ready:
                ev.record(torch.cuda.current_stream(self.device))
        if self.batch:
            self._run_groups(pol_ready)
        else:
            pol_stride = self.n_sub * self.F * self.S           # complex samples
            for s in self.active.values():
                s.stream.wait_event(ready)
                off = s.req.k0 * self.F * self.S * 2                 # bytes (complex int8)
                s.plan.lp_process_block_strided(self.block_dev[off:], pol_stride,
                                                stream=s.stream)
            self.launches.append(sum(s.plan.lp_launches_per_block()
                                     for s in self.active.values()))
        out = {}
        for rid, s in self.active.items():
            trig, n, _ = s.plan.lp_get_triggers()
            s.blocks_done += 1
            out[rid] = (trig, n)
        ready.synchronize()
        copy = start.elapsed_time(ready) if host_block is not None else 0.0
        self.copy_ms = copy if self.copy_ms == 0.0 else 0.8 * self.copy_ms + 0.2 * copy
        return out

    # -- batched launches ------------------------------------------------------
    def _drop_groups(self):
        for g in self.groups:
            g.close()
        self.groups, self.group_key = [], None

    def _run_groups(self, pol_ready):
        """One block for every active session in shared launches: the sessions'
        plans (in admission order) form groups of at most LP_MAX_GROUP plans,
        run one polarisation at a time, each once its slab has arrived."""
        key = tuple(self.active)
        if key != self.group_key:
            self._drop_groups()
            plans = [s.plan for s in self.active.values()]
            self.groups = [lp.Group(plans[i:i + lp.LP_MAX_GROUP])
                           for i in range(0, len(plans), lp.LP_MAX_GROUP)]
            self.group_key = key
        for pol, ev in enumerate(pol_ready):
            self.stream.wait_event(ev)
            for g in self.groups:
                g.lp_group_process_block_pol(self.block_dev, self.n_sub, self.fb0, pol,
                                             stream=self.stream)
        self.launches.append(self.P * sum(g.lp_group_launches_per_block() for g in self.groups))

    def calibrate(self, shapes=((1, 122, 1), (8, 488, 2), (16, 244, 1), (40, 488, 1),
                                (2, 488, 4), (24, 160, 3)), reps=3):
        """Measure the cost model on this GPU: time one block of sessions of the
        given (beams, subbands, trials) shapes -- each alone, then all together
        -- in the launch form the server uses, and fit CostModel by least
        squares.  Runs before any request is admitted; the results of these
        blocks are discarded."""
        torch = self.torch
        if self.active:
            raise RuntimeError("calibrate before admitting requests")
        # seeded noise in the block buffer (a realistic trigger rate)
        g = torch.Generator(device=self.device)
        g.manual_seed(17)
        self.block_dev.copy_(torch.randint(-12, 13, self.block_dev.shape, generator=g,
                                           device=self.device, dtype=torch.int8))
        plans, shp = [], []
        stream = self.stream
        for (nb, ns, nt) in shapes:
            t_set = time.perf_counter()
            plan = lp.Plan(self.S, self.P, ns, nb, nt, self.F, input_dtype="int8",
                           precision=self.precision, first_bin=self.fb0, k_sigma=self.k_sigma,
                           stream=stream)
            plan.lp_set_weights(self.enu, self.grid[:nb], stream=stream)
            plan.lp_set_tec(np.linspace(10.0, 30.0, nt), stream=stream)
            stream.synchronize()
            self.setup_ms.append((time.perf_counter() - t_set) * 1e3)
            plans.append(plan)
            shp.append((self.P, ns, nb, nt))
        combos = [[i] for i in range(len(plans))] + [list(range(len(plans)))]
        samples = []
        pol_stride = self.n_sub * self.F * self.S
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for combo in combos:
            grp = lp.Group([plans[i] for i in combo]) if self.batch else None

            def one_block():
                if grp is not None:
                    grp.lp_group_process_block(self.block_dev, self.n_sub, self.fb0,
                                               stream=stream)
                else:
                    for i in combo:
                        plans[i].lp_process_block_strided(self.block_dev, pol_stride,
                                                          stream=stream)
            one_block()                                   # warm-up
            e0.record(stream)
            for _ in range(reps):
                one_block()
            e1.record(stream)
            e1.synchronize()
            samples.append((self.F, [shp[i] for i in combo], e0.elapsed_time(e1) / reps))
            if grp is not None:
                grp.close()
        for plan in plans:
            plan.close()
        torch.cuda.empty_cache()
        self.model = CostModel.fit(samples)
        self.calibration = [{"sessions": [list(x) for x in ses], "ms": ms}
                            for _, ses, ms in samples]
        return self.model

    def observe(self, block_ms):
        """Update the cost correction from the measured time of the last block."""
        if self.active and self.cost_used > 1e-6 and block_ms > self.copy_ms:
            r = (block_ms - self.copy_ms) / (self._fixed() + self.cost_used)
            self.cost_corr = 0.8 * self.cost_corr + 0.2 * r


def run(args):
    import torch
    import synth
    torch.cuda.set_device(0)
    w = synth.SERVING
    enu, grid, _ = synth.make_geometry(w)
    period = w.block_len * M / FS_HZ
    srv = Server(w.stations, w.pols, w.subbands, w.first_bin, w.block_len, enu, grid,
                 args.budget_gb * 1e9, precision=args.precision, use_graph=args.graph,
                 time_budget_ms=args.time_budget * period * 1e3 if args.time_budget > 0 else None,
                 batch=args.batch)
    srv.calibrate()
    reqs = make_requests(args.seed, args.blocks, max_beams=args.max_beams)
    # a few distinct blocks of station data, reused cyclically (pinned host memory)
    hosts = []
    for i in range(args.distinct_blocks):
        xb = synth.device_noise_block(w, 4000 + i, srv.device)
        h = torch.empty(xb.numel(), dtype=torch.int8, pin_memory=True)
        h.copy_(xb.view(-1))
        hosts.append(h)
        del xb
    torch.cuda.synchronize()
    lat, dev_busy, n_sessions, n_out, late = [], [], [], 0, []
    qi = 0
    # requests that arrived before the first block join it
    while qi < len(reqs) and reqs[qi].arrival <= 0:
        srv.submit(reqs[qi])
        qi += 1
    srv.admit()
    t0 = time.perf_counter()
    for b in range(args.blocks):
        arrival = t0 + b * period if args.realtime else time.perf_counter()
        if args.realtime:
            dt = arrival - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        ts = time.perf_counter()
        out = srv.run_block(hosts[b % len(hosts)])
        te = time.perf_counter()
        srv.observe((te - ts) * 1e3)
        lat.append(te - arrival)
        dev_busy.append(te - ts)
        if te - arrival > period:
            late.append({"block": b, "wait_ms": (ts - arrival) * 1e3,
                         "busy_ms": (te - ts) * 1e3, "sessions": len(out)})
        n_sessions.append(len(out))
        n_out += sum(len(s.req.beams) * len(s.req.tec) * w.pols for s in srv.active.values())
        # between blocks, off the latency path: finished sessions leave, and the
        # requests that have arrived by now are set up (plan, workspace, tables)
        # to join from the next block
        while qi < len(reqs) and reqs[qi].arrival <= b:
            srv.submit(reqs[qi])
            qi += 1
        srv.retire()
        srv.admit(until=t0 + (b + 1) * period if args.realtime else None)
    wall = time.perf_counter() - t0
    lat_ms = np.array(lat) * 1e3
    res = {
        "blocks": args.blocks, "realtime_arrivals": bool(args.realtime),
        "block_seconds": period, "p50_ms": float(np.percentile(lat_ms, 50)),
        "p99_ms": float(np.percentile(lat_ms, 99)), "max_ms": float(lat_ms.max()),
        "deadline_ms": period * 1e3,
        "missed_deadline": int(np.sum(lat_ms > period * 1e3)),
        "sessions_mean": float(np.mean(n_sessions)), "sessions_max": int(np.max(n_sessions)),
        "requests": len(reqs), "refused": sum(1 for e in srv.log if e[0] == "refused"),
        "hbm_budget_gb": args.budget_gb,
        "batched": srv.batch,
        "launches_per_block": {"mean": float(np.mean(srv.launches)),
                               "max": int(np.max(srv.launches))},
        "cost_model": srv.model.as_dict(), "calibration": srv.calibration,
        "time_budget_frac": args.time_budget, "cost_correction": srv.cost_corr,
        "ingest_ms": srv.copy_ms,
        "setup_ms": {"mean": float(np.mean(srv.setup_ms)) if srv.setup_ms else 0.0,
                     "max": float(np.max(srv.setup_ms)) if srv.setup_ms else 0.0,
                     "n": len(srv.setup_ms)},
        "admissions_deferred": srv.deferred,
        "late_blocks": late[:20],
        "busy_ms_p50": float(np.percentile(np.array(dev_busy) * 1e3, 50)),
        "busy_ms_max": float(np.max(dev_busy) * 1e3),
        "sustained_blocks_per_s": args.blocks / wall,
        "stream_samples_per_s": n_out * w.block_len * M / wall,
        "station_samples_per_s": args.blocks * w.pols * w.subbands * w.block_len * w.stations / wall,
    }
    return res


def build_parser():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--blocks", type=int, default=1000)
    ap.add_argument("--budget-gb", type=float, default=160.0)
    ap.add_argument("--precision", default="fp16", choices=["fp16", "fp32"])
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--max-beams", type=int, default=50)
    ap.add_argument("--distinct-blocks", type=int, default=2)
    ap.add_argument("--graph", action="store_true")
    ap.add_argument("--batch", action=argparse.BooleanOptionalAction, default=True,
                    help="sessions' blocks in shared launches (lp_group; FP16 form)")
    ap.add_argument("--realtime", action=argparse.BooleanOptionalAction, default=True)
    ap.add_argument("--time-budget", type=float, default=0.75,
                    help="admit while the predicted block time stays below this fraction "
                         "of the block period (0: memory budget only)")
    return ap


def main(argv=None):
    args = build_parser().parse_args(argv)
    print(json.dumps(run(args)))


if __name__ == "__main__":
    main()
