"""Streaming request loop: continuous batching of pipeline sessions on one GPU.

A station stream (48 stations x 2 pols x 488 subbands, complex int8) delivers
one block of 65536 frames every 0.336 s.  Requests subscribe to it with their
own shape: a subset of the 50 beams, a contiguous range of 122..488 subbands,
1..4 STEC trials, for a number of blocks.  Each admitted request is a session:
one plan of the C ABI with its own workspace (synthesis history and running
noise level stay on the device between blocks) and its own CUDA stream.

Per block: the block is copied once from pinned host memory into a device
buffer shared by all sessions; every active session launches its whole
pipeline on its stream against its subband range of that buffer (a strided
view, no copy), so sessions overlap on the device; each session's triggers
come back to the host.  Requests that arrive wait in a queue and are admitted
at a block boundary as soon as their workspace fits in the HBM budget next to
the sessions already running; finished sessions free theirs.

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


# Device time of one session per block, ms, on GB300 (FP16 form), measured
# alone: the synthesis costs ~0.30 ms per stream of 65536 frames whatever the
# subband count (the inverse DFT is always 1024 points); the beamformer ~7.5 ms
# per 50 beams x 2 pols x 488 subbands.  Sessions sharing the GPU run slower
# than the sum of their lone times suggests (small grids, interference), so
# admission multiplies the sum by a correction learned from the measured block
# times, starting from a conservative value.
MS_PER_STREAM = 0.30
MS_PER_BEAM_POL_SUBBAND = 7.5 / (50 * 2 * 488)
INITIAL_CORRECTION = 2.0


def session_cost_ms(P, K, B, Tr, F):
    scale = F / 65536.0
    return scale * (MS_PER_STREAM * B * Tr * P + MS_PER_BEAM_POL_SUBBAND * B * P * K)


class Server:
    """Continuous-batching loop over one station stream.

    A request is admitted when both its workspace fits in the HBM budget and
    the predicted device time of all sessions per block fits in the time
    budget (a fraction of the block period), so that blocks keep up with the
    realtime stream.
    """

    def __init__(self, stations, pols, n_sub, first_bin, block_len, station_enu, beam_grid,
                 hbm_budget_bytes, precision="fp16", k_sigma=6.0, use_graph=False, device=0,
                 time_budget_ms=None):
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
        return session_cost_ms(self.P, req.nsub, len(req.beams), len(req.tec), self.F)

    def admit(self):
        """Admit queued requests, in arrival order, while memory and time fit."""
        admitted = []
        while self.pending:
            req = self.pending[0]
            need = self._ws(req)
            cost = self._cost(req)
            too_slow = (self.time_budget_ms is not None
                        and self.copy_ms + cost * self.cost_corr > self.time_budget_ms)
            if need > self.budget or too_slow:
                self.pending.popleft()          # can never fit: refuse
                self.log.append(("refused", req.rid, need))
                continue
            if self.used + need > self.budget:
                break                           # wait for memory to free up
            if (self.time_budget_ms is not None and self.active and
                    self.copy_ms + (self.cost_used + cost) * self.cost_corr > self.time_budget_ms):
                break                           # wait for a time slot
            self.pending.popleft()
            stream = self.torch.cuda.Stream(device=self.device)
            plan = lp.Plan(self.S, self.P, req.nsub, len(req.beams), len(req.tec), self.F,
                           input_dtype="int8", precision=self.precision,
                           first_bin=self.fb0 + req.k0, k_sigma=self.k_sigma,
                           use_graph=self.use_graph, stream=stream)
            plan.lp_set_weights(self.enu, self.grid[req.beams], stream=stream)
            plan.lp_set_tec(req.tec, stream=stream)
            self.active[req.rid] = Session(req, plan, stream)
            self.used += need
            self.cost_used += cost
            admitted.append(req.rid)
        return admitted

    def retire(self):
        gone = [rid for rid, s in self.active.items() if s.blocks_done >= s.req.blocks]
        for rid in gone:
            s = self.active.pop(rid)
            s.plan.close()
            self.used -= self._ws(s.req)
            self.cost_used -= self._cost(s.req)
        return gone

    # -- one block -----------------------------------------------------------
    def run_block(self, host_block=None):
        """Launch every active session on the resident block; returns when all
        triggers are on the host.  host_block: pinned uint8/int8 tensor to copy
        in first (the block's arrival), or None if the buffer is already filled."""
        torch = self.torch
        ready = torch.cuda.Event(enable_timing=True)
        start = torch.cuda.Event(enable_timing=True)
        if host_block is not None:
            with torch.cuda.stream(self.copy_stream):
                start.record(self.copy_stream)
                self.block_dev.copy_(host_block.view(torch.int8), non_blocking=True)
                ready.record(self.copy_stream)
        else:
            start.record(torch.cuda.current_stream(self.device))
            ready.record(torch.cuda.current_stream(self.device))
        pol_stride = self.n_sub * self.F * self.S           # complex samples
        for s in self.active.values():
            s.stream.wait_event(ready)
            off = s.req.k0 * self.F * self.S * 2                 # bytes (complex int8)
            s.plan.lp_process_block_strided(self.block_dev[off:], pol_stride, stream=s.stream)
        out = {}
        for rid, s in self.active.items():
            trig, n, _ = s.plan.lp_get_triggers()
            s.blocks_done += 1
            out[rid] = (trig, n)
        ready.synchronize()
        copy = start.elapsed_time(ready) if host_block is not None else 0.0
        self.copy_ms = copy if self.copy_ms == 0.0 else 0.8 * self.copy_ms + 0.2 * copy
        return out

    def observe(self, block_ms):
        """Update the cost correction from the measured time of the last block."""
        if self.cost_used > 0 and block_ms > self.copy_ms:
            r = (block_ms - self.copy_ms) / self.cost_used
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
                 time_budget_ms=args.time_budget * period * 1e3 if args.time_budget > 0 else None)
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
    lat, dev_busy, n_sessions, n_out = [], [], [], 0
    qi = 0
    t0 = time.perf_counter()
    for b in range(args.blocks):
        arrival = t0 + b * period if args.realtime else time.perf_counter()
        if args.realtime:
            dt = arrival - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
        while qi < len(reqs) and reqs[qi].arrival <= b:
            srv.submit(reqs[qi])
            qi += 1
        srv.retire()
        srv.admit()
        ts = time.perf_counter()
        out = srv.run_block(hosts[b % len(hosts)])
        te = time.perf_counter()
        srv.observe((te - ts) * 1e3)
        lat.append(te - arrival)
        dev_busy.append(te - ts)
        n_sessions.append(len(out))
        n_out += sum(len(s.req.beams) * len(s.req.tec) * w.pols for s in srv.active.values())
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
        "time_budget_frac": args.time_budget, "cost_correction": srv.cost_corr,
        "ingest_ms": srv.copy_ms,
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
