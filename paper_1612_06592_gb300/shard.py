"""Beam sharding across GPUs (the multi-GPU form of the pipeline).

Sec. 4 of the paper distributes all station data to every processing node
(broadcast, Figs. 2-3) and divides the ~50 beams that cover the Moon among the
nodes.  Streams (beam, STEC trial, polarisation) are independent once the
beams are formed, and every beam needs the whole station block, so the
partition is by beams: rank r of N owns the contiguous beam range
``beam_range(B, N, r)``, receives the full station block (its own host-to-
device copy, or a device copy made by the caller), runs the whole pipeline on
its beams with one plan, and keeps only their triggers.  There is no exchange
in the data path; the trigger lists meet on the host, relabelled to global
beam and stream indices and merged in the ABI's order (beam, tec, pol, n).

The partition and merge are plain host functions (``beam_range``,
``to_global``, ``merge_triggers``, ``gather_triggers``) so that they can be
checked with any per-rank engine; ``BeamShard`` binds them to a GPU plan.
"""

from __future__ import annotations

import numpy as np

TRIGGER_FIELDS = ("n", "beam", "tec", "pol", "stream", "env", "sigma")


def beam_range(n_beams: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous beams [b0, b1) of `rank`: the first n_beams % world ranks take
    one beam more.  Needs 1 <= world <= n_beams (every rank owns a beam)."""
    if not (1 <= world <= n_beams) or not (0 <= rank < world):
        raise ValueError(f"cannot split {n_beams} beams over {world} ranks (rank {rank})")
    base, extra = divmod(n_beams, world)
    b0 = rank * base + min(rank, extra)
    return b0, b0 + base + (1 if rank < extra else 0)


def to_global(trig: np.ndarray, b0: int, tec_trials: int, pols: int) -> np.ndarray:
    """Trigger records of a shard (beam and stream indices local to its plan)
    relabelled to the global beam b0 + b and stream (beam * Tr + tec) * P + pol."""
    out = np.array(trig, copy=True)
    if out.size:
        out["beam"] += b0
        out["stream"] = (out["beam"] * tec_trials + out["tec"]) * pols + out["pol"]
    return out


def merge_triggers(parts) -> np.ndarray:
    """Concatenate the ranks' (global) trigger lists in the ABI's order:
    sorted by (beam, tec, pol, n).  The ranges are disjoint, so no record
    appears twice."""
    parts = [np.asarray(p) for p in parts if p is not None and len(p)]
    if not parts:
        from .lp import TRIGGER_DTYPE
        return np.zeros(0, dtype=TRIGGER_DTYPE)
    allt = np.concatenate(parts)
    order = np.lexsort((allt["n"], allt["pol"], allt["tec"], allt["beam"]))
    return allt[order]


def gather_triggers(local: np.ndarray, group=None, dst: int = 0):
    """Collect every rank's global trigger list on rank `dst` and merge them
    (torch.distributed object gather; works with the gloo and nccl backends).
    Returns the merged list on `dst`, None elsewhere."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    recv = [None] * world if rank == dst else None
    dist.gather_object(local, recv, dst=dst, group=group)
    return merge_triggers(recv) if rank == dst else None


def gather_sigma(local: np.ndarray, group=None, dst: int = 0):
    """Noise levels of every stream in global order (ranks own contiguous
    beams, so their stream ranges are contiguous too) on rank `dst`."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    recv = [None] * world if rank == dst else None
    dist.gather_object(np.asarray(local), recv, dst=dst, group=group)
    return np.concatenate(recv) if rank == dst else None


class BeamShard:
    """One rank's share of a beam-sharded pipeline: an lp.Plan over the rank's
    beams of the full configuration, fed the whole station block."""

    def __init__(self, stations, pols, subbands, beams, tec_trials, block_len, *, rank: int,
                 world: int, **plan_kw):
        from . import lp
        self.b0, self.b1 = beam_range(beams, world, rank)
        self.beams, self.tec_trials, self.pols = beams, tec_trials, pols
        self.plan = lp.Plan(stations, pols, subbands, self.b1 - self.b0, tec_trials, block_len,
                            **plan_kw)

    def lp_set_weights(self, station_enu, beam_dir, stream=None):
        self.plan.lp_set_weights(station_enu, np.asarray(beam_dir)[self.b0:self.b1],
                                 stream=stream)

    def lp_set_tec(self, tec, stream=None):
        self.plan.lp_set_tec(tec, stream=stream)

    def lp_process_block(self, x, stream=None):
        self.plan.lp_process_block(x, stream=stream)

    def lp_get_triggers(self):
        """(global trigger records of this rank's beams, count, status)."""
        trig, n, st = self.plan.lp_get_triggers()
        return to_global(trig, self.b0, self.tec_trials, self.pols), n, st

    def lp_get_sigma(self):
        return self.plan.lp_get_sigma()

    def close(self):
        self.plan.close()
