"""Thin ctypes binding of the C ABI in include/lp.h (argument marshalling only).

Every step of the pipeline runs in the CUDA kernels of liblp.so; this module
only passes pointers and sizes.  Device memory comes from PyTorch (the plan's
workspace is a torch uint8 tensor); streams are torch CUDA streams.  If the
library is missing this module raises at import: there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblp.so")

LP_OK, LP_ERR_ARG, LP_ERR_CUDA, LP_ERR_OOM, LP_ERR_STATE, LP_ERR_OVERFLOW, LP_ERR_TIMEOUT, \
    LP_ERR_BUSY = range(8)
LP_INPUT_INT8, LP_INPUT_INT16 = 1, 2
LP_PREC_FP32, LP_PREC_FP16 = 0, 1
LP_INV_FIR, LP_INV_LSMR = 0, 1
LP_NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024


class lp_config(ctypes.Structure):
    _fields_ = [
        ("input_dtype", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("first_bin", ctypes.c_int32),
        ("taps", ctypes.c_int32),
        ("kaiser_beta", ctypes.c_double),
        ("k_sigma", ctypes.c_double),
        ("sigma_alpha", ctypes.c_double),
        ("nu_ref_hz", ctypes.c_double),
        ("trigger_cap", ctypes.c_int64),
        ("store_timeseries", ctypes.c_int32),
        ("host_input", ctypes.c_int32),
        ("frames_per_cta", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("chunk_frames", ctypes.c_int32),
        ("fine_dedisp", ctypes.c_int32),
        ("inversion", ctypes.c_int32),
        ("lsmr_iters", ctypes.c_int32),
        ("stream_blocks", ctypes.c_int32),
        ("fullrate_dedisp", ctypes.c_int32),
    ]


class lp_trigger(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("beam", ctypes.c_int32),
        ("tec", ctypes.c_int32),
        ("pol", ctypes.c_int32),
        ("stream", ctypes.c_int32),
        ("env", ctypes.c_float),
        ("sigma", ctypes.c_float),
    ]


TRIGGER_DTYPE = np.dtype([("n", "<i8"), ("beam", "<i4"), ("tec", "<i4"), ("pol", "<i4"),
                          ("stream", "<i4"), ("env", "<f4"), ("sigma", "<f4")])

# entry point -> (restype, argtypes); this is also the list of symbols the
# library must export (checked by the CPU tests)
_P = ctypes.c_void_p
SIGNATURES = {
    "lp_config_default": (None, [ctypes.POINTER(lp_config)]),
    "lp_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64]),
    "lp_plan_configure": (ctypes.c_int, [_P, ctypes.POINTER(lp_config)]),
    "lp_plan_workspace_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "lp_plan_bind_workspace": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "lp_set_weights": (ctypes.c_int, [_P, _P, _P, _P]),
    "lp_set_tec": (ctypes.c_int, [_P, _P, _P]),
    "lp_process_block": (ctypes.c_int, [_P, _P, _P]),
    "lp_process_block_strided": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "lp_get_triggers": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "lp_get_triggers_block": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_int64,
                                             ctypes.POINTER(ctypes.c_int64)]),
    "lp_get_timeseries": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "lp_get_beams": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "lp_get_sigma": (ctypes.c_int, [_P, _P]),
    "lp_get_lsmr_sigma": (ctypes.c_int, [_P, _P]),
    "lp_reset_stream": (ctypes.c_int, [_P, _P]),
    "lp_launches_per_block": (ctypes.c_int, [_P]),
    "lp_plan_autotune": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_int32), _P]),
    "lp_plan_gemm_configs": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "lp_plan_set_gemm_config": (ctypes.c_int, [_P, ctypes.c_int]),
    "lp_plan_autotune_gemm": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_int32), _P]),
    "lp_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "lp_profile_read": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int64)]),
    "lp_process_block_noalloc": (ctypes.c_int, [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
        ctypes.POINTER(lp_config), _P, _P, _P, _P, _P, _P, _P, ctypes.c_int64, _P, _P,
        ctypes.c_char_p, ctypes.c_size_t]),
    "lp_plan_destroy": (None, [_P]),
    "lp_prebeam_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int]),
    "lp_prebeam_workspace_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "lp_prebeam_bind_workspace": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "lp_prebeam_set_groups": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "lp_prebeam_group_centres": (ctypes.c_int, [_P, _P]),
    "lp_prebeam_run": (ctypes.c_int, [_P, _P, _P, ctypes.c_float, _P]),
    "lp_prebeam_saturated": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "lp_prebeam_last_error": (ctypes.c_char_p, [_P]),
    "lp_prebeam_destroy": (None, [_P]),
    "lp_group_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int]),
    "lp_group_process_block": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "lp_group_process_block_pol": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.c_int32, _P]),
    "lp_group_size": (ctypes.c_int, [_P]),
    "lp_group_launches_per_block": (ctypes.c_int, [_P]),
    "lp_group_last_error": (ctypes.c_char_p, [_P]),
    "lp_group_destroy": (None, [_P]),
    "lp_last_error": (ctypes.c_char_p, [_P]),
    "lp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}
LP_MAX_GROUP = 32


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


class LPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.lp_status_string(status).decode()}: {msg}")
        self.status = status


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr()


def config_default() -> lp_config:
    c = lp_config()
    _lib.lp_config_default(ctypes.byref(c))
    return c


class Plan:
    """One pipeline instance: shape, configuration, device workspace, state.

    The workspace is a torch uint8 tensor on the current CUDA device; it is
    released with the plan.
    """

    def __init__(self, stations, pols, subbands, beams, tec_trials, block_len, *,
                 input_dtype="int8", precision="fp32", first_bin=12, k_sigma=6.0,
                 sigma_alpha=0.25, nu_ref_hz=0.0, trigger_cap=1 << 20,
                 store_timeseries=False, host_input=False, frames_per_cta=0,
                 kaiser_beta=9.0, use_graph=False, chunk_frames=0, fine_dedisp=False,
                 inversion="fir", lsmr_iters=25, stream_blocks=False, fullrate_dedisp=False,
                 stream=None, workspace=None):
        import torch
        self.shape = (stations, pols, subbands, beams, tec_trials, block_len)
        self._h = _P()
        self._check(_lib.lp_plan_create(ctypes.byref(self._h), stations, pols, subbands, beams,
                                        tec_trials, block_len), "lp_plan_create")
        c = config_default()
        c.input_dtype = LP_INPUT_INT8 if input_dtype == "int8" else LP_INPUT_INT16
        c.precision = LP_PREC_FP16 if precision == "fp16" else LP_PREC_FP32
        c.first_bin = first_bin
        c.k_sigma = k_sigma
        c.sigma_alpha = sigma_alpha
        c.nu_ref_hz = nu_ref_hz
        c.trigger_cap = trigger_cap
        c.store_timeseries = int(bool(store_timeseries))
        c.host_input = int(bool(host_input))
        c.frames_per_cta = frames_per_cta
        c.kaiser_beta = kaiser_beta
        c.use_graph = int(bool(use_graph))
        c.chunk_frames = int(chunk_frames)
        c.fine_dedisp = int(bool(fine_dedisp))
        c.inversion = LP_INV_LSMR if inversion == "lsmr" else LP_INV_FIR
        c.lsmr_iters = int(lsmr_iters)
        c.stream_blocks = int(bool(stream_blocks))
        c.fullrate_dedisp = int(bool(fullrate_dedisp))
        self.config = c
        self._check(_lib.lp_plan_configure(self._h, ctypes.byref(c)), "lp_plan_configure")
        nbytes = ctypes.c_size_t()
        self._check(_lib.lp_plan_workspace_bytes(self._h, ctypes.byref(nbytes)), "workspace_bytes")
        self.workspace_bytes = nbytes.value
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        self._check(_lib.lp_plan_bind_workspace(self._h, workspace.data_ptr(), workspace.numel(),
                                                _stream_ptr(stream)), "bind_workspace")
        self.blocks = 0       # blocks processed since bind or the last reset (block numbers)

    # -- helpers ------------------------------------------------------------
    def _check(self, st, what):
        if st != LP_OK:
            msg = _lib.lp_last_error(self._h).decode() if self._h else ""
            raise LPError(st, f"{what}: {msg}")

    @property
    def n_streams(self):
        _, P, _, B, Tr, _ = self.shape
        return B * Tr * P

    # -- the C entry points, same names -------------------------------------
    def lp_set_weights(self, station_enu, beam_dir, stream=None):
        enu = np.ascontiguousarray(station_enu, dtype=np.float64)
        dirs = np.ascontiguousarray(beam_dir, dtype=np.float64)
        S, _, _, B, _, _ = self.shape
        if enu.shape != (S, 3) or dirs.shape != (B, 3):
            raise ValueError("station_enu must be [S,3] and beam_dir [B,3]")
        self._check(_lib.lp_set_weights(self._h, _ptr(enu), _ptr(dirs), _stream_ptr(stream)),
                    "lp_set_weights")

    def lp_set_tec(self, tec, stream=None):
        t = np.ascontiguousarray(tec, dtype=np.float64)
        if t.shape != (self.shape[4],):
            raise ValueError("tec must have one value per trial")
        self._check(_lib.lp_set_tec(self._h, _ptr(t), _stream_ptr(stream)), "lp_set_tec")

    def lp_process_block(self, x, stream=None):
        """x: torch tensor (device) or numpy array (host) [P, K, F, S, 2] int8/int16."""
        S, P, K, B, Tr, F = self.shape
        shape = tuple(x.shape)
        if shape != (P, K, F, S, 2):
            raise ValueError(f"block shape {shape} != {(P, K, F, S, 2)}")
        self.blocks += 1
        self._check(_lib.lp_process_block(self._h, _ptr(x), _stream_ptr(stream)),
                    "lp_process_block")

    def lp_process_block_strided(self, x, pol_stride, stream=None):
        """x: tensor whose data_ptr is pol 0 / subband 0 of the view; pol_stride in
        complex samples."""
        self.blocks += 1
        self._check(_lib.lp_process_block_strided(self._h, _ptr(x), int(pol_stride),
                                                  _stream_ptr(stream)), "lp_process_block_strided")

    def lp_get_triggers(self, cap=None):
        n = ctypes.c_int64()
        if cap is None:
            self._check_overflow_ok(_lib.lp_get_triggers(self._h, None, 0, ctypes.byref(n)))
            cap = n.value
        out = np.zeros(max(cap, 1), dtype=TRIGGER_DTYPE)
        st = _lib.lp_get_triggers(self._h, out.ctypes.data, cap, ctypes.byref(n))
        if st not in (LP_OK, LP_ERR_OVERFLOW):
            self._check(st, "lp_get_triggers")
        return out[:min(cap, n.value)], n.value, st

    def lp_get_triggers_block(self, block, cap=None):
        """Triggers of one of the last two processed blocks (0-based block count);
        with stream_blocks the next block may still be running."""
        n = ctypes.c_int64()
        if cap is None:
            self._check_overflow_ok(_lib.lp_get_triggers_block(self._h, int(block), None, 0,
                                                               ctypes.byref(n)))
            cap = n.value
        out = np.zeros(max(cap, 1), dtype=TRIGGER_DTYPE)
        st = _lib.lp_get_triggers_block(self._h, int(block), out.ctypes.data, cap,
                                        ctypes.byref(n))
        if st not in (LP_OK, LP_ERR_OVERFLOW):
            self._check(st, "lp_get_triggers_block")
        return out[:min(cap, n.value)], n.value, st

    def _check_overflow_ok(self, st):
        if st not in (LP_OK, LP_ERR_OVERFLOW):
            self._check(st, "lp_get_triggers")

    def lp_get_timeseries(self, beam, tec, pol):
        F = self.shape[5]
        out = np.empty(F * 1024, dtype=np.float32)
        self._check(_lib.lp_get_timeseries(self._h, beam, tec, pol, out.ctypes.data),
                    "lp_get_timeseries")
        return out

    def lp_get_beams(self, beam, tec, pol):
        K, F = self.shape[2], self.shape[5]
        out = np.empty((K, F, 2), dtype=np.float32)
        self._check(_lib.lp_get_beams(self._h, beam, tec, pol, out.ctypes.data), "lp_get_beams")
        return out[..., 0] + 1j * out[..., 1]

    def lp_get_sigma(self):
        out = np.empty(self.n_streams, dtype=np.float64)
        self._check(_lib.lp_get_sigma(self._h, out.ctypes.data), "lp_get_sigma")
        return out

    def lp_get_lsmr_sigma(self):
        """Per-phase noise levels of the LSMR series, [n_streams, 1024]."""
        out = np.empty((self.n_streams, 1024), dtype=np.float64)
        self._check(_lib.lp_get_lsmr_sigma(self._h, out.ctypes.data), "lp_get_lsmr_sigma")
        return out

    def lp_reset_stream(self, stream=None):
        self._check(_lib.lp_reset_stream(self._h, _stream_ptr(stream)), "lp_reset_stream")
        self.blocks = 0

    def lp_launches_per_block(self):
        return _lib.lp_launches_per_block(self._h)

    def lp_plan_autotune(self, x, stream=None):
        """Process block x while picking the synthesis tiling by timing; returns
        (frames_per_cta, {candidate: ms})."""
        best = ctypes.c_int32()
        ms = np.zeros(7, dtype=np.float64)
        self.blocks += 1
        self._check(_lib.lp_plan_autotune(self._h, _ptr(x), _stream_ptr(stream),
                                          ctypes.byref(best), ms.ctypes.data), "lp_plan_autotune")
        cand = (64, 128, 256, 512, 1024, 2048, 0)       # 0: the balanced tiling
        return best.value, {c: m for c, m in zip(cand, ms.tolist()) if m > 0}

    MAX_GEMM_CONFIGS = 8

    def lp_plan_gemm_configs(self):
        """Beamformer configurations: [(input stages, FP16 stages)] for the FP16
        form, [(beams per pass, 0)] for the FP32 form."""
        desc = np.zeros(2 * self.MAX_GEMM_CONFIGS, dtype=np.int32)
        n = _lib.lp_plan_gemm_configs(self._h, desc.ctypes.data, self.MAX_GEMM_CONFIGS)
        if n < 0:
            raise LPError(LP_ERR_STATE, "lp_plan_gemm_configs: plan not bound")
        return [(int(desc[2 * i]), int(desc[2 * i + 1])) for i in range(n)]

    def lp_plan_set_gemm_config(self, index):
        self._check(_lib.lp_plan_set_gemm_config(self._h, int(index)), "lp_plan_set_gemm_config")

    def lp_plan_autotune_gemm(self, x, stream=None):
        """Process block x while picking the beamformer configuration by timing;
        returns (index, {configuration: ms})."""
        best = ctypes.c_int32()
        ms = np.zeros(self.MAX_GEMM_CONFIGS, dtype=np.float64)
        self.blocks += 1
        self._check(_lib.lp_plan_autotune_gemm(self._h, _ptr(x), _stream_ptr(stream),
                                               ctypes.byref(best), ms.ctypes.data),
                    "lp_plan_autotune_gemm")
        cfgs = self.lp_plan_gemm_configs()
        return best.value, {c: m for c, m in zip(cfgs, ms.tolist()) if m > 0}

    STAGES = ("h2d", "beamform", "sigma", "synth", "shift", "fine", "fullrate")

    def lp_profile_enable(self, enable=True):
        self._check(_lib.lp_profile_enable(self._h, int(bool(enable))), "lp_profile_enable")

    def lp_profile_read(self):
        """{stage: total ms} over the blocks recorded since the last read, and their count."""
        ms = np.zeros(len(self.STAGES), dtype=np.float64)
        n = ctypes.c_int64()
        self._check(_lib.lp_profile_read(self._h, ms.ctypes.data, ctypes.byref(n)), "lp_profile_read")
        return dict(zip(self.STAGES, ms.tolist())), n.value

    def close(self):
        if self._h:
            _lib.lp_plan_destroy(self._h)
            self._h = _P()
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Plans whose blocks run in shared launches (lp_group): one beamformer,
    noise-level, synthesis and history-shift launch per block for all of them.
    The plans stay the caller's and must outlive the group."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (_P * len(self.plans))(*[p._h for p in self.plans])
        self._h = _P()
        st = _lib.lp_group_create(ctypes.byref(self._h), arr, len(self.plans))
        if st != LP_OK:
            raise LPError(st, "lp_group_create: the plans cannot form a group")

    def lp_group_process_block(self, x, subbands, first_bin, stream=None):
        """x: device block [P, subbands, F, S, 2] int8 or int16, the plans' type
        (bins first_bin ...)."""
        st = _lib.lp_group_process_block(self._h, _ptr(x), int(subbands), int(first_bin),
                                          _stream_ptr(stream))
        if st != LP_OK:
            raise LPError(st, "lp_group_process_block: " + _lib.lp_group_last_error(self._h).decode())

    def lp_group_process_block_pol(self, x, subbands, first_bin, pol, stream=None):
        """One polarisation of the block (pol 0, then 1, ...): the same layout and
        results as lp_group_process_block; only polarisation pol's slab is read."""
        st = _lib.lp_group_process_block_pol(self._h, _ptr(x), int(subbands), int(first_bin),
                                             int(pol), _stream_ptr(stream))
        if st != LP_OK:
            raise LPError(st, "lp_group_process_block_pol: " +
                          _lib.lp_group_last_error(self._h).decode())

    def lp_group_launches_per_block(self):
        return _lib.lp_group_launches_per_block(self._h)

    def close(self):
        if self._h:
            _lib.lp_group_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Prebeam:
    """Preliminary beams of station groups (the first stage of two-stage
    beamforming): station block [P, K, F, S, 2] int8/int16 on the device ->
    int16 [P, K, F, G, 2], the input of a Plan with stations = G.  The device
    workspace is a torch uint8 tensor on the current CUDA device."""

    def __init__(self, stations, pols, subbands, block_len, groups, *, first_bin=12,
                 input_dtype="int8", stream=None, workspace=None):
        import torch
        self.shape = (stations, pols, subbands, block_len, groups)
        self._h = _P()
        dt = LP_INPUT_INT8 if input_dtype == "int8" else LP_INPUT_INT16
        st = _lib.lp_prebeam_create(ctypes.byref(self._h), stations, pols, subbands, block_len,
                                    groups, first_bin, dt)
        if st != LP_OK:
            raise LPError(st, "lp_prebeam_create: shape out of range")
        nbytes = ctypes.c_size_t()
        self._check(_lib.lp_prebeam_workspace_bytes(self._h, ctypes.byref(nbytes)),
                    "lp_prebeam_workspace_bytes")
        if workspace is None:
            workspace = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        self._check(_lib.lp_prebeam_bind_workspace(self._h, workspace.data_ptr(),
                                                   workspace.numel(), _stream_ptr(stream)),
                    "lp_prebeam_bind_workspace")

    def _check(self, st, what):
        if st != LP_OK:
            msg = _lib.lp_prebeam_last_error(self._h).decode() if self._h else ""
            raise LPError(st, f"{what}: {msg}")

    def lp_prebeam_set_groups(self, group_of_station, station_enu, group_dir, stream=None):
        S, G = self.shape[0], self.shape[4]
        grp = np.ascontiguousarray(group_of_station, dtype=np.int32)
        enu = np.ascontiguousarray(station_enu, dtype=np.float64)
        gd = np.ascontiguousarray(group_dir, dtype=np.float64)
        if grp.shape != (S,) or enu.shape != (S, 3) or gd.shape != (G, 3):
            raise ValueError("group_of_station must be [S], station_enu [S,3], group_dir [G,3]")
        self._check(_lib.lp_prebeam_set_groups(self._h, grp.ctypes.data, enu.ctypes.data,
                                               gd.ctypes.data, _stream_ptr(stream)),
                    "lp_prebeam_set_groups")

    def lp_prebeam_group_centres(self):
        out = np.zeros((self.shape[4], 3), dtype=np.float64)
        self._check(_lib.lp_prebeam_group_centres(self._h, out.ctypes.data),
                    "lp_prebeam_group_centres")
        return out

    def lp_prebeam_run(self, x, y, scale, stream=None):
        S, P, K, F, G = self.shape
        if tuple(x.shape) != (P, K, F, S, 2) or tuple(y.shape) != (P, K, F, G, 2):
            raise ValueError(f"x must be {(P, K, F, S, 2)} and y {(P, K, F, G, 2)}")
        self._check(_lib.lp_prebeam_run(self._h, _ptr(x), _ptr(y), float(scale),
                                        _stream_ptr(stream)), "lp_prebeam_run")

    def lp_prebeam_saturated(self):
        n = ctypes.c_int64()
        self._check(_lib.lp_prebeam_saturated(self._h, ctypes.byref(n)), "lp_prebeam_saturated")
        return n.value

    def close(self):
        if self._h:
            _lib.lp_prebeam_destroy(self._h)
            self._h = _P()
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
