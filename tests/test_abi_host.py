"""CPU-side checks of the C ABI: the library builds, loads, exports every
entry point include/lp.h declares, and its host-only calls validate arguments.
No CUDA call is made here (no GPU in this environment)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1612_06592_gb300 import build
    build()
    from paper_1612_06592_gb300 import lp
    return lp


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = declared_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib._lib, n), n
        assert n in lib.SIGNATURES, n


def test_struct_layouts(lib):
    assert ctypes.sizeof(lib.lp_trigger) == 32
    assert lib.TRIGGER_DTYPE.itemsize == 32
    assert ctypes.sizeof(lib.lp_config) == 96
    assert lib.lp_config.stream_blocks.offset == 88
    assert lib.lp_config.fullrate_dedisp.offset == 92


def _create(lib, *shape):
    h = ctypes.c_void_p()
    st = lib._lib.lp_plan_create(ctypes.byref(h), *shape)
    return st, h


def test_plan_create_validates_shape(lib):
    ok, h = _create(lib, 48, 2, 488, 50, 1, 65536)
    assert ok == lib.LP_OK and h.value
    lib._lib.lp_plan_destroy(h)
    for bad in [(0, 2, 16, 1, 1, 64), (6, 3, 16, 1, 1, 64), (6, 2, 0, 1, 1, 64),
                (6, 2, 16, 0, 1, 64), (6, 2, 16, 1, 0, 64), (6, 2, 16, 1, 1, 8),
                (6, 2, 16, 1, 1, 100), (65, 2, 16, 1, 1, 64)]:
        st, h = _create(lib, *bad)
        assert st == lib.LP_ERR_ARG and not h.value, bad


def test_configure_validates_and_sizes_workspace(lib):
    st, h = _create(lib, 6, 2, 16, 1, 1, 4096)
    assert st == lib.LP_OK
    c = lib.config_default()
    c.first_bin = 154
    c.input_dtype = lib.LP_INPUT_INT16
    assert lib._lib.lp_plan_configure(h, ctypes.byref(c)) == lib.LP_OK
    n = ctypes.c_size_t()
    assert lib._lib.lp_plan_workspace_bytes(h, ctypes.byref(n)) == lib.LP_OK
    # beams intermediate dominates: J * K * (F + 16) complex floats
    assert n.value >= 2 * 16 * (4096 + 16) * 8
    bad = lib.config_default()
    bad.first_bin = 500                       # 500 + 16 > 512
    assert lib._lib.lp_plan_configure(h, ctypes.byref(bad)) == lib.LP_ERR_ARG
    bad = lib.config_default()
    bad.first_bin = 154
    bad.precision = lib.LP_PREC_FP16
    bad.input_dtype = lib.LP_INPUT_INT16     # FP16 form: a multiple of 4 stations (6 is not)
    assert lib._lib.lp_plan_configure(h, ctypes.byref(bad)) == lib.LP_ERR_ARG
    assert b"multiple of 4" in lib._lib.lp_last_error(h)
    bad = lib.config_default()
    bad.first_bin = 154
    bad.taps = 8
    assert lib._lib.lp_plan_configure(h, ctypes.byref(bad)) == lib.LP_ERR_ARG
    bad.taps = 16
    bad.frames_per_cta = 12
    assert lib._lib.lp_plan_configure(h, ctypes.byref(bad)) == lib.LP_ERR_ARG
    lib._lib.lp_plan_destroy(h)


def test_calls_before_bind_report_state_errors(lib):
    st, h = _create(lib, 6, 2, 16, 1, 1, 64)
    n = ctypes.c_int64()
    assert lib._lib.lp_get_triggers(h, None, 0, ctypes.byref(n)) == lib.LP_ERR_STATE
    assert lib._lib.lp_process_block(h, None, None) == lib.LP_ERR_STATE
    # workspace size needs a configuration first
    assert lib._lib.lp_plan_workspace_bytes(h, ctypes.byref(ctypes.c_size_t())) == lib.LP_ERR_STATE
    # the autotuners, the configuration list and the LSMR levels need a bound plan
    best = ctypes.c_int32()
    assert lib._lib.lp_plan_gemm_configs(h, None, 0) == -1
    assert lib._lib.lp_plan_set_gemm_config(h, 0) == lib.LP_ERR_STATE
    assert lib._lib.lp_plan_autotune_gemm(h, None, None, ctypes.byref(best), None) == lib.LP_ERR_STATE
    assert lib._lib.lp_plan_autotune(h, None, None, ctypes.byref(best), None) == lib.LP_ERR_STATE
    assert lib._lib.lp_get_lsmr_sigma(h, None) in (lib.LP_ERR_STATE, lib.LP_ERR_ARG)
    out = (ctypes.c_double * 4)()
    assert lib._lib.lp_get_lsmr_sigma(h, out) == lib.LP_ERR_STATE
    assert lib._lib.lp_get_sigma(h, out) == lib.LP_ERR_STATE
    assert lib._lib.lp_plan_autotune_gemm(h, None, None, None, None) == lib.LP_ERR_ARG
    lib._lib.lp_plan_destroy(h)


def test_prebeam_validates_shape_and_groups_before_any_cuda_call(lib):
    import numpy as np
    c = lib._lib
    h = ctypes.c_void_p()
    for bad in [(0, 2, 16, 64, 1, 12, 1), (6, 3, 16, 64, 1, 12, 1), (6, 2, 0, 64, 1, 12, 1),
                (6, 2, 16, 0, 1, 12, 1), (6, 2, 16, 64, 0, 12, 1), (6, 2, 16, 64, 7, 12, 1),
                (6, 2, 16, 64, 2, 0, 1), (6, 2, 16, 64, 2, 500, 1), (6, 2, 16, 64, 2, 12, 3)]:
        assert c.lp_prebeam_create(ctypes.byref(h), *bad) == lib.LP_ERR_ARG, bad
        assert not h.value
    assert c.lp_prebeam_create(ctypes.byref(h), 6, 2, 16, 64, 2, 12, 1) == lib.LP_OK and h.value
    enu = np.zeros((6, 3))
    dirs = np.array([[0.0, 0.0, 1.0], [0.0, 0.6, 0.8]])
    for grp, d in [([0, 0, 0, 0, 0, 0], dirs),            # group 1 empty
                   ([0, 1, 2, 0, 1, 0], dirs),            # group index out of range
                   ([0, 1, -2, 0, 1, 0], dirs),
                   ([0, 1, 0, 1, 0, 1], dirs * 1.01)]:    # not unit vectors
        g = np.array(grp, dtype=np.int32)
        dd = np.ascontiguousarray(d)
        assert c.lp_prebeam_set_groups(h, g.ctypes.data, enu.ctypes.data, dd.ctypes.data,
                                       None) == lib.LP_ERR_ARG
        assert c.lp_prebeam_last_error(h)
    # a valid table still needs a bound workspace (the plan allocates nothing)
    g = np.array([0, 1, 0, 1, 0, 1], dtype=np.int32)
    assert c.lp_prebeam_set_groups(h, g.ctypes.data, enu.ctypes.data, dirs.ctypes.data,
                                   None) == lib.LP_ERR_STATE
    nbytes = ctypes.c_size_t(0)
    assert c.lp_prebeam_workspace_bytes(h, ctypes.byref(nbytes)) == lib.LP_OK
    assert nbytes.value >= 8 * 16 * 6 and nbytes.value % 256 == 0
    assert c.lp_prebeam_bind_workspace(h, None, nbytes.value, None) == lib.LP_ERR_ARG
    assert c.lp_prebeam_bind_workspace(h, 4096 + 16, nbytes.value, None) == lib.LP_ERR_ARG
    assert c.lp_prebeam_bind_workspace(h, 4096, nbytes.value - 1, None) == lib.LP_ERR_OOM
    out = np.zeros((2, 3))
    assert c.lp_prebeam_group_centres(h, out.ctypes.data) == lib.LP_ERR_STATE
    assert c.lp_prebeam_run(h, 16, 16, ctypes.c_float(1.0), None) == lib.LP_ERR_STATE
    n = ctypes.c_int64(5)
    assert c.lp_prebeam_saturated(h, ctypes.byref(n)) == lib.LP_OK and n.value == 0
    c.lp_prebeam_destroy(h)


def _workspace(lib, shape, **fields):
    st, h = _create(lib, *shape)
    assert st == lib.LP_OK
    c = lib.config_default()
    c.first_bin = 100
    for k, v in fields.items():
        setattr(c, k, v)
    st = lib._lib.lp_plan_configure(h, ctypes.byref(c))
    n = ctypes.c_size_t()
    if st == lib.LP_OK:
        assert lib._lib.lp_plan_workspace_bytes(h, ctypes.byref(n)) == lib.LP_OK
    err = lib._lib.lp_last_error(h)
    lib._lib.lp_plan_destroy(h)
    return st, n.value, err


def test_fine_and_lsmr_options_validate_and_size_the_workspace(lib):
    """Host-side checks of the optional paths: their options are validated and
    the workspace grows by exactly their buffers (256-byte aligned pieces)."""
    S, P, K, B, Tr, F = 6, 2, 16, 2, 3, 512
    shape = (S, P, K, B, Tr, F)
    J = B * Tr * P
    st, base, _ = _workspace(lib, shape)
    assert st == lib.LP_OK
    # fine de-dispersion: a second beam-row buffer and 17 taps per (subband, trial)
    st, fine, _ = _workspace(lib, shape, fine_dedisp=1)
    assert st == lib.LP_OK
    rows = J * K * (F + 16) * 8
    taps = K * Tr * 17 * 16
    assert 0 <= fine - base - rows - taps < 3 * 256
    # LSMR: phase-major windowed sums, the series, per-phase noise levels
    st, lsmr, _ = _workspace(lib, shape, inversion=lib.LP_INV_LSMR)
    assert st == lib.LP_OK
    extra = J * 1024 * (F + 16) * 8 + J * 1024 * F * 8 + J * 1024 * (8 + 4)
    assert 0 <= lsmr - base - extra < 5 * 256
    for bad in [dict(fine_dedisp=2), dict(inversion=2),
                dict(inversion=lib.LP_INV_LSMR, lsmr_iters=0),
                dict(inversion=lib.LP_INV_LSMR, lsmr_iters=1001),
                dict(fine_dedisp=1, precision=lib.LP_PREC_FP16, chunk_frames=2048)]:
        st, _, err = _workspace(lib, (8, 1, 4, 1, 1, 4096), **bad)
        assert st == lib.LP_ERR_ARG, bad
        assert err
    # LSMR windows need block_len a multiple of 256
    st, _, err = _workspace(lib, (S, P, K, B, Tr, 264), inversion=lib.LP_INV_LSMR)
    assert st == lib.LP_ERR_ARG and b"256" in err
    st, _, _ = _workspace(lib, (8, 1, 4, 1, 1, 4096), inversion=lib.LP_INV_LSMR,
                          precision=lib.LP_PREC_FP16, chunk_frames=2048)
    assert st == lib.LP_ERR_ARG


def test_fullrate_options_validate_and_size_the_workspace(lib):
    """Full-rate de-dispersion: the series rows (2048 history samples, then the
    block) per stream, the taps' spectrum per trial, the
    FFT twiddles and the FP64 set-up scratch; refused with chunks, the fine
    filter and streaming blocks."""
    S, P, K, B, Tr, F = 6, 2, 16, 2, 3, 512
    shape = (S, P, K, B, Tr, F)
    J = B * Tr * P
    st, base, _ = _workspace(lib, shape)
    assert st == lib.LP_OK
    st, full, _ = _workspace(lib, shape, fullrate_dedisp=1)
    assert st == lib.LP_OK
    extra = (J * (2048 + F * 1024) * 8 + Tr * 8192 * 8 + (16 * 512 + 16 * 32) * 8
             + 2048 * 16 + 2 * 8192 * 16)
    assert 0 <= full - base - extra < 7 * 256
    st, _, _ = _workspace(lib, shape, fullrate_dedisp=1, inversion=lib.LP_INV_LSMR)
    assert st == lib.LP_OK
    for bad in [dict(fullrate_dedisp=2), dict(fullrate_dedisp=1, fine_dedisp=1),
                dict(fullrate_dedisp=1, precision=lib.LP_PREC_FP16, chunk_frames=2048),
                dict(fullrate_dedisp=1, host_input=1, stream_blocks=1)]:
        st, _, err = _workspace(lib, (8, 1, 4, 1, 1, 4096), **bad)
        assert st == lib.LP_ERR_ARG, bad
        assert err


def test_launch_counts_of_the_paths(lib):
    """lp_launches_per_block is host arithmetic: 4 kernels for a device block,
    one more with the fine filter, six with the LSMR inversion, two more with
    the full-rate filter (after the LSMR inversion too)."""
    for fields, want in [({}, 4), ({"fine_dedisp": 1}, 5),
                         ({"inversion": lib.LP_INV_LSMR}, 6),
                         ({"inversion": lib.LP_INV_LSMR, "fine_dedisp": 1}, 7),
                         ({"fullrate_dedisp": 1}, 6),
                         ({"inversion": lib.LP_INV_LSMR, "fullrate_dedisp": 1}, 8)]:
        st, h = _create(lib, 6, 2, 16, 2, 1, 512)
        c = lib.config_default()
        c.first_bin = 100
        for k, v in fields.items():
            setattr(c, k, v)
        assert lib._lib.lp_plan_configure(h, ctypes.byref(c)) == lib.LP_OK
        assert lib._lib.lp_launches_per_block(h) == want, fields
        lib._lib.lp_plan_destroy(h)


def test_stream_blocks_configuration_is_checked(lib):
    c = lib._lib
    st, h = _create(lib, 4, 2, 8, 2, 1, 256)
    cfg = lib.config_default()
    assert cfg.stream_blocks == 0
    for bad in (dict(stream_blocks=2), dict(stream_blocks=1, use_graph=1)):
        k = lib.config_default()
        for f, v in bad.items():
            setattr(k, f, v)
        assert c.lp_plan_configure(h, ctypes.byref(k)) == lib.LP_ERR_ARG, bad
    k = lib.config_default()
    k.stream_blocks = 1
    k.host_input = 1
    assert c.lp_plan_configure(h, ctypes.byref(k)) == lib.LP_OK
    # two staging buffers and two trigger lists
    n2 = ctypes.c_size_t()
    assert c.lp_plan_workspace_bytes(h, ctypes.byref(n2)) == lib.LP_OK
    c.lp_plan_destroy(h)
    st, h = _create(lib, 4, 2, 8, 2, 1, 256)
    k.stream_blocks = 0
    assert c.lp_plan_configure(h, ctypes.byref(k)) == lib.LP_OK
    n1 = ctypes.c_size_t()
    assert c.lp_plan_workspace_bytes(h, ctypes.byref(n1)) == lib.LP_OK
    one_block = 2 * 8 * 256 * 4 * 2
    assert n2.value - n1.value >= one_block + 32 * k.trigger_cap
    n = ctypes.c_int64()
    assert c.lp_get_triggers_block(h, 0, None, 0, ctypes.byref(n)) == lib.LP_ERR_STATE
    c.lp_plan_destroy(h)
