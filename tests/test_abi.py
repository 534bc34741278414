"""The CUDA library builds for sm_103a, loads, and exports every entry point
that include/lr.h declares.  No compute call is made (no GPU needed)."""
import ctypes

import pytest

from paper_2208_13409_gb300 import lr, problems as P


def test_header_declares_the_boundary():
    names = lr.declared_symbols()
    for core in ("lr_create", "lr_set_materials", "lr_init", "lr_step", "lr_run", "lr_get_fields",
                 "lr_destroy", "lr_last_error"):
        assert core in names


def test_library_exports_every_declared_symbol():
    L = lr.load()
    missing = [n for n in lr.declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_host_side_validation_without_gpu():
    L = lr.load()
    cfg = lr.make_config(P.sod(nx=16))
    nbytes = ctypes.c_size_t()
    assert L.lr_workspace_bytes(ctypes.byref(cfg), ctypes.byref(nbytes)) == lr.OK
    assert nbytes.value > 16 * 4 * 8
    bad = lr.make_config(P.sod(nx=16))
    bad.nx = 1
    h = ctypes.c_void_p()
    assert L.lr_create(ctypes.byref(bad), ctypes.byref(h)) == lr.ERR_ARG and not h.value
    bad = lr.make_config(P.sod(nx=16))
    bad.nmat = 4
    assert L.lr_workspace_bytes(ctypes.byref(bad), ctypes.byref(nbytes)) == lr.ERR_ARG
    bad = lr.make_config(P.sod(nx=16))
    bad.bc[0] = lr.BC_PERIODIC  # xlo != xhi
    assert L.lr_workspace_bytes(ctypes.byref(bad), ctypes.byref(nbytes)) == lr.ERR_ARG
    for lanes, ok in ((0, True), (1, True), (4, True), (8, True), (3, False), (16, False), (-1, False)):
        cfg = lr.make_config(P.sod(nx=16), mixed_lanes=lanes)
        rc = L.lr_workspace_bytes(ctypes.byref(cfg), ctypes.byref(nbytes))
        assert rc == (lr.OK if ok else lr.ERR_ARG), lanes
    assert L.lr_last_error(None) == b"null context"


def test_batch_host_side_validation_without_gpu():
    L = lr.load()
    cfg = lr.BatchConfig()
    L.lr_batch_config_default(ctypes.byref(cfg))
    assert (cfg.precision, cfg.nmat_max, cfg.capacity_members) == (lr.FP64, 3, 16)
    n = ctypes.c_size_t()
    assert L.lr_batch_workspace_bytes(ctypes.byref(cfg), ctypes.byref(n)) == lr.OK
    u = ctypes.c_size_t()
    assert L.lr_batch_unit_bytes(ctypes.byref(cfg), ctypes.byref(u)) == lr.OK
    # the pool dominates: workspace ~ units x unit bytes (+ staging and scratch)
    assert cfg.capacity_units * u.value <= n.value <= 2 * cfg.capacity_units * u.value + (64 << 20) * 8
    # FP32 halves the real arrays; fewer material planes shrink the unit
    f32 = lr.BatchConfig.from_buffer_copy(cfg)
    f32.precision = lr.FP32
    u32 = ctypes.c_size_t()
    assert L.lr_batch_unit_bytes(ctypes.byref(f32), ctypes.byref(u32)) == lr.OK and u32.value < u.value
    for field, bad in (("nmat_max", 4), ("nmat_max", 0), ("capacity_members", 0), ("capacity_units", 3),
                       ("precision", 7), ("max_member_cells", 1)):
        c = lr.BatchConfig.from_buffer_copy(cfg)
        setattr(c, field, bad)
        assert L.lr_batch_workspace_bytes(ctypes.byref(c), ctypes.byref(n)) == lr.ERR_ARG, field
    assert L.lr_batch_last_error(None) == b"null batch"


def test_arith_check_and_async_reads_validate_without_gpu():
    L = lr.load()
    vp = ctypes.c_void_p
    # unknown operation, or missing buffers: refused before any device call
    assert L.lr_arith_check(7, vp(), vp(), vp(), 4, vp()) == lr.ERR_ARG
    assert L.lr_arith_check(lr.ARITH_DIV, vp(), vp(), vp(), 4, vp()) == lr.ERR_ARG
    assert L.lr_arith_check(lr.ARITH_SQRT, vp(), vp(), vp(), 0, vp()) == lr.OK  # nothing to do
    buf = (ctypes.c_double * 4)()
    assert L.lr_get_fields_async(None, lr.F_K, buf, 4) == lr.ERR_ARG
