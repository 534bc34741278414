"""Thin ctypes binding of the C ABI in include/lr.h (argument marshalling
only; every phase of the step runs in the CUDA library).

PyTorch supplies the device memory (one arena tensor per simulation, from
its caching allocator) and the CUDA stream (torch's current stream) when it
is available; the library allocates its own otherwise.  ``load()`` raises if
the library cannot be built or loaded: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import re
import os
from typing import Optional

import numpy as np

from . import build as _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lr.h")
BATCH_HEADER = os.path.join(os.path.dirname(HEADER), "lr_batch.h")
SERVE_HEADER = os.path.join(os.path.dirname(HEADER), "lr_serve.h")

OK, ERR_ARG, ERR_OOM, ERR_NUMERIC, ERR_TIMEOUT, ERR_STATE, ERR_CUDA = 0, -1, -2, -3, -4, -5, -6
BC_REFLECT, BC_PERIODIC = 0, 1
CORNER_UPWIND, CORNER_DIAG = 0, 1
REMAP_DIRECTCF, REMAP_DIRECT, REMAP_AD = 0, 1, 2
FP64, DF64, FP32 = 0, 1, 2
F_K, F_RHO_MAT, F_E_MAT, F_P, F_RHO, F_E, F_UX, F_UY, F_CONS, F_C = range(10)
F_UHX, F_UHY, F_VOL_LAGCF, F_E_LAG, F_FX, F_FY, F_FC, F_MX, F_MY, F_MC, F_Q, F_DT = range(20, 32)
F_CUTS, F_XA, F_YA, F_CA, F_NMIXED = range(32, 37)
ARITH_DIV, ARITH_SQRT = 0, 1


class LrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lr status {status}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("nmat", ctypes.c_int),
        ("cfl", ctypes.c_double), ("a1", ctypes.c_double), ("a2", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("precision", ctypes.c_int), ("face_order", ctypes.c_int), ("corner_recon", ctypes.c_int),
        ("dt_fixed", ctypes.c_double),
        ("mixed_lanes", ctypes.c_int),
        ("remap", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p),
    ]


class BatchConfig(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int), ("nmat_max", ctypes.c_int),
        ("capacity_units", ctypes.c_long), ("capacity_members", ctypes.c_int),
        ("max_member_cells", ctypes.c_long), ("cuda_stream", ctypes.c_void_p),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [("batch", BatchConfig), ("max_chunk_steps", ctypes.c_int), ("max_bypass", ctypes.c_int),
                ("device", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_long), ("admitted", ctypes.c_long), ("completed", ctypes.c_long),
                ("failed", ctypes.c_long), ("pending", ctypes.c_long), ("resident", ctypes.c_long),
                ("cell_updates", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("steps_launched", ctypes.c_long)]


class Material(ctypes.Structure):
    _fields_ = [("eos", ctypes.c_int), ("gamma", ctypes.c_double), ("pi", ctypes.c_double)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def declared_symbols() -> list:
    """Names of the functions declared in include/lr.h, lr_batch.h and lr_serve.h."""
    names = set()
    for h in (HEADER, BATCH_HEADER, SERVE_HEADER):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(lr_[a-z_]+)\s*\(", text))
    return sorted(names)


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library; raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    L.lr_config_default.argtypes = [ctypes.POINTER(Config)]
    L.lr_config_default.restype = None
    L.lr_workspace_bytes.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_size_t)]
    L.lr_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
    L.lr_create_in.argtypes = [ctypes.POINTER(Config), vp, ctypes.c_size_t, ctypes.POINTER(vp)]
    L.lr_set_materials.argtypes = [vp, ctypes.c_int, ctypes.POINTER(Material)]
    L.lr_init.argtypes = [vp, _dp, _dp, _dp, _dp, _dp]
    L.lr_set_prescribed_velocity.argtypes = [vp, _dp, _dp]
    L.lr_step.argtypes = [vp, ctypes.c_double, _dp]
    L.lr_run.argtypes = [vp, ctypes.c_double, ctypes.c_long, ctypes.POINTER(ctypes.c_long), _dp]
    L.lr_sync.argtypes = [vp]
    L.lr_field_size.argtypes = [vp, ctypes.c_int]
    L.lr_field_size.restype = ctypes.c_size_t
    L.lr_get_fields.argtypes = [vp, ctypes.c_int, _dp, ctypes.c_size_t]
    L.lr_get_fields_device.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t]
    L.lr_time.argtypes = [vp, _dp, _dp]
    L.lr_launches_per_step.argtypes = [vp]
    L.lr_launches_per_step.restype = ctypes.c_int
    L.lr_set_profiling.argtypes = [vp, ctypes.c_int]
    L.lr_checkpoint_bytes.argtypes = [vp]
    L.lr_checkpoint_bytes.restype = ctypes.c_size_t
    L.lr_checkpoint_save.argtypes = [vp, vp, ctypes.c_size_t]
    L.lr_checkpoint_save.restype = ctypes.c_int
    L.lr_checkpoint_load.argtypes = [vp, vp, ctypes.c_size_t]
    L.lr_checkpoint_load.restype = ctypes.c_int
    L.lr_set_tiled.argtypes = [vp, ctypes.c_int]
    L.lr_get_tiled.argtypes = [vp]
    L.lr_get_tiled.restype = ctypes.c_int
    L.lr_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_long),
                                  _dp, ctypes.c_int]
    L.lr_kernel_times.restype = ctypes.c_int
    L.lr_destroy.argtypes = [vp]
    L.lr_destroy.restype = None
    L.lr_last_error.argtypes = [vp]
    L.lr_last_error.restype = ctypes.c_char_p
    L.lr_cfl_dt_noalloc.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(Material), vp, vp, vp, vp, vp, vp]
    L.lr_cfl_dt_noalloc.restype = ctypes.c_int
    L.lr_get_fields_async.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]
    L.lr_get_fields_async.restype = ctypes.c_int
    L.lr_arith_check.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_size_t, vp]
    L.lr_arith_check.restype = ctypes.c_int
    L.lr_fp64_fma_probe.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
    L.lr_fp64_fma_probe.restype = ctypes.c_int
    bp = ctypes.POINTER(BatchConfig)
    L.lr_batch_config_default.argtypes = [bp]
    L.lr_batch_config_default.restype = None
    L.lr_batch_workspace_bytes.argtypes = [bp, ctypes.POINTER(ctypes.c_size_t)]
    L.lr_batch_unit_bytes.argtypes = [bp, ctypes.POINTER(ctypes.c_size_t)]
    L.lr_batch_create.argtypes = [bp, ctypes.POINTER(vp)]
    L.lr_batch_destroy.argtypes = [vp]
    L.lr_batch_destroy.restype = None
    L.lr_batch_last_error.argtypes = [vp]
    L.lr_batch_last_error.restype = ctypes.c_char_p
    L.lr_batch_add.argtypes = [vp, ctypes.POINTER(Config), ctypes.POINTER(Material), _dp, _dp, _dp, _dp, _dp,
                               ctypes.c_double, ctypes.c_long, ctypes.POINTER(ctypes.c_int)]
    L.lr_batch_remove.argtypes = [vp, ctypes.c_int]
    L.lr_batch_set_limits.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_long]
    L.lr_batch_step.argtypes = [vp, ctypes.c_int]
    L.lr_batch_sync.argtypes = [vp]
    L.lr_batch_status.argtypes = [vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_int)]
    L.lr_batch_status_all.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_long), ctypes.c_int]
    L.lr_batch_field_size.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.lr_batch_field_size.restype = ctypes.c_size_t
    L.lr_batch_get_fields.argtypes = [vp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_size_t]
    L.lr_batch_autotune.argtypes = [vp, ctypes.c_int]
    L.lr_batch_schedule.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]
    L.lr_batch_launches_per_step.argtypes = [vp]
    L.lr_batch_launches_per_step.restype = ctypes.c_int
    L.lr_batch_set_profiling.argtypes = [vp, ctypes.c_int]
    L.lr_batch_set_persistent.argtypes = [vp, ctypes.c_int]
    L.lr_batch_set_persistent.restype = ctypes.c_int
    L.lr_batch_get_persistent.argtypes = [vp]
    L.lr_batch_get_persistent.restype = ctypes.c_int
    L.lr_batch_test_barrier.argtypes = [vp, ctypes.c_uint, ctypes.c_double]
    L.lr_batch_test_barrier.restype = ctypes.c_int
    L.lr_batch_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_long),
                                        _dp, ctypes.c_int]
    L.lr_batch_kernel_times.restype = ctypes.c_int
    sp = ctypes.POINTER(ServerConfig)
    L.lr_server_config_default.argtypes = [sp]
    L.lr_server_config_default.restype = None
    L.lr_server_create.argtypes = [sp, ctypes.POINTER(vp)]
    L.lr_server_destroy.argtypes = [vp]
    L.lr_server_destroy.restype = None
    L.lr_server_last_error.argtypes = [vp]
    L.lr_server_last_error.restype = ctypes.c_char_p
    L.lr_server_submit.argtypes = [vp, ctypes.POINTER(Config), ctypes.POINTER(Material), _dp, _dp, _dp, _dp, _dp,
                                   ctypes.c_double, ctypes.c_long, ctypes.POINTER(ctypes.c_long)]
    L.lr_server_wait.argtypes = [vp, ctypes.c_long, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
    L.lr_server_drain.argtypes = [vp, ctypes.c_double]
    L.lr_server_info.argtypes = [vp, ctypes.c_long, _dp, _dp, _dp, _dp, ctypes.POINTER(ctypes.c_long)]
    L.lr_server_result_size.argtypes = [vp, ctypes.c_long, ctypes.c_int]
    L.lr_server_result_size.restype = ctypes.c_size_t
    L.lr_server_result.argtypes = [vp, ctypes.c_long, ctypes.c_int, _dp, ctypes.c_size_t]
    L.lr_server_release.argtypes = [vp, ctypes.c_long]
    L.lr_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.lr_server_clock.argtypes = [vp]
    L.lr_server_clock.restype = ctypes.c_double
    for name in ("lr_server_create", "lr_server_submit", "lr_server_wait", "lr_server_drain", "lr_server_info",
                 "lr_server_result", "lr_server_release", "lr_server_get_stats"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("lr_batch_workspace_bytes", "lr_batch_unit_bytes", "lr_batch_create", "lr_batch_add",
                 "lr_batch_remove", "lr_batch_set_limits", "lr_batch_step", "lr_batch_sync", "lr_batch_status", "lr_batch_status_all",
                 "lr_batch_get_fields", "lr_batch_autotune", "lr_batch_schedule", "lr_batch_set_profiling"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("lr_workspace_bytes", "lr_create", "lr_create_in", "lr_set_materials", "lr_init",
                 "lr_set_prescribed_velocity", "lr_step", "lr_run", "lr_sync", "lr_get_fields",
                 "lr_get_fields_device", "lr_time", "lr_set_profiling", "lr_set_tiled"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def arith_check(op: int, a, b, out, stream: int = 0) -> None:
    """lr_arith_check on device buffers: a, b, out are contiguous float64
    CUDA tensors of one size (out may be a or b); enqueued on ``stream``."""
    L = load()
    n = out.numel()
    if a.numel() != n or b.numel() != n:
        raise LrError(ERR_ARG, "lr_arith_check: a, b and out differ in size")
    rc = L.lr_arith_check(op, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                          ctypes.c_void_p(out.data_ptr()), n, ctypes.c_void_p(stream))
    if rc != OK:
        raise LrError(rc, "lr_arith_check failed")


def fp64_fma_probe(out, blocks: int, threads: int, iters: int, stream: int = 0) -> float:
    """Enqueue lr_fp64_fma_probe into the float64 CUDA tensor ``out`` (at
    least blocks * threads elements) on ``stream``; returns the flops it
    performs (16 per thread and iteration)."""
    if out.numel() < blocks * threads:
        raise LrError(ERR_ARG, "lr_fp64_fma_probe: output too small")
    rc = load().lr_fp64_fma_probe(ctypes.c_void_p(out.data_ptr()), blocks, threads, iters, ctypes.c_void_p(stream))
    if rc != OK:
        raise LrError(rc, "lr_fp64_fma_probe failed")
    return 16.0 * iters * blocks * threads


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def make_config(problem, stream: Optional[int] = None, precision: int = FP64, mixed_lanes: int = 0) -> Config:
    c = Config()
    load().lr_config_default(ctypes.byref(c))
    c.nx, c.ny = problem.nx, problem.ny
    c.x0, c.x1, c.y0, c.y1 = problem.x0, problem.x1, problem.y0, problem.y1
    c.nmat = problem.nmat
    c.cfl, c.a1, c.a2 = problem.cfl, problem.a1, problem.a2
    for q in range(4):
        c.bc[q] = problem.bc[q]
    c.precision = precision
    c.face_order = problem.face_order
    c.corner_recon = problem.corner_recon
    c.dt_fixed = problem.dt_fixed
    c.mixed_lanes = mixed_lanes
    c.remap = getattr(problem, "remap", 0)
    c.cuda_stream = stream
    return c


def _shape_field(out: np.ndarray, field: int, problem) -> np.ndarray:
    nx, ny, M = problem.nx, problem.ny, problem.nmat
    if field in (F_K, F_RHO_MAT, F_E_MAT, F_E_LAG):
        return out.reshape(M, ny, nx)
    if field in (F_P, F_RHO, F_E, F_C, F_VOL_LAGCF, F_Q):
        return out.reshape(ny, nx)
    if field in (F_UX, F_UY, F_UHX, F_UHY, F_FC, F_MC):
        return out.reshape(ny + 1, nx + 1)
    if field in (F_FX, F_MX):
        return out.reshape(ny, nx + 1)
    if field in (F_FY, F_MY):
        return out.reshape(ny + 1, nx)
    if field == F_CUTS:
        return out.reshape(6, ny, nx)
    if field == F_XA:
        return out.reshape(M, ny, nx + 1)
    if field == F_YA:
        return out.reshape(M, ny + 1, nx)
    if field == F_CA:
        return out.reshape(M, ny + 1, nx + 1)
    return out


def _materials(problem):
    mats = (Material * problem.nmat)()
    for a in range(problem.nmat):
        mats[a].eos = 1 if problem.pinf[a] > 0 else 0
        mats[a].gamma = float(problem.gamma[a])
        mats[a].pi = float(problem.pinf[a])
    return mats


class Sim:
    """One simulation on the GPU behind the C ABI."""

    def __init__(self, problem, use_torch: bool = True, precision: int = FP64, mixed_lanes: int = 0):
        L = load()
        self.p = problem
        self._arena = None
        self.stream = None
        stream = None
        if use_torch:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("CUDA device required")
            cs = torch.cuda.current_stream()
            # the library runs on a real stream so that torch events can be
            # recorded on it; the legacy default stream gets a private one
            self.stream = cs if cs.cuda_stream != 0 else torch.cuda.Stream()
            stream = self.stream.cuda_stream
        self.cfg = make_config(problem, stream, precision, mixed_lanes)
        self.precision = precision
        h = ctypes.c_void_p()
        if use_torch:
            import torch
            nbytes = ctypes.c_size_t()
            self._check(L.lr_workspace_bytes(ctypes.byref(self.cfg), ctypes.byref(nbytes)), None)
            self._arena = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device="cuda")
            base = self._arena.data_ptr()
            base = (base + 255) & ~255
            rc = L.lr_create_in(ctypes.byref(self.cfg), ctypes.c_void_p(base), nbytes.value, ctypes.byref(h))
        else:
            rc = L.lr_create(ctypes.byref(self.cfg), ctypes.byref(h))
        if rc != OK or not h.value:
            raise LrError(rc, "lr_create failed")
        self._h = h
        self._check(L.lr_set_materials(self._h, problem.nmat, _materials(problem)))
        self.init(problem)

    def _check(self, rc, h="self"):
        if rc != OK:
            msg = load().lr_last_error(self._h if h == "self" else None)
            raise LrError(rc, msg.decode() if msg else "")

    def init(self, problem):
        k, r, p = _c64(problem.k), _c64(problem.rho), _c64(problem.p)
        ux, uy = _c64(problem.ux), _c64(problem.uy)
        self._check(load().lr_init(self._h, _ptr(k), _ptr(r), _ptr(p), _ptr(ux), _ptr(uy)))

    def set_prescribed(self, ux, uy):
        self._pv = (_c64(ux), _c64(uy))
        self._check(load().lr_set_prescribed_velocity(self._h, _ptr(self._pv[0]), _ptr(self._pv[1])))

    def step(self, t_end: float = 1e300, sync: bool = True) -> Optional[float]:
        if sync:
            dt = ctypes.c_double()
            self._check(load().lr_step(self._h, t_end, ctypes.byref(dt)))
            return dt.value
        self._check(load().lr_step(self._h, t_end, None))
        return None

    def run(self, nsteps: int, t_end: float = 1e300):
        n = ctypes.c_long()
        t = ctypes.c_double()
        self._check(load().lr_run(self._h, t_end, nsteps, ctypes.byref(n), ctypes.byref(t)))
        return n.value, t.value

    def sync(self):
        self._check(load().lr_sync(self._h))

    @property
    def t(self) -> float:
        t = ctypes.c_double()
        self._check(load().lr_time(self._h, ctypes.byref(t), None))
        return t.value

    def dt_next(self) -> float:
        d = ctypes.c_double()
        self._check(load().lr_time(self._h, None, ctypes.byref(d)))
        return d.value

    def get(self, field: int) -> np.ndarray:
        L = load()
        n = L.lr_field_size(self._h, field)
        out = np.empty(n, dtype=np.float64)
        self._check(L.lr_get_fields(self._h, field, _ptr(out), n))
        return _shape_field(out, field, self.p)

    def get_device(self, field: int, out_ptr: int, n: int):
        self._check(load().lr_get_fields_device(self._h, field, ctypes.c_void_p(out_ptr), n))

    def launches_per_step(self) -> int:
        return load().lr_launches_per_step(self._h)

    def set_profiling(self, on: bool):
        self._check(load().lr_set_profiling(self._h, 1 if on else 0))

    def checkpoint(self) -> np.ndarray:
        """The exact state (lr_checkpoint_save) as a byte array."""
        L = load()
        n = L.lr_checkpoint_bytes(self._h)
        buf = np.empty(n, dtype=np.uint8)
        self._check(L.lr_checkpoint_save(self._h, buf.ctypes.data_as(ctypes.c_void_p), n))
        return buf

    def restore(self, buf: np.ndarray):
        """Continue from a checkpoint of the same configuration."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(load().lr_checkpoint_load(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.size))

    def set_tiled(self, on: bool):
        """Switch the tiled (fused, shared-memory) step kernels on or off."""
        self._check(load().lr_set_tiled(self._h, 1 if on else 0))

    @property
    def tiled(self) -> bool:
        return bool(load().lr_get_tiled(self._h))

    def kernel_times(self):
        L = load()
        n = 16
        names = (ctypes.c_char_p * n)()
        cnt = (ctypes.c_long * n)()
        ms = (ctypes.c_double * n)()
        k = L.lr_kernel_times(self._h, names, cnt, ms, n)
        return {names[q].decode(): (cnt[q], ms[q]) for q in range(min(k, n))}

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().lr_destroy(h)
            self._h = ctypes.c_void_p()
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TILE_SHAPES = ((32, 8), (64, 4), (16, 16), (128, 2))
RUNNING, DONE, FAILED, EMPTY = 0, 1, -1, -2


def batch_units(problem) -> int:
    """Units of a batch pool that one member on this grid occupies."""
    return (problem.nx + 2) * (problem.ny + 2)


class Batch:
    """Many simulations advanced together behind the batch C ABI
    (include/lr_batch.h): admission by pool units, one batched launch per
    kernel of the step, per-member CFL time steps."""

    def __init__(self, capacity_units: int, capacity_members: int, precision: int = FP64, nmat_max: int = 3,
                 max_member_cells: int = 1 << 20, use_torch: bool = True):
        L = load()
        self.stream = None
        cfg = BatchConfig()
        L.lr_batch_config_default(ctypes.byref(cfg))
        cfg.precision = precision
        cfg.nmat_max = nmat_max
        cfg.capacity_units = int(capacity_units)
        cfg.capacity_members = int(capacity_members)
        cfg.max_member_cells = int(max_member_cells)
        if use_torch:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("CUDA device required")
            self.stream = torch.cuda.Stream()
            cfg.cuda_stream = self.stream.cuda_stream
        self.cfg = cfg
        self.precision = precision
        self._h = ctypes.c_void_p()
        rc = L.lr_batch_create(ctypes.byref(cfg), ctypes.byref(self._h))
        if rc != OK or not self._h.value:
            raise LrError(rc, "lr_batch_create failed")
        self.problems = {}

    @staticmethod
    def unit_bytes(precision: int = FP64, nmat_max: int = 3) -> int:
        cfg = BatchConfig()
        load().lr_batch_config_default(ctypes.byref(cfg))
        cfg.precision, cfg.nmat_max = precision, nmat_max
        n = ctypes.c_size_t()
        rc = load().lr_batch_unit_bytes(ctypes.byref(cfg), ctypes.byref(n))
        if rc != OK:
            raise LrError(rc, "lr_batch_unit_bytes")
        return n.value

    def _check(self, rc):
        if rc != OK:
            msg = load().lr_batch_last_error(self._h)
            raise LrError(rc, msg.decode() if msg else "")

    def add(self, problem, t_end: Optional[float] = None, max_steps: int = 0) -> Optional[int]:
        """Admit a member; returns its id, or None when the pool or the
        member slots are full right now."""
        cfg = make_config(problem, None, self.precision)
        k, r, p = _c64(problem.k), _c64(problem.rho), _c64(problem.p)
        ux, uy = _c64(problem.ux), _c64(problem.uy)
        m = ctypes.c_int(-1)
        te = problem.t_end if t_end is None else t_end
        rc = load().lr_batch_add(self._h, ctypes.byref(cfg), _materials(problem), _ptr(k), _ptr(r), _ptr(p),
                                 _ptr(ux), _ptr(uy), float(te), int(max_steps), ctypes.byref(m))
        if rc == ERR_OOM:
            return None
        if rc != OK and m.value >= 0:  # admitted but its initial state is invalid: release it
            msg = load().lr_batch_last_error(self._h)
            load().lr_batch_remove(self._h, m.value)
            raise LrError(rc, msg.decode() if msg else "")
        self._check(rc)
        self.problems[m.value] = problem
        return m.value

    def set_limits(self, m: int, t_end: float = 1e300, max_steps: int = 0):
        self._check(load().lr_batch_set_limits(self._h, m, float(t_end), int(max_steps)))

    def remove(self, m: int):
        self._check(load().lr_batch_remove(self._h, m))
        self.problems.pop(m, None)

    def step(self, nsteps: int = 1):
        self._check(load().lr_batch_step(self._h, int(nsteps)))

    def sync(self):
        self._check(load().lr_batch_sync(self._h))

    def status(self, m: int):
        t = ctypes.c_double()
        n = ctypes.c_long()
        st = ctypes.c_int()
        self._check(load().lr_batch_status(self._h, m, ctypes.byref(t), ctypes.byref(n), ctypes.byref(st)))
        return t.value, n.value, st.value

    def status_all(self):
        S = self.cfg.capacity_members
        st = (ctypes.c_int * S)()
        n = (ctypes.c_long * S)()
        self._check(load().lr_batch_status_all(self._h, st, n, S))
        return list(st), list(n)

    def get(self, m: int, field: int) -> np.ndarray:
        L = load()
        n = L.lr_batch_field_size(self._h, m, field)
        out = np.empty(n, dtype=np.float64)
        self._check(L.lr_batch_get_fields(self._h, m, field, _ptr(out), n))
        return _shape_field(out, field, self.problems[m])

    def autotune(self, trial_steps: int = 3):
        self._check(load().lr_batch_autotune(self._h, int(trial_steps)))

    def schedule(self):
        sh = (ctypes.c_int * 9)()
        bp = (ctypes.c_int * 9)()
        ln = ctypes.c_int()
        self._check(load().lr_batch_schedule(self._h, sh, bp, ctypes.byref(ln)))
        return [TILE_SHAPES[q] for q in sh], list(bp), ln.value

    def launches_per_step(self) -> int:
        return load().lr_batch_launches_per_step(self._h)

    def set_persistent(self, on: bool):
        """One cooperative launch per step (on) or one launch per kernel."""
        self._check(load().lr_batch_set_persistent(self._h, 1 if on else 0))

    @property
    def persistent(self) -> bool:
        return bool(load().lr_batch_get_persistent(self._h))

    def test_barrier(self, extra_arrivals: int, limit_s: float):
        """Test hook: the persistent step's barriers wait for arrivals no
        block makes and give up after limit_s."""
        self._check(load().lr_batch_test_barrier(self._h, extra_arrivals, limit_s))

    def set_profiling(self, on: bool):
        self._check(load().lr_batch_set_profiling(self._h, 1 if on else 0))

    def kernel_times(self):
        L = load()
        n = 16
        names = (ctypes.c_char_p * n)()
        cnt = (ctypes.c_long * n)()
        ms = (ctypes.c_double * n)()
        k = L.lr_batch_kernel_times(self._h, names, cnt, ms, n)
        return {names[q].decode(): (cnt[q], ms[q]) for q in range(min(k, n))}

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().lr_batch_destroy(h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SERVE_FIELDS = (F_K, F_RHO_MAT, F_E_MAT, F_P, F_UX, F_UY)


class Server:
    """Continuous-batching request loop behind include/lr_serve.h: requests
    are admitted into a resident batch as pool units free up, advance
    together, and are retired with their final fields on the host."""

    def __init__(self, capacity_units: int, capacity_members: int, precision: int = FP64, nmat_max: int = 2,
                 max_member_cells: int = 1 << 22, max_chunk_steps: int = 64, max_bypass: int = 8, device: int = 0):
        L = load()
        cfg = ServerConfig()
        L.lr_server_config_default(ctypes.byref(cfg))
        cfg.batch.precision = precision
        cfg.batch.nmat_max = nmat_max
        cfg.batch.capacity_units = int(capacity_units)
        cfg.batch.capacity_members = int(capacity_members)
        cfg.batch.max_member_cells = int(max_member_cells)
        cfg.max_chunk_steps = int(max_chunk_steps)
        cfg.max_bypass = int(max_bypass)
        cfg.device = int(device)
        self.cfg = cfg
        self.precision = precision
        self._h = ctypes.c_void_p()
        rc = L.lr_server_create(ctypes.byref(cfg), ctypes.byref(self._h))
        if rc != OK or not self._h.value:
            raise LrError(rc, "lr_server_create failed")
        self.problems = {}

    def _check(self, rc):
        if rc != OK:
            msg = load().lr_server_last_error(self._h)
            raise LrError(rc, msg.decode() if msg else "")

    def submit(self, problem, t_end: Optional[float] = None, max_steps: int = 0) -> int:
        cfg = make_config(problem, None, self.precision)
        k, r, p = _c64(problem.k), _c64(problem.rho), _c64(problem.p)
        ux, uy = _c64(problem.ux), _c64(problem.uy)
        rid = ctypes.c_long(-1)
        te = problem.t_end if t_end is None else t_end
        self._check(load().lr_server_submit(self._h, ctypes.byref(cfg), _materials(problem), _ptr(k), _ptr(r),
                                            _ptr(p), _ptr(ux), _ptr(uy), float(te), int(max_steps),
                                            ctypes.byref(rid)))
        self.problems[rid.value] = problem
        return rid.value

    def wait(self, rid: int, timeout: float = -1.0) -> int:
        st = ctypes.c_int(0)
        rc = load().lr_server_wait(self._h, rid, float(timeout), ctypes.byref(st))
        if rc not in (OK, ERR_TIMEOUT):
            self._check(rc)
        return st.value

    def drain(self, timeout: float = -1.0) -> bool:
        rc = load().lr_server_drain(self._h, float(timeout))
        if rc not in (OK, ERR_TIMEOUT):
            self._check(rc)
        return rc == OK

    def info(self, rid: int) -> dict:
        a, b, c, t = (ctypes.c_double() for _ in range(4))
        n = ctypes.c_long()
        self._check(load().lr_server_info(self._h, rid, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                          ctypes.byref(t), ctypes.byref(n)))
        return {"submit": a.value, "admit": b.value, "done": c.value, "t": t.value, "steps": n.value}

    def result(self, rid: int, field: int) -> np.ndarray:
        L = load()
        n = L.lr_server_result_size(self._h, rid, field)
        if n == 0:
            raise LrError(ERR_STATE, f"no result field {field} for request {rid}")
        out = np.empty(n, dtype=np.float64)
        self._check(L.lr_server_result(self._h, rid, field, _ptr(out), n))
        return _shape_field(out, field, self.problems[rid])

    def release(self, rid: int):
        self._check(load().lr_server_release(self._h, rid))
        self.problems.pop(rid, None)

    def stats(self) -> dict:
        st = ServerStats()
        self._check(load().lr_server_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def clock(self) -> float:
        return load().lr_server_clock(self._h)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().lr_server_destroy(h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
