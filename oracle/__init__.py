"""ctypes wrapper around the plain FP64 CPU oracle (``lr_oracle.c``).

TEST INFRASTRUCTURE: imported only by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The CUDA product never imports
this package, and this package imports nothing from the product.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lr_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblr_oracle.so")

BC_REFLECT, BC_PERIODIC = 0, 1
CORNER_UPWIND, CORNER_DIAG = 0, 1

F_K, F_RHO_MAT, F_E_MAT, F_P, F_RHO, F_E, F_UX, F_UY, F_CONS, F_C = range(10)
F_UHX, F_UHY, F_VOL_LAGCF, F_E_LAG, F_FX, F_FY, F_FC, F_MX, F_MY, F_MC, F_Q, F_DT = range(20, 32)
F_CUTS, F_XA, F_YA, F_CA = range(32, 36)
F_SCLIP = 37
F_MP_NEW, F_DUAL = 38, 39
DUAL_X, DUAL_Y, DUAL_PP, DUAL_PM = range(4)


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("nmat", ctypes.c_int),
        ("cfl", ctypes.c_double), ("a1", ctypes.c_double), ("a2", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("face_order", ctypes.c_int), ("corner_recon", ctypes.c_int),
        ("dt_fixed", ctypes.c_double),
        ("remap", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(Config), dp, dp]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_init.restype = ctypes.c_int
        L.orc_init.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
        L.orc_set_prescribed.restype = ctypes.c_int
        L.orc_set_prescribed.argtypes = [ctypes.c_void_p, dp, dp]
        L.orc_set_remap_velocity.restype = ctypes.c_int
        L.orc_set_remap_velocity.argtypes = [ctypes.c_void_p, dp, dp]
        L.orc_step.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_double, dp]
        L.orc_get.restype = ctypes.c_int
        L.orc_get.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, ctypes.c_long]
        L.orc_size.restype = ctypes.c_long
        L.orc_size.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_time.restype = ctypes.c_double
        L.orc_time.argtypes = [ctypes.c_void_p]
        L.orc_t_cell_volume.restype = ctypes.c_double
        L.orc_t_cell_volume.argtypes = [dp]
        L.orc_t_vanleer.restype = ctypes.c_double
        L.orc_t_vanleer.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_t_halfplane_area.restype = ctypes.c_double
        L.orc_t_halfplane_area.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_t_plic.restype = ctypes.c_double
        L.orc_t_plic.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_t_eos.restype = None
        L.orc_t_eos.argtypes = [ctypes.c_double] * 4 + [dp, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Oracle:
    """One simulation held by the oracle.  Arrays follow the C layout:
    cells [nmat][ny][nx], nodes [ny+1][nx+1]."""

    def __init__(self, problem):
        L = lib()
        self.p = problem
        c = Config()
        c.nx, c.ny = problem.nx, problem.ny
        c.x0, c.x1, c.y0, c.y1 = problem.x0, problem.x1, problem.y0, problem.y1
        c.nmat = problem.nmat
        c.cfl, c.a1, c.a2 = problem.cfl, problem.a1, problem.a2
        for q in range(4):
            c.bc[q] = problem.bc[q]
        c.face_order = problem.face_order
        c.corner_recon = problem.corner_recon
        c.dt_fixed = problem.dt_fixed
        c.remap = getattr(problem, "remap", 0)
        g = _c64(problem.gamma)
        pi = _c64(problem.pinf)
        self._h = L.orc_create(ctypes.byref(c), _dp(g), _dp(pi))
        if not self._h:
            raise ValueError("orc_create rejected the configuration")
        self._keep = [g, pi]
        k, r, p = _c64(problem.k), _c64(problem.rho), _c64(problem.p)
        ux, uy = _c64(problem.ux), _c64(problem.uy)
        rc = L.orc_init(self._h, _dp(k), _dp(r), _dp(p), _dp(ux), _dp(uy))
        if rc != 0:
            raise ValueError(f"orc_init failed ({rc})")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_prescribed(self, ux, uy):
        self._pv = (_c64(ux), _c64(uy))
        lib().orc_set_prescribed(self._h, _dp(self._pv[0]), _dp(self._pv[1]))

    def set_remap_velocity(self, ux, uy):
        """Test hook: with a prescribed velocity set, the dual remap carries
        this node field as u^{lag} (the flux geometry still follows the
        prescribed velocity)."""
        self._rv = (_c64(ux), _c64(uy))
        lib().orc_set_remap_velocity(self._h, _dp(self._rv[0]), _dp(self._rv[1]))

    def step(self, t_end: float = 1e300) -> float:
        dt = ctypes.c_double(0.0)
        rc = lib().orc_step(self._h, t_end, ctypes.byref(dt))
        if rc != 0:
            raise RuntimeError(f"oracle step failed ({rc})")
        return dt.value

    def run(self, nsteps: int, t_end: float = 1e300) -> int:
        n = 0
        for _ in range(nsteps):
            if self.step(t_end) <= 0.0:
                break
            n += 1
        return n

    @property
    def t(self) -> float:
        return lib().orc_time(self._h)

    def get(self, field: int) -> np.ndarray:
        L = lib()
        n = L.orc_size(self._h, field)
        out = np.empty(n, dtype=np.float64)
        rc = L.orc_get(self._h, field, _dp(out), n)
        if rc != 0:
            raise ValueError(f"orc_get({field}) failed")
        nx, ny, M = self.p.nx, self.p.ny, self.p.nmat
        if field in (F_K, F_RHO_MAT, F_E_MAT, F_E_LAG, F_SCLIP):
            return out.reshape(M, ny, nx)
        if field in (F_P, F_RHO, F_E, F_C, F_VOL_LAGCF, F_Q):
            return out.reshape(ny, nx)
        if field in (F_UX, F_UY, F_UHX, F_UHY, F_FC, F_MC, F_MP_NEW):
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
        if field == F_DUAL:
            return out.reshape(4, 3, ny + 1, nx + 1)
        return out


def cell_volume(xy8) -> float:
    a = _c64(xy8)
    return lib().orc_t_cell_volume(_dp(a))


def vanleer(dm: float, dp: float) -> float:
    return lib().orc_t_vanleer(dm, dp)


def halfplane_area(poly, n, d) -> float:
    a = _c64(poly).ravel()
    return lib().orc_t_halfplane_area(_dp(a), len(a) // 2, n[0], n[1], d)


def plic(poly, n, target) -> float:
    a = _c64(poly).ravel()
    return lib().orc_t_plic(_dp(a), len(a) // 2, n[0], n[1], target)


def eos(gamma, pinf, rho, e):
    p = ctypes.c_double()
    c2 = ctypes.c_double()
    lib().orc_t_eos(gamma, pinf, rho, e, ctypes.byref(p), ctypes.byref(c2))
    return p.value, c2.value
