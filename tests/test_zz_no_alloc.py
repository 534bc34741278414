"""lr_cfl_dt_noalloc: the CFL time step for callers that may not allocate
device memory (their device memory is already reserved by another
allocator, or they run in a loop that must not call cudaMalloc).  The state
and the output live in the caller's own device buffers; the entry point uses
only scratch compiled into the library.  Its result must equal the time
step the allocating path (lr_init / lr_step, read back with lr_time)
computes for the same state, on two calls in a row.  Every buffer handed
to it is a real device buffer of the size its grid needs, allocated and
written on the stream the call runs on."""
import ctypes
import math

import numpy as np
import pytest

from paper_2208_13409_gb300 import lr, problems as P

pytestmark = pytest.mark.gpu


def _mats(pr):
    mats = (lr.Material * pr.nmat)()
    for a in range(pr.nmat):
        mats[a].gamma = float(pr.gamma[a])
        mats[a].pi = float(pr.pinf[a])
    return mats


def _call(cfg, mats, bufs, out):
    L = lr.load()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    return L.lr_cfl_dt_noalloc(ctypes.byref(cfg), mats, ptr(bufs["k"]), ptr(bufs["rho"]), ptr(bufs["e"]),
                               ptr(bufs["ux"]), ptr(bufs["uy"]), ptr(out))


def _noalloc_dt(sim, torch):
    """The entry point on the simulation's current state, copied into
    caller-owned device buffers on the simulation's stream."""
    L = lr.load()
    names = {lr.F_K: "k", lr.F_RHO_MAT: "rho", lr.F_E_MAT: "e", lr.F_UX: "ux", lr.F_UY: "uy"}
    with torch.cuda.stream(sim.stream):
        bufs = {}
        for f, name in names.items():
            n = L.lr_field_size(sim._h, f)
            t = torch.empty(n, dtype=torch.float64, device="cuda")
            sim.get_device(f, t.data_ptr(), n)
            bufs[name] = t
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        rc = _call(sim.cfg, _mats(sim.p), bufs, out)
    assert rc == lr.OK
    sim.stream.synchronize()
    return float(out.item())


@pytest.mark.parametrize("make", [lambda: P.triple_point(140, 60),
                                  lambda: P.random_box(41, nx=37, ny=29, nmat=2, velocity=0.3).copy(
                                      bc=(P.BC_PERIODIC,) * 4)])
def test_noalloc_cfl_matches_allocating_path_twice(make):
    torch = pytest.importorskip("torch")
    pr = make()
    sim = lr.Sim(pr)
    first = _noalloc_dt(sim, torch)          # fresh state after lr_init
    assert first == pytest.approx(sim.dt_next(), rel=1e-12)
    for _ in range(3):
        sim.step()
    second = _noalloc_dt(sim, torch)         # the scratch keeps the last call's data
    assert second == pytest.approx(sim.dt_next(), rel=1e-12)
    assert second != first
    sim.close()


def _host_state(pr, torch):
    """Device copies of a problem's initial state as the entry point reads
    it (k, rho, e = (p + pi) / ((gamma - 1) rho), node velocities)."""
    g = pr.gamma[:, None, None]
    pi = pr.pinf[:, None, None]
    rho = np.where(pr.k > 0, pr.rho, 0.0)
    e = np.where(pr.k > 0, (pr.p + pi) / ((g - 1.0) * np.where(pr.k > 0, pr.rho, 1.0)), 0.0)
    arrs = {"k": pr.k, "rho": rho, "e": e, "ux": pr.ux, "uy": pr.uy}
    return {n: torch.tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda") for n, a in arrs.items()}


def test_noalloc_nan_state_gives_nan():
    """A state that is not finite gives a NaN time step, not a quiet one."""
    torch = pytest.importorskip("torch")
    pr = P.random_box(42, nx=20, ny=16, nmat=2, velocity=0.2)
    bufs = _host_state(pr, torch)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    cfg = lr.make_config(pr)
    assert _call(cfg, _mats(pr), bufs, out) == lr.OK
    torch.cuda.synchronize()
    assert math.isfinite(out.item()) and out.item() > 0.0
    bufs["rho"][5] = float("nan")
    bufs["rho"][0] = float("nan")
    assert _call(cfg, _mats(pr), bufs, out) == lr.OK
    torch.cuda.synchronize()
    assert math.isnan(out.item())


def test_noalloc_rejects_bad_configurations():
    """Rejected before any launch; the buffers are real and sized for the
    grid, so nothing could read outside them either way."""
    torch = pytest.importorskip("torch")
    pr = P.random_box(43, nx=20, ny=16, nmat=2, velocity=0.2)
    bufs = _host_state(pr, torch)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    mats = _mats(pr)
    bad = []
    c = lr.make_config(pr); c.bc[0] = c.bc[1] = 7; bad.append(c)              # unknown boundary kind
    c = lr.make_config(pr); c.cfl = 1.5; bad.append(c)                        # cfl > 1
    c = lr.make_config(pr); c.cfl = 0.0; bad.append(c)
    c = lr.make_config(pr); c.bc[0] = lr.BC_PERIODIC; bad.append(c)           # xlo != xhi
    c = lr.make_config(pr); c.nmat = 4; bad.append(c)
    for cfg in bad:
        assert _call(cfg, mats, bufs, out) == lr.ERR_ARG
    torch.cuda.synchronize()
    assert out.item() == -1.0


def test_noalloc_rejects_oversize():
    """2^21 cells exceed the 2^20-cell scratch: rejected before any launch.
    The buffers are real device buffers of the full grid's size."""
    torch = pytest.importorskip("torch")
    nx, ny = 2048, 1024
    pr = P.uniform(nx, ny)
    cfg = lr.make_config(pr)
    mats = _mats(pr)
    nc, nn = nx * ny, (nx + 1) * (ny + 1)
    bufs = {"k": torch.ones(nc, dtype=torch.float64, device="cuda"),
            "rho": torch.ones(nc, dtype=torch.float64, device="cuda"),
            "e": torch.full((nc,), 2.5, dtype=torch.float64, device="cuda"),
            "ux": torch.zeros(nn, dtype=torch.float64, device="cuda"),
            "uy": torch.zeros(nn, dtype=torch.float64, device="cuda")}
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert _call(cfg, mats, bufs, out) == lr.ERR_ARG
    torch.cuda.synchronize()
    assert out.item() == -1.0
