"""lr_cfl_dt_noalloc: the CFL time step for callers that may not allocate
device memory (their device memory is already reserved by another
allocator, or they run in a loop that must not call cudaMalloc).  The state
and the output live in the caller's own device buffers; the entry point uses
only scratch compiled into the library.  Its result must equal the time
step the allocating path (lr_init / lr_step, read back with lr_time)
computes for the same state, on two calls in a row."""
import ctypes

import pytest

from paper_2208_13409_gb300 import lr, problems as P

pytestmark = pytest.mark.gpu


def _noalloc_dt(sim, torch):
    L = lr.load()
    bufs = {}
    for f in (lr.F_K, lr.F_RHO_MAT, lr.F_E_MAT, lr.F_UX, lr.F_UY):
        n = L.lr_field_size(sim._h, f)
        t = torch.empty(n, dtype=torch.float64, device="cuda")
        sim.get_device(f, t.data_ptr(), n)
        bufs[f] = t
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    mats = (lr.Material * sim.p.nmat)()
    for a in range(sim.p.nmat):
        mats[a].gamma = float(sim.p.gamma[a])
        mats[a].pi = float(sim.p.pinf[a])
    ptr = lambda f: ctypes.c_void_p(bufs[f].data_ptr())
    rc = L.lr_cfl_dt_noalloc(ctypes.byref(sim.cfg), mats, ptr(lr.F_K), ptr(lr.F_RHO_MAT), ptr(lr.F_E_MAT),
                             ptr(lr.F_UX), ptr(lr.F_UY), ctypes.c_void_p(out.data_ptr()))
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


def test_noalloc_rejects_oversize():
    pr = P.uniform(2048, 1024)               # 2^21 cells > the 2^20 scratch
    L = lr.load()
    cfg = lr.make_config(pr)
    mats = (lr.Material * 1)()
    mats[0].gamma = 1.4
    fake = ctypes.c_void_p(256)              # never dereferenced: rejected before any launch
    rc = L.lr_cfl_dt_noalloc(ctypes.byref(cfg), mats, fake, fake, fake, fake, fake, fake)
    assert rc == lr.ERR_ARG
