"""GPU (CUDA, through the C ABI) against the FP64 oracle, element by element.

Tolerances: after one step the per-field max relative difference
(max|g-o| / max|o|) must be <= 1e-11; after 100 steps the per-field L1
relative difference (sum|g-o| / sum|o|) must be <= 1e-9.  Both sides run the
same scheme in IEEE double; the tolerance absorbs FMA contraction and
operation order only.
"""
import numpy as np
import pytest

import oracle
from paper_2208_13409_gb300 import lr, problems as P
from parity import compare, l1_rel, max_rel

pytestmark = pytest.mark.gpu

TOL_1 = 1e-11
TOL_100 = 1e-9


def _pair(pr, precision=lr.FP64):
    return lr.Sim(pr, precision=precision), oracle.Oracle(pr)


def _steps(sim, orc, n, t_end=1e300):
    for q in range(n):
        dg = sim.step(t_end)
        do = orc.step(t_end)
        assert dg == pytest.approx(do, rel=1e-12, abs=1e-300), (q, dg, do)


def _assert_close(res, tol, what):
    bad = {k: v for k, v in res.items() if not (v <= tol)}
    assert not bad, f"{what}: {bad}"


CASES_1 = {
    "sod_256x4": lambda: P.sod(),
    "sod_transposed": lambda: P.sod(nx=64, transpose=True),
    "triple_point_140x60": lambda: P.triple_point(140, 60),
    "shock_bubble_256x64": lambda: P.shock_bubble(256, 64),
    "random2_walls_velocity": lambda: P.random_box(21, nx=77, ny=45, nmat=2, velocity=0.3),
    "random3_walls_velocity": lambda: P.random_box(22, nx=53, ny=70, nmat=3, velocity=0.3),
    "random3_periodic": lambda: P.random_box(23, nx=66, ny=39, nmat=3, velocity=0.4).copy(bc=(P.BC_PERIODIC,) * 4),
    "mixed_bc_xper": lambda: P.random_box(24, nx=40, ny=33, nmat=2, velocity=0.2).copy(
        bc=(P.BC_PERIODIC, P.BC_PERIODIC, P.BC_REFLECT, P.BC_REFLECT)),
    "mono_uniform_diag": lambda: P.uniform(37, 29, rho=1.2, p=0.8, u=(0.3, -0.25)),
    "upwind_o1": lambda: P.random_box(25, nx=48, ny=48, nmat=2, velocity=0.3).copy(
        face_order=1, corner_recon=P.CORNER_UPWIND),
    "tiny_2x2": lambda: P.random_box(26, nx=2, ny=2, nmat=2, velocity=0.1),
    "tiny_3x5_periodic": lambda: P.random_box(27, nx=3, ny=5, nmat=3, velocity=0.1).copy(bc=(P.BC_PERIODIC,) * 4),
    "air_water_128": lambda: P.air_water(5, side=128),
}


PRECISIONS = {"fp64": lr.FP64, "df64": lr.DF64}


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
@pytest.mark.parametrize("name", sorted(CASES_1))
def test_parity_one_and_five_steps(name, prec):
    pr = CASES_1[name]()
    sim, orc = _pair(pr, PRECISIONS[prec])
    # init: e from p through the EOS; stiffened-gas p = (g-1) rho e - pi
    # cancels (pi = 2.6e9 against p = 1e5), so allow a few ulps of pi
    _assert_close(compare(sim, orc), 1e-13, f"{name} init")
    _steps(sim, orc, 1)
    _assert_close(compare(sim, orc), TOL_1, f"{name} 1 step")
    _steps(sim, orc, 4)
    _assert_close(compare(sim, orc), 1e-10, f"{name} 5 steps")


def test_intermediates_after_one_step():
    """Per-phase parity: u^{n+1/2}, Q, face/corner volume and mass fluxes,
    Lagrangian volume, e^{lag}."""
    pr = P.random_box(31, nx=61, ny=47, nmat=3, velocity=0.3)
    sim, orc = _pair(pr)
    _steps(sim, orc, 3)
    fields = {"uhx": lr.F_UHX, "uhy": lr.F_UHY, "q": lr.F_Q, "fx": lr.F_FX, "fy": lr.F_FY,
              "fc": lr.F_FC, "mx": lr.F_MX, "my": lr.F_MY, "mc": lr.F_MC, "vol_lagcf": lr.F_VOL_LAGCF,
              "c": lr.F_C}
    res = {k: max_rel(sim.get(f), orc.get(f)) for k, f in fields.items()}
    k = orc.get(oracle.F_K)
    res["k_elag"] = max_rel(k * sim.get(lr.F_E_LAG), k * orc.get(oracle.F_E_LAG))
    _assert_close(res, TOL_1, "intermediates")


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
@pytest.mark.parametrize("name,make", [
    ("sod_256x4", lambda: P.sod()),
    ("triple_point_140x60", lambda: P.triple_point(140, 60)),
    ("shock_bubble_256x64", lambda: P.shock_bubble(256, 64)),
])
def test_parity_100_steps_l1(name, make, prec):
    pr = make()
    sim, orc = _pair(pr, PRECISIONS[prec])
    for _ in range(100):
        sim.step(pr.t_end, sync=False)
        orc.step(pr.t_end)
    sim.sync()
    assert sim.t == pytest.approx(orc.t, rel=1e-12)
    _assert_close(compare(sim, orc, l1_rel), TOL_100, f"{name} 100 steps")


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
@pytest.mark.parametrize("name,make", [
    ("random2_walls_velocity", lambda: P.random_box(21, nx=77, ny=45, nmat=2, velocity=0.3)),
    ("random3_walls_velocity", lambda: P.random_box(22, nx=53, ny=70, nmat=3, velocity=0.3)),
])
def test_mixed_lanes_and_clipping(name, make, lanes, prec):
    """Every lanes-per-mixed-cell setting of the interface kernel against the
    oracle, over steps where the oracle clips some material's outgoing volume
    (so the rescaling pass of the kernel runs)."""
    pr = make()
    sim = lr.Sim(pr, precision=PRECISIONS[prec], mixed_lanes=lanes)
    orc = oracle.Oracle(pr)
    clipped = 0
    for q in range(16):
        _steps(sim, orc, 1)
        clipped += int((orc.get(oracle.F_SCLIP) < 1.0).sum())
        _assert_close(compare(sim, orc), TOL_1 if q == 0 else 1e-10, f"{name} L={lanes} step {q + 1}")
    assert clipped > 0


def test_lr_run_matches_stepwise_and_oracle():
    """lr_run (CUDA graphs, dt kept on the device) against the oracle."""
    pr = P.triple_point(140, 60)
    sim, orc = _pair(pr)
    n, t = sim.run(37)
    assert n == 37
    for _ in range(37):
        orc.step()
    assert t == pytest.approx(orc.t, rel=1e-12)
    _assert_close(compare(sim, orc), 1e-10, "lr_run 37 steps")


def test_sod_to_t_end():
    pr = P.sod()
    sim, orc = _pair(pr)
    n, t = sim.run(10000, pr.t_end)
    no = orc.run(10000, pr.t_end)
    assert n == no and t == pytest.approx(0.2, rel=1e-14)
    _assert_close(compare(sim, orc, l1_rel), TOL_100, "sod t_end")
    # a further step past t_end changes nothing
    before = sim.get(lr.F_RHO)
    assert sim.step(pr.t_end) == 0.0
    np.testing.assert_array_equal(sim.get(lr.F_RHO), before)


def test_prescribed_one_node_displacement():
    """Remap-only path (section 3.2 set-up) on the GPU matches the oracle and
    the closed form 1 + eps/(1+eps) + eps^2."""
    n, eps = 5, 0.1
    pr = P.uniform(n, n, periodic=True)
    pr.rho[0, 2, 2] = 2.0
    dt = 1e-3
    pr = pr.copy(dt_fixed=dt, face_order=1, corner_recon=P.CORNER_UPWIND)
    dx = 1.0 / n
    vx = np.zeros((n + 1, n + 1))
    vx[3, 3] = eps * dx / dt
    sim, orc = _pair(pr)
    sim.set_prescribed(vx, vx)
    orc.set_prescribed(vx, vx)
    _steps(sim, orc, 1)
    v = sim.get(lr.F_VOL_LAGCF)[2, 2] / dx ** 2
    assert v == pytest.approx(1 + eps / (1 + eps) + eps ** 2, rel=1e-13)
    _assert_close(compare(sim, orc), TOL_1, "prescribed")


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
def test_full_size_one_step_triple_point(prec):
    """The bench workload (1400 x 600, three materials) after warm-up steps:
    every field against the oracle."""
    pr = P.triple_point()
    sim, orc = _pair(pr, PRECISIONS[prec])
    _steps(sim, orc, 3)
    _assert_close(compare(sim, orc), TOL_1, "triple point 1400x600")


def test_full_size_one_step_shock_bubble():
    pr = P.shock_bubble()
    sim, orc = _pair(pr)
    _steps(sim, orc, 1)
    _assert_close(compare(sim, orc), TOL_1, "shock bubble 4096x1024")


def test_invalid_input_is_rejected():
    pr = P.sod(nx=16)
    bad = pr.copy()
    bad.k[0, 0, 0] = 0.7  # sum k != 1
    with pytest.raises(lr.LrError):
        lr.Sim(bad)
    bad = pr.copy()
    bad.rho[0, 0, 0] = -1.0
    with pytest.raises(lr.LrError):
        lr.Sim(bad)


def test_conservation_on_gpu():
    pr = P.random_box(7, nx=32, ny=28, nmat=3, velocity=0.3).copy(bc=(P.BC_PERIODIC,) * 4)
    sim = lr.Sim(pr)
    c0 = sim.get(lr.F_CONS)
    sim.run(25)
    c1 = sim.get(lr.F_CONS)
    for a in range(3):
        assert c1[a] == pytest.approx(c0[a], rel=1e-12)
    assert c1[3] == pytest.approx(c0[3], rel=1e-13)
    orc = oracle.Oracle(pr)
    orc.run(25)
    np.testing.assert_allclose(c1, orc.get(oracle.F_CONS), rtol=1e-11, atol=1e-14)


REMAPS = {"direct": P.REMAP_DIRECT, "ad": P.REMAP_AD}
REMAP_CASES = {
    "sod_256x4": lambda: P.sod(),
    "triple_point_140x60": lambda: P.triple_point(140, 60),
    "random2_walls_velocity": lambda: P.random_box(21, nx=77, ny=45, nmat=2, velocity=0.3),
    "random3_walls_velocity": lambda: P.random_box(22, nx=53, ny=70, nmat=3, velocity=0.3),
    "random3_periodic": lambda: P.random_box(23, nx=66, ny=39, nmat=3, velocity=0.4).copy(bc=(P.BC_PERIODIC,) * 4),
    "mixed_bc_xper": lambda: P.random_box(24, nx=40, ny=33, nmat=2, velocity=0.2).copy(
        bc=(P.BC_PERIODIC, P.BC_PERIODIC, P.BC_REFLECT, P.BC_REFLECT)),
    "upwind_o1": lambda: P.random_box(25, nx=48, ny=48, nmat=2, velocity=0.3).copy(
        face_order=1, corner_recon=P.CORNER_UPWIND),
    "air_water_128": lambda: P.air_water(5, side=128),
}


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
@pytest.mark.parametrize("remap", sorted(REMAPS))
@pytest.mark.parametrize("name", sorted(REMAP_CASES))
def test_comparator_remaps_one_and_six_steps(name, remap, prec):
    """Direct and alternate-directions remaps (section 2) against the
    oracle; six steps cover both sweep orders of the AD remap."""
    pr = REMAP_CASES[name]().copy(remap=REMAPS[remap])
    sim, orc = _pair(pr, PRECISIONS[prec])
    _steps(sim, orc, 1)
    _assert_close(compare(sim, orc), TOL_1, f"{name} {remap} 1 step")
    _steps(sim, orc, 5)
    _assert_close(compare(sim, orc), 1e-10, f"{name} {remap} 6 steps")


@pytest.mark.parametrize("remap", sorted(REMAPS))
def test_comparator_remaps_100_steps_and_graphs(remap):
    """100 steps through lr_run (CUDA graphs; the AD sweep order read from
    the device step count) against the oracle, L1."""
    pr = P.triple_point(140, 60).copy(remap=REMAPS[remap])
    sim, orc = _pair(pr)
    n, t = sim.run(100)
    assert n == 100
    for _ in range(100):
        orc.step()
    assert t == pytest.approx(orc.t, rel=1e-12)
    _assert_close(compare(sim, orc, l1_rel), TOL_100, f"{remap} 100 steps")


CORNERS = {"avg": P.CORNER_AVG, "xy": P.CORNER_XY, "lsq": P.CORNER_LSQ}
CORNER_CASES = {
    "triple_point_140x60": lambda: P.triple_point(140, 60),
    "random3_walls_velocity": lambda: P.random_box(22, nx=53, ny=70, nmat=3, velocity=0.3),
    "random2_periodic": lambda: P.random_box(23, nx=66, ny=39, nmat=2, velocity=0.4).copy(bc=(P.BC_PERIODIC,) * 4),
    "mono_smooth_periodic": lambda: P.uniform(40, 36, rho=1.0, p=1.0, u=(0.3, -0.2)).copy(
        rho=np.array([1.0 + 0.3 * np.sin(np.linspace(0, 6.28, 40))[None, :] * np.cos(np.linspace(0, 6.28, 36))[:, None]])),
}


@pytest.mark.parametrize("prec", sorted(PRECISIONS))
@pytest.mark.parametrize("corner", sorted(CORNERS))
@pytest.mark.parametrize("name", sorted(CORNER_CASES))
def test_corner_variants_one_and_six_steps(name, corner, prec):
    """Average, x-y and least-squares corner values (section 3.3) against
    the oracle."""
    pr = CORNER_CASES[name]().copy(corner_recon=CORNERS[corner])
    sim, orc = _pair(pr, PRECISIONS[prec])
    _steps(sim, orc, 1)
    _assert_close(compare(sim, orc), TOL_1, f"{name} {corner} 1 step")
    _steps(sim, orc, 5)
    _assert_close(compare(sim, orc), 1e-10, f"{name} {corner} 6 steps")


@pytest.mark.parametrize("remap", sorted(REMAPS))
def test_least_squares_faces_with_comparator_remaps(remap):
    pr = P.random_box(22, nx=53, ny=70, nmat=3, velocity=0.3).copy(corner_recon=P.CORNER_LSQ, remap=REMAPS[remap])
    sim, orc = _pair(pr)
    _steps(sim, orc, 6)
    _assert_close(compare(sim, orc), 1e-10, f"lsq {remap} 6 steps")


@pytest.mark.parametrize("prec", [lr.FP64, lr.DF64, lr.FP32])
def test_two_stream_schedule_matches_serial(prec):
    """The step's second stream (interface kernels beside lr_cell_cf and
    lr_mat_flux, lr_dual_flux beside lr_cell_update) gives the same bits as
    the profiling mode, which runs every kernel on one stream in order: the
    kernels that run side by side write disjoint arrays."""
    pr = P.triple_point(280, 120)
    a, b = lr.Sim(pr, precision=prec), lr.Sim(pr, precision=prec)
    b.set_profiling(True)
    for _ in range(40):
        a.step()                    # two streams
        b.step()                    # one stream, kernel by kernel
    for f in (lr.F_K, lr.F_RHO_MAT, lr.F_E_MAT, lr.F_UX, lr.F_UY):
        assert np.array_equal(a.get(f), b.get(f)), f
    assert a.t == b.t
    a.close(); b.close()


def test_fields_into_page_locked_memory():
    """lr_get_fields into page-locked host memory (the view kernel writes it
    directly) gives the same values as into pageable memory."""
    torch = pytest.importorskip("torch")
    import ctypes
    pr = P.random_box(31, nx=91, ny=57, nmat=3, velocity=0.3)
    sim = lr.Sim(pr)
    sim.run(5)
    L = lr.load()
    fields = (lr.F_K, lr.F_RHO_MAT, lr.F_E_MAT, lr.F_UX, lr.F_UY, lr.F_P, lr.F_C, lr.F_DT, lr.F_NMIXED, lr.F_CONS)
    P_ = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for f in fields:
        ref = sim.get(f).ravel()
        pinned = torch.zeros(ref.size, dtype=torch.float64).pin_memory().numpy()
        assert L.lr_get_fields(sim._h, f, P_(pinned), pinned.size) == 0
        assert np.array_equal(pinned, ref), f
    # several fields enqueued, one synchronisation
    outs = {f: torch.zeros(sim.get(f).size, dtype=torch.float64).pin_memory().numpy()
            for f in fields if f != lr.F_CONS}
    for f, a in outs.items():
        assert L.lr_get_fields_async(sim._h, f, P_(a), a.size) == 0
    sim.sync()
    for f, a in outs.items():
        assert np.array_equal(a, sim.get(f).ravel()), f
    plain = np.zeros(sim.get(lr.F_K).size)
    assert L.lr_get_fields_async(sim._h, lr.F_K, P_(plain), plain.size) == 0  # pageable: copied on return
    assert np.array_equal(plain, sim.get(lr.F_K).ravel())
    assert L.lr_get_fields_async(sim._h, lr.F_CONS, P_(plain), plain.size) != 0
    sim.close()
