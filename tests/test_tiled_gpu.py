"""The tiled step (fused kernel pairs over shared-memory tiles, boundary
conditions applied once at staging) against the FP64 oracle, element by
element, at the same bars as the unfused step: per-field max relative
difference <= 1e-11 after one step, <= 1e-10 after five, L1 <= 1e-9 after
100 (FP64 and double-float arithmetic).  In FP32 the tiled and unfused
steps evaluate the same expressions with a different contraction of a few
multiply-adds, so they agree to float round-off."""
import numpy as np
import pytest

import oracle
from paper_2208_13409_gb300 import lr, problems as P
from parity import compare, l1_rel

pytestmark = pytest.mark.gpu

CASES = {
    "sod_256x4": lambda: P.sod(),
    "sod_transposed": lambda: P.sod(nx=64, transpose=True),
    "triple_point_140x60": lambda: P.triple_point(140, 60),
    "shock_bubble_256x64": lambda: P.shock_bubble(256, 64),
    "random2_walls_velocity": lambda: P.random_box(21, nx=77, ny=45, nmat=2, velocity=0.3),
    "random3_walls_velocity": lambda: P.random_box(22, nx=53, ny=70, nmat=3, velocity=0.3),
    "random3_periodic": lambda: P.random_box(23, nx=66, ny=39, nmat=3, velocity=0.4).copy(bc=(P.BC_PERIODIC,) * 4),
    "mixed_bc_xper": lambda: P.random_box(24, nx=40, ny=33, nmat=2, velocity=0.2).copy(
        bc=(P.BC_PERIODIC, P.BC_PERIODIC, P.BC_REFLECT, P.BC_REFLECT)),
    "mixed_bc_yper": lambda: P.random_box(28, nx=35, ny=41, nmat=3, velocity=0.3).copy(
        bc=(P.BC_REFLECT, P.BC_REFLECT, P.BC_PERIODIC, P.BC_PERIODIC)),
    "mono_uniform_diag": lambda: P.uniform(37, 29, rho=1.2, p=0.8, u=(0.3, -0.25)),
    "upwind_o1": lambda: P.random_box(25, nx=48, ny=48, nmat=2, velocity=0.3).copy(
        face_order=1, corner_recon=P.CORNER_UPWIND),
    "tiny_2x2": lambda: P.random_box(26, nx=2, ny=2, nmat=2, velocity=0.1),
    "tiny_3x5_periodic": lambda: P.random_box(27, nx=3, ny=5, nmat=3, velocity=0.1).copy(bc=(P.BC_PERIODIC,) * 4),
    "tile_edges_33x9": lambda: P.random_box(29, nx=33, ny=9, nmat=3, velocity=0.3),
    "tile_edges_32x8_periodic": lambda: P.random_box(30, nx=32, ny=8, nmat=2, velocity=0.3).copy(
        bc=(P.BC_PERIODIC,) * 4),
    "air_water_128": lambda: P.air_water(5, side=128),
    "random2_128x40": lambda: P.random_box(32, nx=128, ny=40, nmat=2, velocity=0.3),
}


def _tiled(pr, precision):
    sim = lr.Sim(pr, precision=precision)
    sim.set_tiled(True)
    assert sim.tiled
    return sim


def _steps(sim, orc, n):
    for q in range(n):
        dg, do = sim.step(), orc.step()
        assert dg == pytest.approx(do, rel=1e-12, abs=1e-300), (q, dg, do)


def _assert_close(res, tol, what):
    bad = {k: v for k, v in res.items() if not (v <= tol)}
    assert not bad, f"{what}: {bad}"


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_tiled_parity_one_and_five_steps(name, prec):
    pr = CASES[name]()
    sim, orc = _tiled(pr, {"fp64": lr.FP64, "df64": lr.DF64}[prec]), oracle.Oracle(pr)
    _steps(sim, orc, 1)
    _assert_close(compare(sim, orc), 1e-11, f"{name} 1 step")
    _steps(sim, orc, 4)
    _assert_close(compare(sim, orc), 1e-10, f"{name} 5 steps")
    sim.close()


@pytest.mark.parametrize("name", ["triple_point_140x60", "shock_bubble_256x64", "random3_periodic"])
def test_tiled_parity_100_steps_graphs(name):
    """100 steps through lr_run (CUDA graphs of the tiled step)."""
    pr = CASES[name]()
    sim, orc = _tiled(pr, lr.FP64), oracle.Oracle(pr)
    n, _ = sim.run(100)
    assert n == 100
    orc.run(100)
    _assert_close(compare(sim, orc, l1_rel), 1e-9, f"{name} 100 steps")
    sim.close()


@pytest.mark.parametrize("name", ["triple_point_140x60", "random3_periodic", "mixed_bc_yper", "tiny_2x2",
                                  "shock_bubble_256x64", "random2_128x40"])
def test_tiled_fp32_matches_unfused_fp32(name):
    """Also the FP32 staging by float4 (two materials, rows of a multiple of
    four cells, interior tiles: the shock-bubble and the 128 x 40 box)."""
    pr = CASES[name]()
    a = lr.Sim(pr, precision=lr.FP32)
    assert a.tiled  # the default in FP32
    b = lr.Sim(pr, precision=lr.FP32)
    b.set_tiled(False)
    for _ in range(20):
        da, db = a.step(), b.step()
        assert da == pytest.approx(db, rel=1e-5)
    for f in (lr.F_K, lr.F_RHO, lr.F_P, lr.F_UX, lr.F_UY):
        assert l1_rel(a.get(f), b.get(f)) <= 1e-5, f
    a.close()
    b.close()


def test_tiled_switch_rejected_for_other_remaps():
    pr = P.random_box(40, nx=20, ny=20, nmat=2, velocity=0.2).copy(remap=P.REMAP_DIRECT)
    sim = lr.Sim(pr)
    assert not sim.tiled
    with pytest.raises(lr.LrError):
        sim.set_tiled(True)
    pr = P.random_box(40, nx=20, ny=20, nmat=2, velocity=0.2).copy(corner_recon=P.CORNER_LSQ)
    sim2 = lr.Sim(pr, precision=lr.FP32)
    assert not sim2.tiled
    sim.close()
    sim2.close()


def test_tiled_prescribed_velocity_remap():
    """Imposed velocity (momentum equation and dual remap skipped): the tiled
    node kernel keeps the prescribed field."""
    n = 24
    pr = P.random_box(41, nx=n, ny=n, nmat=2).copy(bc=(P.BC_PERIODIC,) * 4, dt_fixed=1e-3)
    vx = np.full((n + 1, n + 1), 3.0)
    vy = np.full((n + 1, n + 1), -2.0)
    sim, orc = _tiled(pr, lr.FP64), oracle.Oracle(pr)
    sim.set_prescribed(vx, vy)
    orc.set_prescribed(vx, vy)
    _steps(sim, orc, 5)
    _assert_close(compare(sim, orc), 1e-11, "prescribed")
    sim.close()


def test_tiled_mass_flux_intermediates():
    """Total mass fluxes the tiled cell kernel stores for the dual remap (the
    objects each tile owns, pure and mixed donors) against the oracle's."""
    from parity import max_rel
    pr = P.random_box(31, nx=61, ny=47, nmat=3, velocity=0.3)
    sim, orc = _tiled(pr, lr.FP64), oracle.Oracle(pr)
    _steps(sim, orc, 3)
    for name, f in (("mx", lr.F_MX), ("my", lr.F_MY), ("mc", lr.F_MC), ("fx", lr.F_FX), ("fc", lr.F_FC)):
        assert max_rel(sim.get(f), orc.get(f)) <= 1e-11, name
    sim.close()
