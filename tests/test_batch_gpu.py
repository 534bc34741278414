"""The batched step (include/lr_batch.h) against lone simulations and the
oracle: every member's result is the same alone and in any mix (same
arithmetic, its own CFL time step), in the persistent step (one cooperative
launch per step, the tiled step's tile functions; compared with lone tiled
runs) and in the per-kernel step (one launch per kernel and group, under
every schedule the autotuner can pick; compared with lone unfused runs),
across admission, removal, step limits and t_end.  The persistent step's
barriers give up after their limit with LR_ERR_TIMEOUT."""
import numpy as np
import pytest

import oracle
from paper_2208_13409_gb300 import lr, problems as P
from parity import compare, l1_rel, max_rel

pytestmark = pytest.mark.gpu

FIELDS = (lr.F_K, lr.F_RHO_MAT, lr.F_E_MAT, lr.F_UX, lr.F_UY, lr.F_P)


def _mix():
    return [
        P.random_box(101, nx=40, ny=33, nmat=2, velocity=0.3),
        P.random_box(102, nx=64, ny=64, nmat=3, velocity=0.2),
        P.uniform(23, 17, rho=1.3, p=0.7, u=(0.2, -0.1)),
        P.random_box(103, nx=21, ny=50, nmat=3, velocity=0.4).copy(bc=(P.BC_PERIODIC,) * 4),
        P.random_box(104, nx=96, ny=30, nmat=2, velocity=0.25).copy(
            bc=(P.BC_PERIODIC, P.BC_PERIODIC, P.BC_REFLECT, P.BC_REFLECT)),
        P.triple_point(70, 30),
    ]


def _units(probs):
    return sum(lr.batch_units(p) for p in probs)


def _alone(pr, nsteps, precision=lr.FP64, tiled=False):
    """The problem run alone, on the path the batch runs: the tiled step for
    a persistent batch, the unfused one otherwise."""
    sim = lr.Sim(pr, precision=precision)
    sim.set_tiled(tiled)
    for _ in range(nsteps):
        sim.step(1e300, sync=False)
    sim.sync()
    return sim


def _same(bt, m, sim, tol=0.0, tol_l1=0.0):
    worst = worst_l1 = 0.0
    for f in FIELDS:
        a, b = bt.get(m, f), sim.get(f)
        worst = max(worst, max_rel(a, b))
        worst_l1 = max(worst_l1, l1_rel(a, b))
    assert worst <= tol and worst_l1 <= tol_l1, (m, worst, worst_l1)
    return worst


# FP64 and double-float members are bit-identical to lone runs.  In the FP32
# bulk mode the compiler may fuse float multiply-adds differently in the
# batched and the lone instantiation of a kernel: the two start 1 float ulp
# apart and that grows over the steps (a limiter or threshold decision can
# flip), still far inside the FP32 mode's own error against the FP64 oracle.
TOL_ALONE = {lr.FP64: 0.0, lr.DF64: 0.0, lr.FP32: 1e-3}
TOL_ALONE_L1 = {lr.FP64: 0.0, lr.DF64: 0.0, lr.FP32: 1e-5}
# The persistent step and the lone tiled kernels run the same tile functions;
# in double-float arithmetic (float operations) the two instantiations may
# also contract differently, so those members agree to the FP64 parity bar.
TOL_ALONE_PERSIST = {lr.FP64: 0.0, lr.DF64: 1e-11, lr.FP32: 1e-3}
TOL_ALONE_PERSIST_L1 = {lr.FP64: 0.0, lr.DF64: 1e-12, lr.FP32: 1e-5}


@pytest.mark.parametrize("persistent", [True, False])
@pytest.mark.parametrize("prec", [lr.FP64, lr.DF64, lr.FP32])
def test_members_equal_alone(prec, persistent):
    probs = _mix()
    bt = lr.Batch(_units(probs), 8, precision=prec)
    bt.set_persistent(persistent)
    assert bt.persistent == persistent
    ids = [bt.add(p, t_end=1e300) for p in probs]
    assert all(i is not None for i in ids)
    bt.step(12)
    bt.sync()
    assert bt.launches_per_step() == (1 if persistent else bt.launches_per_step())
    for pr, m in zip(probs, ids):
        t, n, st = bt.status(m)
        assert n == 12 and st == lr.RUNNING
        sim = _alone(pr, 12, prec, tiled=persistent)
        tol = TOL_ALONE_PERSIST if persistent else TOL_ALONE
        tol_l1 = TOL_ALONE_PERSIST_L1 if persistent else TOL_ALONE_L1
        assert t == pytest.approx(sim.t, rel=tol_l1[prec], abs=0.0)
        _same(bt, m, sim, tol[prec], tol_l1[prec])


@pytest.mark.parametrize("persistent", [True, False])
def test_members_match_oracle(persistent):
    probs = [P.random_box(111, nx=30, ny=26, nmat=3, velocity=0.3), P.sod(nx=64), P.triple_point(70, 30)]
    bt = lr.Batch(_units(probs), 4)
    bt.set_persistent(persistent)
    ids = [bt.add(p, t_end=1e300) for p in probs]
    orcs = [oracle.Oracle(p) for p in probs]
    for q in range(5):
        bt.step(1)
        for o in orcs:
            o.step()
    for pr, m, o in zip(probs, ids, orcs):
        sim_like = _BatchMember(bt, m, pr)
        res = compare(sim_like, o)
        bad = {k: v for k, v in res.items() if not v <= 1e-10}
        assert not bad, (pr.name, bad)


class _BatchMember:
    """The Sim interface compare() uses, for one batch member."""

    def __init__(self, bt, m, pr):
        self.bt, self.m, self.p = bt, m, pr

    def get(self, f):
        return self.bt.get(self.m, f)


def test_step_limit_and_t_end():
    a = P.random_box(121, nx=32, ny=32, nmat=2, velocity=0.3)
    b = P.random_box(122, nx=48, ny=40, nmat=3, velocity=0.3)
    c = P.sod(nx=64)
    bt = lr.Batch(_units([a, b, c]), 4)
    ma = bt.add(a, t_end=1e300, max_steps=5)
    mb = bt.add(b, t_end=1e300)
    sim_c = lr.Sim(c)
    sim_c.run(7)
    t7 = sim_c.t
    mc = bt.add(c, t_end=t7)
    bt.step(11)
    bt.sync()
    t, n, st = bt.status(ma)
    assert (n, st) == (5, lr.DONE)
    _same(bt, ma, _alone(a, 5, tiled=bt.persistent))
    t, n, st = bt.status(mb)
    assert (n, st) == (11, lr.RUNNING)
    _same(bt, mb, _alone(b, 11, tiled=bt.persistent))
    t, n, st = bt.status(mc)
    assert st == lr.DONE and n == 7 and t == t7
    sim_c2 = lr.Sim(c)   # the same t_end caps the last step alone too
    sim_c2.set_tiled(bt.persistent)
    for _ in range(9):
        sim_c2.step(t7)
    assert sim_c2.t == t7
    _same(bt, mc, sim_c2)


def test_admission_by_pool_units_and_reuse():
    a = P.random_box(131, nx=40, ny=40, nmat=2, velocity=0.2)
    b = P.random_box(132, nx=30, ny=20, nmat=3, velocity=0.2)
    c = P.random_box(133, nx=36, ny=36, nmat=2, velocity=0.2)
    cap = lr.batch_units(a) + lr.batch_units(b)
    bt = lr.Batch(cap, 4)
    ma = bt.add(a, t_end=1e300)
    mb = bt.add(b, t_end=1e300)
    assert bt.add(c, t_end=1e300) is None        # does not fit now
    bt.step(3)
    bt.remove(ma)                                # frees a's range
    mc = bt.add(c, t_end=1e300)                  # fits in it
    assert mc is not None
    bt.step(4)
    bt.sync()
    _same(bt, mb, _alone(b, 7, tiled=bt.persistent))
    _same(bt, mc, _alone(c, 4, tiled=bt.persistent))
    # slots: a batch of one member slot admits one member
    bt1 = lr.Batch(10 * cap, 1)
    assert bt1.add(a) is not None and bt1.add(b) is None


def test_autotune_keeps_results_and_state():
    probs = _mix()
    bt = lr.Batch(_units(probs), 8)
    ids = [bt.add(p, t_end=1e300) for p in probs]
    bt.step(2)
    bt.autotune(trial_steps=2)
    shapes, bps, lanes = bt.schedule()
    assert len(shapes) == 9 and lanes in (2, 4, 8)
    for m in ids:
        assert bt.status(m)[1] == 2               # trial steps were rolled back
    bt.step(6)
    bt.sync()
    for pr, m in zip(probs, ids):
        _same(bt, m, _alone(pr, 8, tiled=bt.persistent))


def test_persistent_default_by_arithmetic():
    """The persistent step is the default where it is the faster path
    (FP32); FP64 and double-float batches start with one launch per kernel."""
    probs = _mix()
    for prec, want in ((lr.FP32, True), (lr.FP64, False), (lr.DF64, False)):
        bt = lr.Batch(_units(probs), 8, precision=prec)
        assert bt.persistent == want, prec
        bt.close()


@pytest.mark.parametrize("on", [True, False])
def test_autotune_keeps_an_explicit_step_path(on):
    """The autotuner chooses between the per-kernel and the persistent step
    only when the caller has not set one."""
    probs = _mix()
    bt = lr.Batch(_units(probs), 8, precision=lr.FP32)
    bt.set_persistent(on)
    ids = [bt.add(p, t_end=1e300) for p in probs]
    bt.step(1)
    bt.autotune(trial_steps=1)
    assert bt.persistent == on
    for m in ids:
        assert bt.status(m)[1] == 1
    bt.close()


def test_invalid_member_is_refused_and_failure_stays_local():
    good = P.random_box(141, nx=32, ny=24, nmat=2, velocity=0.3)
    bad = good.copy()
    bad.k[0, 3, 3] = 0.6  # sum k != 1
    bt = lr.Batch(3 * lr.batch_units(good), 3)
    mg = bt.add(good, t_end=1e300)
    with pytest.raises(lr.LrError):
        bt.add(bad, t_end=1e300)
    # a member that tangles: fixed dt far above the CFL limit
    wild = P.random_box(142, nx=32, ny=24, nmat=2, velocity=0.9).copy(dt_fixed=0.5)
    mw = bt.add(wild, t_end=1e300)
    bt.step(6)
    bt.sync()
    assert bt.status(mw)[2] == lr.FAILED
    _same(bt, mg, _alone(good, 6, tiled=bt.persistent))


def test_persistent_is_one_launch_per_step():
    probs = _mix()
    bt = lr.Batch(_units(probs), 8, precision=lr.FP32)
    assert bt.persistent  # the default
    for p in probs:
        bt.add(p, t_end=1e300)
    bt.step(3)
    bt.sync()
    assert bt.launches_per_step() == 1
    bt.set_persistent(False)
    bt.step(1)
    bt.sync()
    assert bt.launches_per_step() > 1


def test_persistent_barrier_limit_runs_out():
    """A barrier waiting for an arrival no block makes gives up after its
    limit: the step is abandoned and reported as LR_ERR_TIMEOUT, the device
    stays usable (a fresh batch steps normally afterwards)."""
    import time
    probs = _mix()[:3]
    bt = lr.Batch(_units(probs), 4)
    bt.set_persistent(True)
    for p in probs:
        bt.add(p, t_end=1e300)
    bt.step(2)
    bt.sync()
    bt.test_barrier(1, 0.2)
    t0 = time.perf_counter()
    bt.step(1)
    with pytest.raises(lr.LrError) as ei:
        bt.sync()
    assert ei.value.status == lr.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(lr.LrError):        # the batch stays in error
        bt.step(1)
    bt.close()
    fresh = lr.Batch(_units(probs), 4)
    fresh.set_persistent(True)
    ids = [fresh.add(p, t_end=1e300) for p in probs]
    fresh.step(2)
    fresh.sync()
    for pr, m in zip(probs, ids):
        _same(fresh, m, _alone(pr, 2, tiled=True))
