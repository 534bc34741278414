"""Checkpoint and resume: N steps, lr_checkpoint_save, lr_checkpoint_load
(into a fresh context, or back into the same one), N steps equal 2N steps
bit for bit, in every arithmetic mode and in the tiled step.  Restarting
through lr_get_fields + lr_init instead re-derives the energies from the
pressures and the sound speeds from the state, so it agrees with the
continued run to round-off only."""
import numpy as np
import pytest

from paper_2208_13409_gb300 import lr, problems as P
from parity import compare, max_rel

pytestmark = pytest.mark.gpu

FIELDS = (lr.F_K, lr.F_RHO_MAT, lr.F_E_MAT, lr.F_UX, lr.F_UY)


def _state(sim):
    return [sim.get(f) for f in FIELDS] + [np.array([sim.t, sim.dt_next()])]


@pytest.mark.parametrize("prec,tiled", [(lr.FP64, False), (lr.DF64, False), (lr.FP32, True), (lr.FP32, False),
                                        (lr.FP64, True)])
def test_checkpoint_resume_is_bitwise(prec, tiled):
    pr = P.triple_point(140, 60)
    n = 15
    a = lr.Sim(pr, precision=prec)
    a.set_tiled(tiled)
    for _ in range(2 * n):
        a.step()
    ref = _state(a)
    b = lr.Sim(pr, precision=prec)
    b.set_tiled(tiled)
    for _ in range(n):
        b.step()
    buf = b.checkpoint()
    # a fresh context resumes from the checkpoint
    c = lr.Sim(pr, precision=prec)
    c.set_tiled(tiled)
    c.restore(buf)
    for _ in range(n):
        c.step()
    for x, y in zip(_state(c), ref):
        assert np.array_equal(x, y)
    # the same context rewinds to the checkpoint
    for _ in range(n):
        b.step()
    for _ in range(3):
        b.step()
    b.restore(buf)
    for _ in range(n):
        b.step()
    for x, y in zip(_state(b), ref):
        assert np.array_equal(x, y)
    for s in (a, b, c):
        s.close()


def test_checkpoint_rejects_other_configuration():
    pr = P.triple_point(140, 60)
    a = lr.Sim(pr)
    a.step()
    buf = a.checkpoint()
    other = lr.Sim(P.triple_point(70, 30))
    with pytest.raises(lr.LrError):
        other.restore(buf)
    other32 = lr.Sim(pr, precision=lr.FP32)
    with pytest.raises(lr.LrError):
        other32.restore(buf)
    with pytest.raises(lr.LrError):
        a.restore(buf[:100])
    for s in (a, other, other32):
        s.close()


def test_restart_through_fields_and_init_matches_to_roundoff():
    """The restart a user can write with lr_get_fields and lr_init (pressures
    from the EOS, velocities as stored): the next N steps match the
    continued run to the FP64 parity bar."""
    pr = P.triple_point(140, 60)
    n = 10
    a = lr.Sim(pr)
    for _ in range(n):
        a.step()
    k, r, e = a.get(lr.F_K), a.get(lr.F_RHO_MAT), a.get(lr.F_E_MAT)
    g = pr.gamma[:, None, None]
    pi = pr.pinf[:, None, None]
    present = k > 0
    p = np.where(present, (g - 1.0) * r * e - pi, 1.0)
    restart = pr.copy(k=k, rho=np.where(present, r, 1.0), p=p, ux=a.get(lr.F_UX), uy=a.get(lr.F_UY))
    b = lr.Sim(restart)
    for _ in range(n):
        a.step()
        b.step()
    bad = {key: v for key, v in compare(b, a).items() if not (v <= 1e-11)}
    assert not bad, bad
    a.close()
    b.close()
