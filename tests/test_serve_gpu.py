"""The serving loop (include/lr_serve.h): requests arriving while others run
are admitted as pool units free up, overlap on the device, and each result
is the same as the request run alone (bit-identical in FP64)."""
import time

import numpy as np
import pytest

from paper_2208_13409_gb300 import lr, problems as P
from parity import max_rel

pytestmark = pytest.mark.gpu


def _alone(pr, nsteps):
    sim = lr.Sim(pr)
    sim.run(nsteps)
    return sim


def _check_same(srv, rid, pr, nsteps):
    sim = _alone(pr, nsteps)
    for f in lr.SERVE_FIELDS:
        d = max_rel(srv.result(rid, f), sim.get(f))
        assert d == 0.0, (rid, f, d)


def test_alone_equals_mix_with_queueing_and_overlap():
    sides = [48, 64, 40, 72, 56, 32, 64, 48]
    probs = [P.air_water(300 + q, side=s, steps_range=(15, 60)) for q, s in enumerate(sides)]
    units = lr.batch_units(probs[1]) + lr.batch_units(probs[3]) + 64   # room for about two at once
    srv = lr.Server(units, 4, max_member_cells=max(p.cells for p in probs), max_chunk_steps=8)
    ids = []
    for q, pr in enumerate(probs):
        ids.append(srv.submit(pr, max_steps=pr.steps))
        if q == 3:
            time.sleep(0.05)  # later arrivals join a running batch
    assert srv.drain(timeout=300.0)
    info = [srv.info(r) for r in ids]
    for r, pr, inf in zip(ids, probs, info):
        assert srv.wait(r, 0.0) == 1
        assert inf["steps"] == pr.steps
        _check_same(srv, r, pr, pr.steps)
    # queueing happened (the pool held about two) and requests overlapped
    assert any(inf["admit"] > min(i["done"] for i in info) for inf in info)
    overlap = any(a["admit"] < b["admit"] < a["done"] for a in info for b in info if a is not b)
    assert overlap
    st = srv.stats()
    assert st["completed"] == len(probs) and st["failed"] == 0 and st["pending"] == 0
    assert st["cell_updates"] == sum(p.cells * p.steps for p in probs)
    srv.close()


def test_refusals_and_failures_stay_local():
    good = P.air_water(401, side=40, steps_range=(10, 20))
    srv = lr.Server(3 * lr.batch_units(good), 3, max_member_cells=64 * 64)
    with pytest.raises(lr.LrError):          # can never fit this pool
        srv.submit(P.air_water(402, side=200))
    bad = good.copy()
    bad.rho[1][bad.k[1] > 0] = -1.0           # invalid initial state
    rb = srv.submit(bad, max_steps=5)
    rg = srv.submit(good, max_steps=good.steps)
    assert srv.wait(rb, 60.0) == lr.FAILED
    assert srv.wait(rg, 60.0) == lr.DONE
    _check_same(srv, rg, good, good.steps)
    srv.release(rg)
    with pytest.raises(lr.LrError):
        srv.result(rg, lr.F_K)
    srv.close()
