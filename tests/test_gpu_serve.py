"""Solve server: continuous batching over cached hierarchies.

Requests arrive while others are on the GPU and are admitted as slots free
up. Every result must be the same as the same request served alone: the
server fixes the per-row lane width, so a column's arithmetic does not depend
on the other columns in flight, and the comparison is exact."""
import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W

from gpu_util import setup

pytestmark = pytest.mark.gpu


def _hierarchies():
    mats = [W.poisson3d(24), W.poisson2d_aniso(96, 80, 1e-2), W.varcoef3d(24, seed=2)]
    hs = [setup(mats[0], precision=1), setup(mats[1], precision=1), setup(mats[2], precision=1, krylov=1)]
    return mats, hs


def _drain(srv, done):
    while True:
        pending = srv.step()
        for r in srv.poll():
            done[r["id"]] = r
        if pending == 0:
            return


def test_continuous_batching_mix_equals_alone():
    from paper_2006_16147_gb300 import amg
    mats, hs = _hierarchies()
    rng = np.random.default_rng(6)
    reqs = []
    for t in range(24):
        hid = int(rng.integers(0, 3))
        k = int(rng.integers(1, 7))
        reqs.append((hid, W.rhs_normal(mats[hid].n, 100 + t, k)))
    srv = amg.Server(hs, slots=16, rtol=1e-6)
    ids, done = [], {}
    # arrivals in waves while earlier requests are still iterating
    for wave in range(0, 24, 6):
        for hid, B in reqs[wave:wave + 6]:
            ids.append(srv.submit(hid, B)[0])
        for _ in range(3):
            srv.step()
            for r in srv.poll():
                done[r["id"]] = r
    _drain(srv, done)
    st = srv.stats()
    assert st["completed"] == 24 and st["columns_completed"] == sum(B.shape[1] for _, B in reqs)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()
    for (hid, B), rid in zip(reqs, ids):
        r = done[rid]
        assert r["status"] == 0 and r["relres"] <= 1e-6
        S = mats[hid].scipy()
        for c in range(B.shape[1]):
            assert np.linalg.norm(B[:, c] - S @ r["X"][:, c]) <= 1e-6 * np.linalg.norm(B[:, c])
    # the same requests served one at a time by a fresh server: identical results
    for (hid, B), rid in list(zip(reqs, ids))[::5]:
        alone = amg.Server(hs, slots=16, rtol=1e-6)
        aid, X = alone.submit(hid, B)
        got = {}
        _drain(alone, got)
        alone.close()
        assert np.array_equal(got[aid]["X"], done[rid]["X"])
        assert got[aid]["iterations"] == done[rid]["iterations"]
    for h in hs:
        h.close()


def test_budget_limits_columns_in_flight():
    from paper_2006_16147_gb300 import amg
    mats, hs = _hierarchies()
    rng = np.random.default_rng(2)
    budget = 3 * 1024 * 1024 * 8     # room for a few columns at a time
    srv = amg.Server(hs, slots=8, budget_bytes=budget, rtol=1e-6)
    ids = []
    reqs = []
    for t in range(10):
        hid = int(rng.integers(0, 3))
        reqs.append((hid, W.rhs_normal(mats[hid].n, 200 + t, int(rng.integers(1, 3)))))
    for hid, B in reqs:
        ids.append(srv.submit(hid, B)[0])
    done = {}
    _drain(srv, done)
    st = srv.stats()
    assert st["completed"] == 10 and st["peak_bytes"] <= budget
    with pytest.raises(amg.AmgError) as e:
        srv.submit(0, np.ones((mats[0].n, 9)))          # more columns than slots
    assert e.value.status == -8
    tiny = amg.Server(hs, slots=8, budget_bytes=1024)
    with pytest.raises(amg.AmgError) as e:
        tiny.submit(0, np.ones((mats[0].n, 1)))        # above the budget
    assert e.value.status == -9
    tiny.close()
    srv.close()
    for h in hs:
        h.close()
