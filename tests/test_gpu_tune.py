"""Autotuned launch shapes (options.autotune).

A launch shape only changes which thread handles which rows: every row of a
SELL sweep or restriction is computed by one lane in a fixed order, and the
reducing kernels keep their fixed grid. So a V-cycle and a PCG solve give the
same bits with and without tuning. For block solves the lanes per row change
the rows each block reduces, so per-column dot products may differ in the
last bits: iteration counts within +-1 and residuals below the tolerance.
"""
import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W

from gpu_util import dev, setup, solve, vcycle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_tuned_vcycle_and_pcg_bitwise_equal(precision):
    from paper_2006_16147_gb300 import amg
    amg.amg_tune_clear()
    A = W.poisson3d(40, 33, 21)
    b, _ = W.rhs_uniform(A, 1)
    h0 = setup(A, precision=precision, max_coarse=40)
    n0 = amg.amg_tune_size()
    h1 = setup(A, precision=precision, max_coarse=40, autotune=1)
    nlev = amg.amg_hierarchy_info(h1)["num_levels"]
    assert amg.amg_tune_size() - n0 == 3 * (nlev - 1)       # pre, post, restriction per level
    r = np.random.default_rng(3).normal(size=A.n)
    assert np.array_equal(vcycle(h0, r), vcycle(h1, r))
    x0, i0 = solve(h0, b)
    x1, i1 = solve(h1, b)
    assert i0["iterations"] == i1["iterations"] and np.array_equal(x0, x1)
    # a second hierarchy of the same shape reuses the cache: nothing new timed
    before = amg.amg_tune_size()
    h2 = setup(A, precision=precision, max_coarse=40, autotune=1)
    assert amg.amg_tune_size() == before
    assert np.array_equal(vcycle(h2, r), vcycle(h1, r))
    for h in (h0, h1, h2):
        h.close()


def test_tuned_cache_round_trip_applies(tmp_path):
    from paper_2006_16147_gb300 import amg
    amg.amg_tune_clear()
    A = W.poisson3d(24)
    h = setup(A, autotune=1)
    f = tmp_path / "tune.txt"
    amg.amg_tune_save(str(f))
    saved = f.read_text().splitlines()
    assert len(saved) == amg.amg_tune_size() > 0
    for line in saved:
        key, val = line.split()
        assert int(val) >= 1 and "/sm" in key
    amg.amg_tune_clear()
    amg.amg_tune_load(str(f))
    h2 = setup(A, autotune=1)
    assert amg.amg_tune_size() == len(saved)
    r = np.random.default_rng(1).normal(size=A.n)
    assert np.array_equal(vcycle(h, r), vcycle(h2, r))
    h.close()
    h2.close()


@pytest.mark.parametrize("k", [5, 64])
def test_tuned_block_solve(k):
    import torch
    from paper_2006_16147_gb300 import amg
    amg.amg_tune_clear()
    A = W.poisson3d(28, 24, 20)
    B = W.rhs_normal(A.n, seed=4, k=k)
    res = {}
    for tune in (0, 1):
        h = setup(A, precision=1, autotune=tune)
        X = torch.zeros(A.n, k, dtype=torch.float64, device="cuda:0")
        infos = amg.amg_solve_batch(h, dev(B), X, rtol=1e-6)
        Xh = X.cpu().numpy()
        R = B - A.scipy() @ Xh
        assert np.all(np.linalg.norm(R, axis=0) <= 1e-6 * np.linalg.norm(B, axis=0))
        res[tune] = [i["iterations"] for i in infos]
        h.close()
    assert all(abs(a - c) <= 1 for a, c in zip(res[0], res[1]))
    assert any(key.startswith("block/") for key in _keys())


def _keys():
    import os
    import tempfile
    from paper_2006_16147_gb300 import amg
    fd, path = tempfile.mkstemp()
    os.close(fd)
    try:
        amg.amg_tune_save(path)
        return [line.split()[0] for line in open(path).read().splitlines()]
    finally:
        os.remove(path)


def test_tuned_many_systems():
    import torch
    from paper_2006_16147_gb300 import amg
    mats = [W.poisson3d(e) for e in (9, 14, 6, 11)]
    U, offs = W.block_diagonal(mats)
    b = np.random.default_rng(2).normal(size=U.n)
    xs = []
    for tune in (0, 1):
        systems = [(dev(M.row_ptr), dev(M.col), dev(M.val), dev(np.ones(M.n))) for M in mats]
        h = amg.amg_setup_many(systems, autotune=tune)
        x = torch.zeros(U.n, dtype=torch.float64, device="cuda:0")
        amg.amg_solve_many(h, dev(b), x, len(mats))
        xs.append(x.cpu().numpy())
        h.close()
    assert np.array_equal(xs[0], xs[1])
