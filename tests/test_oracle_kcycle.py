"""Oracle K-cycle (two FCG iterations as the coarse correction on every
intermediate level, cycle=32: the paper's cycle for the unsmoothed
prolongator, Section 3.2; cycle=c limits that to coarse levels 1..c).

Pins: with two levels there is no intermediate level, so the K-cycle is the
V-cycle bit for bit; on a level whose coarse level has two rows, two flexible
CG steps span R^2 and solve the coarse system exactly, so the K-cycle there
equals the two-grid cycle with an exact coarse solve (computed densely here);
and the K-cycle preconditioner needs fewer outer iterations than the V-cycle
(the reason the paper pairs it with unsmoothed aggregation).
"""
import numpy as np
import pytest

import oracle
from paper_2006_16147_gb300 import workloads as W


def _dense_level(H, l):
    lv = H.level(l)
    A = W.Csr(lv.row_ptr, lv.col, lv.val).to_dense()
    return lv, A


def _two_grid_exact(H, l, b):
    """Pre-smooth, exact coarse solve on level l+1, post-smooth (omega = 1)."""
    lv, A = _dense_level(H, l)
    _, Ac = _dense_level(H, l + 1)
    n, nc = A.shape[0], Ac.shape[0]
    P = np.zeros((n, nc))
    P[np.arange(n), lv.agg] = lv.p
    Minv = np.diag(lv.minv)
    x = Minv @ b
    r = b - A @ x
    x = x + P @ np.linalg.solve(Ac, P.T @ r)
    return x + Minv @ (b - A @ x)


def test_two_levels_k_equals_v():
    A = W.poisson3d(8)
    b = np.random.default_rng(0).normal(size=A.n)
    Hv = oracle.Hierarchy(A)
    Hk = oracle.Hierarchy(A, cycle=32)
    assert Hk.num_levels == 2
    assert np.array_equal(Hv.vcycle(b), Hk.vcycle(b))


@pytest.mark.parametrize("mk,sweeps", [(lambda: W.poisson3d(2, 2, 2), 1), (lambda: W.poisson3d(3, 3, 2), 2),
                                       (lambda: W.poisson2d_aniso(4, 2, 1e-2), 1)])
def test_kcycle_exact_on_two_row_coarse_level(mk, sweeps):
    A = mk()
    H = oracle.Hierarchy(A, sweeps=sweeps, max_coarse=1, min_ratio=1.0, cycle=32)
    sizes = [s[0] for s in H.sizes()]
    l = sizes.index(2) - 1          # the level whose coarse level has two rows
    assert l >= 1 and sizes[l + 1] == 2 and len(sizes) > l + 2     # level l+1 is intermediate
    b = np.random.default_rng(l).normal(size=sizes[l])
    zk = H.vcycle(b, level=l)
    zt = _two_grid_exact(H, l, b)
    assert np.linalg.norm(zk - zt) <= 1e-13 * np.linalg.norm(zt)


def test_vcycle_is_not_exact_there():
    # on the unsymmetric 3x3x2 grid the V-cycle on that level differs from the
    # exact two-grid cycle, so the pin above is not vacuous
    A = W.poisson3d(3, 3, 2)
    H = oracle.Hierarchy(A, sweeps=2, max_coarse=1, min_ratio=1.0)
    sizes = [s[0] for s in H.sizes()]
    l = sizes.index(2) - 1
    b = np.random.default_rng(l).normal(size=sizes[l])
    zt = _two_grid_exact(H, l, b)
    assert np.linalg.norm(H.vcycle(b, level=l) - zt) > 1e-8 * np.linalg.norm(zt)


@pytest.mark.parametrize("mk,mc", [(lambda: W.poisson3d(32), 200), (lambda: W.poisson2d_aniso(96, 80, 1e-2), 40)])
def test_kcycle_needs_fewer_iterations(mk, mc):
    A = mk()
    b = np.random.default_rng(1).normal(size=A.n)
    its = {}
    for cyc in (0, 32):
        H = oracle.Hierarchy(A, cycle=cyc, max_coarse=mc)
        assert H.num_levels >= 3
        x, info = H.pcg(b, rtol=1e-6, flexible=True)
        assert info["status"] == 0
        assert np.linalg.norm(b - A.scipy() @ x) <= 1e-6 * np.linalg.norm(b)
        its[cyc] = info["iterations"]
    assert its[32] < its[0]


def test_kcycle_depth_one_uses_vcycle_below():
    # with the FCG correction on level 1 only, a level-1 cycle is the V-cycle
    # from level 1 (its coarse correction on level 2 is not FCG), bit for bit
    A = W.poisson3d(24)
    H1 = oracle.Hierarchy(A, max_coarse=40, cycle=1)
    Hv = oracle.Hierarchy(A, max_coarse=40)
    assert H1.num_levels >= 4
    r = np.random.default_rng(2).normal(size=H1.sizes()[1][0])
    assert np.array_equal(H1.vcycle(r, level=1), Hv.vcycle(r, level=1))
    r0 = np.random.default_rng(3).normal(size=A.n)
    assert not np.array_equal(H1.vcycle(r0), Hv.vcycle(r0))
