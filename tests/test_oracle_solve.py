"""Pins of the oracle's V-cycle (Eq. 2) and PCG against dense algebra."""
import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W


def _P(n, nc, agg, p):
    P = np.zeros((n, nc))
    P[np.arange(n), agg] = p
    return P


def _dense_B(H, pre=1, post=1):
    """B_0 built from Eq. 2 by dense recursion over the oracle's levels:
    I - B_l A_l = (I - M^-T A)^post (I - P B_{l+1} P^T A) (I - M^-1 A)^pre, B_L = A_L^{-1}."""
    nl = H.num_levels
    levs = [H.level(l) for l in range(nl)]
    dense = [W.Csr(l.row_ptr, l.col, l.val).to_dense() for l in levs]
    B = np.linalg.inv(dense[-1])
    for l in range(nl - 2, -1, -1):
        A = dense[l]
        n = A.shape[0]
        I = np.eye(n)
        Minv = np.diag(levs[l].minv)
        P = _P(n, levs[l + 1].n, levs[l].agg, levs[l].p)
        S_pre = I - Minv @ A
        S_post = I - Minv.T @ A
        E = np.linalg.matrix_power(S_post, post) @ (I - P @ B @ P.T @ A) @ np.linalg.matrix_power(S_pre, pre)
        B = (I - E) @ np.linalg.inv(A)
    return B


CASES = [("poisson", lambda: W.poisson3d(6, 6, 5), None),
         ("spd", lambda: W.random_spd(120, 0.05, 21), 21),
         ("aniso", lambda: W.poisson2d_aniso(12, 10, 1e-2), None)]


def _w(A, seed):
    if seed is None:
        return np.ones(A.n)
    return np.random.default_rng(seed).uniform(0.5, 2.0, A.n)


@pytest.mark.parametrize("name,mk,seed", CASES)
@pytest.mark.parametrize("pre,post", [(1, 1), (2, 2)])
def test_vcycle_matches_dense_error_propagation(orc, name, mk, seed, pre, post):
    A = mk()
    H = orc.Hierarchy(A, _w(A, seed), max_coarse=8, pre=pre, post=post)
    assert H.num_levels >= 3
    B = _dense_B(H, pre, post)
    rng = np.random.default_rng(5)
    for _ in range(3):
        r = rng.normal(size=A.n)
        z = H.vcycle(r)
        assert np.linalg.norm(z - B @ r) <= 1e-12 * np.linalg.norm(B @ r)


@pytest.mark.parametrize("name,mk,seed", CASES)
def test_vcycle_is_spd(orc, name, mk, seed):
    A = mk()
    H = orc.Hierarchy(A, _w(A, seed), max_coarse=8)
    n = A.n
    B = np.column_stack([H.vcycle(e) for e in np.eye(n)])
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    np.linalg.cholesky(0.5 * (B + B.T))


def test_coarse_factor_is_cholesky(orc):
    A = W.random_spd(60, 0.1, 4)
    H = orc.Hierarchy(A, max_coarse=100)
    L = H.coarse_factor()
    assert np.allclose(L, np.linalg.cholesky(A.to_dense()), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("name,mk,seed", CASES)
def test_pcg_matches_dense_solve(orc, name, mk, seed):
    A = mk()
    H = orc.Hierarchy(A, _w(A, seed), max_coarse=8)
    b = np.random.default_rng(9).normal(size=A.n)
    x, info = H.pcg(b, rtol=1e-14, maxit=500)
    xd = np.linalg.solve(A.to_dense(), b)
    assert info["status"] == 0
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_pcg_single_level_is_direct(orc):
    # n <= max_coarse: B = A^{-1}, so PCG converges in one iteration.
    A = W.poisson3d(4, 4, 3)
    H = orc.Hierarchy(A)
    assert H.num_levels == 1
    b = np.random.default_rng(1).normal(size=A.n)
    x, info = H.pcg(b, rtol=1e-12)
    assert info["iterations"] == 1 and info["true_relres"] <= 1e-12


def test_pcg_zero_rhs(orc):
    A = W.poisson3d(6)
    H = orc.Hierarchy(A, max_coarse=8)
    x, info = H.pcg(np.zeros(A.n), x0=np.ones(A.n))
    assert info["iterations"] == 0 and not x.any()


def test_pcg_config1_exact_solution_ones(orc):
    # 32^3 Poisson, b = A*1, x0 = 0, rel-res 1e-6: the error is bounded by
    # cond(A) * relres, and cond(A) < 4 / (6 - 6 cos(pi/33)) ~ 442.
    A = W.poisson3d(32)
    b, xs = W.rhs_ones(A)
    H = orc.Hierarchy(A)
    x, info = H.pcg(b, rtol=1e-6)
    assert info["status"] == 0 and info["true_relres"] <= 1e-6
    assert np.abs(x - xs).max() <= 442 * 1e-6 * np.sqrt(A.n)
    assert 5 <= info["iterations"] <= 60


@pytest.mark.parametrize("name,mk,seed", CASES)
def test_flexible_cg_equals_pcg_for_fixed_preconditioner(orc, name, mk, seed):
    # With a fixed s.p.d. preconditioner z'^T r = 0 in exact arithmetic, so
    # FCG(1)'s beta equals PCG's and the iterates coincide up to rounding.
    A = mk()
    H = orc.Hierarchy(A, _w(A, seed), max_coarse=8)
    b = np.random.default_rng(2).normal(size=A.n)
    x1, i1 = H.pcg(b, rtol=1e-10)
    x2, i2 = H.pcg(b, rtol=1e-10, flexible=True)
    assert i1["status"] == 0 and i2["status"] == 0
    assert abs(i1["iterations"] - i2["iterations"]) <= 1
    xd = np.linalg.solve(A.to_dense(), b)
    assert np.linalg.norm(x2 - xd) <= 1e-8 * np.linalg.norm(xd)
