"""Pins of the oracle's aggregates and prolongator (Eq. 4), Galerkin products
(Section 3.1), level loop and stop rule (Sections 3.2, 5), against dense
algebra and the paper's own hierarchy numbers."""
import os

import numpy as np
import pytest
import scipy.linalg as sl

from paper_2006_16147_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _P(n, nc, agg, p):
    P = np.zeros((n, nc))
    P[np.arange(n), agg] = p
    return P


CASES = [("poisson", lambda: W.poisson3d(6, 5, 4), None),
         ("spd1", lambda: W.random_spd(48, 0.12, 11), 11),
         ("spd2", lambda: W.random_spd(64, 0.08, 12), 12),
         ("aniso", lambda: W.poisson2d_aniso(8, 6, 1e-2), None)]


def _w(A, seed):
    if seed is None:
        return np.ones(A.n)
    rng = np.random.default_rng(seed)
    return rng.uniform(0.3, 2.0, A.n) * rng.choice([-1.0, 1.0], A.n)


@pytest.mark.parametrize("name,mk,seed", CASES)
def test_pairwise_sweeps_partition_and_P(orc, name, mk, seed):
    A = mk()
    w = _w(A, seed)
    H = orc.Hierarchy(A, w, sweeps=3, max_coarse=4, max_levels=3)
    lv = H.level(0)
    wcur = w
    for s in lv.sweeps:
        agg, p, nc = s["agg"], s["p"], s["nc"]
        # partition: every index in one aggregate of 1 or 2, ids numbered by min member
        counts = np.bincount(agg, minlength=nc)
        assert counts.min() >= 1 and counts.max() <= 2 and counts.sum() == s["n"]
        first = np.full(nc, -1)
        for i in range(s["n"]):
            if first[agg[i]] < 0:
                first[agg[i]] = i
        assert np.all(np.diff(first) > 0)
        mate = s["mate"]
        for i in range(s["n"]):
            j = mate[i]
            assert (counts[agg[i]] == 2) == (j >= 0)
            if j >= 0:
                assert agg[j] == agg[i]
        P = _P(s["n"], nc, agg, p)
        # orthonormal columns; range(P) contains w and P w_c = w
        assert np.allclose(P.T @ P, np.eye(nc), atol=4e-16 * 4)
        assert np.allclose(P @ s["wc"], wcur, rtol=1e-15, atol=1e-15 * np.abs(wcur).max())
        wcur = s["wc"]


@pytest.mark.parametrize("name,mk,seed", CASES)
def test_galerkin_equals_dense_product(orc, name, mk, seed):
    A = mk()
    w = _w(A, seed)
    H = orc.Hierarchy(A, w, sweeps=3, max_coarse=2, max_levels=4)
    for l in range(H.num_levels - 1):
        lv = H.level(l)
        Al = W.Csr(lv.row_ptr, lv.col, lv.val).to_dense()
        # sweep by sweep: A^(s+1) = P_s^T A^(s) P_s
        Acur = Al
        for s in lv.sweeps:
            P = _P(s["n"], s["nc"], s["agg"], s["p"])
            Acur = P.T @ Acur @ P
        nxt = H.level(l + 1)
        Anext = W.Csr(nxt.row_ptr, nxt.col, nxt.val).to_dense()
        scale = np.abs(Anext).max()
        assert np.abs(Anext - Acur).max() <= 1e-14 * scale * 4
        assert np.abs(Anext - Anext.T).max() <= 1e-14 * scale * 4
        # the level prolongator is the product of the pairwise ones
        Pl = _P(lv.n, nxt.n, lv.agg, lv.p)
        assert np.abs(Anext - Pl.T @ Al @ Pl).max() <= 1e-13 * scale
        counts = np.bincount(lv.agg, minlength=nxt.n)
        assert counts.max() <= 2 ** len(lv.sweeps)
        # the stored pattern holds every nonzero of the dense product
        pattern = np.zeros_like(Anext, dtype=bool)
        rows = np.repeat(np.arange(nxt.n), np.diff(nxt.row_ptr))
        pattern[rows, nxt.col] = True
        assert not np.any((np.abs(Acur) > 0) & ~pattern)


@pytest.mark.parametrize("row", _read_golden("paper_hierarchy_table.txt"))
def test_paper_hierarchy_80cubed(orc, row):
    sweeps, nl, cr, coarsest, opc = int(row[0]), int(row[1]), float(row[2]), int(row[3]), float(row[4])
    A = W.poisson3d(80)
    H = orc.Hierarchy(A, sweeps=sweeps, max_coarse=200)
    sizes = H.sizes()
    assert len(sizes) == nl
    assert sizes[-1][0] == coarsest
    ratios = [sizes[i][0] / sizes[i + 1][0] for i in range(nl - 1)]
    assert round(float(np.mean(ratios)), 2) == cr
    got_opc = sum(s[1] for s in sizes) / sizes[0][1]
    assert round(got_opc, 3) == opc


def test_stop_rule_and_max_levels(orc):
    A = W.poisson3d(32)
    H = orc.Hierarchy(A)
    assert [s[0] for s in H.sizes()] == [32768, 4096, 512, 64]
    H = orc.Hierarchy(A, max_coarse=512)
    assert [s[0] for s in H.sizes()] == [32768, 4096, 512]
    H = orc.Hierarchy(W.poisson3d(16), max_levels=2)
    assert [s[0] for s in H.sizes()] == [4096, 512]
    small = W.poisson3d(5)
    H = orc.Hierarchy(small)
    assert H.num_levels == 1


def test_l1_jacobi_diagonal(orc):
    A = W.random_spd(30, 0.2, 3)
    H = orc.Hierarchy(A, max_coarse=1000)
    d = A.to_dense()
    m = np.abs(d).sum(1)       # a_ii > 0, so a_ii + sum_{j != i} |a_ij| = row sum of |a|
    assert np.allclose(H.level(0).minv, 1.0 / m, rtol=1e-15)


def _gold_K():
    return {r[0]: (float(r[1]), float(r[2])) for r in _read_golden("paper_table1_K.txt")}


@pytest.mark.slow
def test_paper_table1_convergence_constant(orc):
    # Eq. 7 on the 16^3 Laplacian with the two-level prolongator of the oracle.
    A = W.poisson3d(16)
    n = A.n
    H = orc.Hierarchy(A, max_levels=2)
    lv = H.level(0)
    nc = H.sizes()[1][0]
    assert nc == 512
    P = _P(n, nc, lv.agg, lv.p)
    Ad = A.to_dense()
    D = np.diag(np.diag(Ad))
    S = sl.null_space(P.T @ D)            # columns span ker R, R = (P^T D P)^{-1} P^T D
    SAS = S.T @ Ad @ S

    def K(Mbar):
        SMS = S.T @ Mbar @ S
        SMS = 0.5 * (SMS + SMS.T)
        return 1.0 / sl.eigh(SAS, SMS, eigvals_only=True, subset_by_index=[0, 0])[0]

    gold = _gold_K()
    M = np.tril(Ad)                       # HGS at np = 1 is Gauss-Seidel
    Mbar = M.T @ np.linalg.solve(M.T + M - Ad, M)
    assert abs(K(Mbar) - gold["HGS"][0]) <= gold["HGS"][1]
    Ml1 = np.diag(1.0 / lv.minv)          # the oracle's l1-Jacobi matrix
    assert abs(K(Ml1) - gold["l1-Jacobi"][0]) <= gold["l1-Jacobi"][1]


def _star(n, seed=0):
    # hub 0 joined to every leaf, leaves not joined to each other; SPD by
    # diagonal dominance. Any matching of a star has exactly one pair.
    rng = np.random.default_rng(seed)
    d = np.zeros((n, n))
    off = -rng.uniform(0.1, 1.0, n - 1)
    d[0, 1:] = off
    d[1:, 0] = off
    d[0, 0] = np.abs(off).sum() + 1.0
    d[np.arange(1, n), np.arange(1, n)] = np.abs(off) + rng.uniform(0.5, 1.0, n - 1)
    rows, cols = np.nonzero(d)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    return W.Csr(np.cumsum(rp), cols, d[rows, cols])


def test_stalled_coarsening_stops(orc):
    A = _star(300)
    H = orc.Hierarchy(A, max_coarse=10, sweeps=1)
    # one sweep matches one pair: 300 -> 299 is a ratio below 1.5, so the
    # second level is the last one
    assert [s[0] for s in H.sizes()] == [300, 299]
    H = orc.Hierarchy(A, max_coarse=10, sweeps=1, min_ratio=1.0)
    assert H.num_levels > 2
    # the Laplacian's ratio of 8 is far from the stall rule
    assert [s[0] for s in orc.Hierarchy(W.poisson3d(32)).sizes()] == [32768, 4096, 512, 64]


def test_coarsest_cg_reaches_its_tolerance(orc):
    # coarsest level above max_dense: CG with l1-Jacobi to 1e-4 (Section 5's
    # coarsest-solver setting); on a single level B b is that CG's result
    A = W.poisson3d(10)
    H = orc.Hierarchy(A, max_coarse=2000, max_dense=100)
    assert H.num_levels == 1 and H.coarse_is_cg
    b = np.random.default_rng(3).normal(size=A.n)
    x = H.vcycle(b)
    assert np.linalg.norm(b - A.scipy() @ x) <= 1e-4 * np.linalg.norm(b)
    # and it is a CG iterate, not the exact solution
    assert np.linalg.norm(b - A.scipy() @ x) > 1e-10 * np.linalg.norm(b)


def test_three_sweeps_on_even_grid_give_2x2x2_cubes():
    # Equal weights and the index tiebreak pair along x, then along y on the
    # pairs' graph, then along z: every level-0 aggregate is a 2 x 2 x 2 cube
    import oracle
    oracle.build()
    nx, ny, nz = 8, 6, 4
    A = W.poisson3d(nx, ny, nz)
    H = oracle.Hierarchy(A, max_coarse=1, max_levels=2)
    agg = H.level(0).agg
    idx = np.arange(A.n)
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    cube = (i // 2) + (nx // 2) * ((j // 2) + (ny // 2) * (k // 2))
    assert H.sizes()[1][0] == A.n // 8
    # the same partition (numbering aside): each cube is one aggregate and vice versa
    pairs = set(zip(cube.tolist(), agg.tolist()))
    assert len(pairs) == A.n // 8 == len(set(agg.tolist()))
    assert np.allclose(H.level(0).p, 1.0 / np.sqrt(8.0), rtol=1e-15, atol=0)


def test_coarse_laplacian_is_half_the_coarse_grid_laplacian():
    # with 2 x 2 x 2 cubes and p = 1/sqrt(8), P^T A P has diagonal
    # (8 * 6 - 2 * 12) / 8 = 3 and -4/8 towards each face neighbour: half
    # the 7-point operator of the coarse grid, boundary rows included
    import oracle
    oracle.build()
    nx, ny, nz = 8, 6, 4
    A = W.poisson3d(nx, ny, nz)
    H = oracle.Hierarchy(A, max_coarse=1, max_levels=2)
    C = H.level_csr(1)
    ref = W.poisson3d(nx // 2, ny // 2, nz // 2)
    agg = H.level(0).agg
    # coarse numbering: aggregate of the cube with the smallest member first
    idx = np.arange(A.n)
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    cube = (i // 2) + (nx // 2) * ((j // 2) + (ny // 2) * (k // 2))
    perm = np.empty(ref.n, dtype=np.int64)
    perm[agg] = cube
    Cd = C.to_dense()
    Rd = 0.5 * ref.to_dense()[np.ix_(perm, perm)]
    assert np.array_equal(Cd != 0, Rd != 0)
    assert np.abs(Cd - Rd).max() <= 4e-16 * 3.0
