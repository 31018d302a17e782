"""Pins of the oracle's edge weights (Eq. 3) and matching (Section 3.2)."""
import itertools

import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W


def _edges(A):
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    m = (A.col > rows) & (A.val != 0)
    return rows[m], A.col[m]


def test_weights_laplacian_closed_form(orc):
    # w = 1, a_ii = 6, a_ij = -1: c = 1 + 2/12 = 7/6 on every edge.
    A = W.poisson3d(5, 4, 3)
    c = orc.weights(A, np.ones(A.n))
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    off = A.col != rows
    assert np.all(np.abs(c[off] - 7.0 / 6.0) <= 2.3e-16)
    assert np.all(np.isneginf(c[~off]))


def test_weights_hand_example(orc):
    # A = [[4,-1,0],[-1,5,-2],[0,-2,3]], w = (1,2,1):
    # c_01 = 1 + 2*1*1*2/(4*1 + 5*4) = 7/6, c_12 = 1 + 2*2*2*1/(5*4 + 3*1) = 31/23.
    A = W.Csr([0, 2, 5, 7], [0, 1, 0, 1, 2, 1, 2], [4, -1, -1, 5, -2, -2, 3])
    c = orc.weights(A, np.array([1.0, 2.0, 1.0]))
    assert c[1] == pytest.approx(7 / 6, rel=1e-15) and c[2] == c[1]
    assert c[4] == pytest.approx(31 / 23, rel=1e-15) and c[5] == c[4]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_weights_spd_range_and_symmetry(orc, seed):
    # For s.p.d. A, |a_ij| < sqrt(a_ii a_jj) so 0 < c_ij < 2; c is symmetric.
    A = W.random_spd(40, 0.15, seed)
    w = np.random.default_rng(seed).uniform(0.5, 2.0, A.n) * np.random.default_rng(seed + 7).choice([-1, 1], A.n)
    c = orc.weights(A, w)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    off = A.col != rows
    assert np.all((c[off] > 0) & (c[off] < 2))
    dense = np.zeros((A.n, A.n))
    dense[rows[off], A.col[off]] = c[off]
    assert np.array_equal(dense, dense.T)


def _check_valid_maximal(A, mate):
    n = A.n
    for v in range(n):
        if mate[v] >= 0:
            assert mate[mate[v]] == v and mate[v] != v
    lo, hi = _edges(A)
    both_free = (mate[lo] < 0) & (mate[hi] < 0)
    assert not both_free.any(), "matching is not maximal"
    # matched pairs are edges of the graph
    es = set(zip(lo.tolist(), hi.tolist()))
    for v in range(n):
        if mate[v] > v:
            assert (v, int(mate[v])) in es


@pytest.mark.parametrize("seed", list(range(8)))
def test_greedy_equals_locally_dominant_random(orc, seed):
    rng = np.random.default_rng(100 + seed)
    A = W.random_spd(int(rng.integers(5, 60)), float(rng.uniform(0.05, 0.4)), seed)
    w = rng.uniform(0.2, 3.0, A.n)
    g = orc.match_greedy(A, w)
    ld, rounds = orc.match_ld(A, w)
    assert np.array_equal(g, ld)
    _check_valid_maximal(A, g)


@pytest.mark.parametrize("shape", [(6, 5, 4), (7, 7, 1), (9, 3, 2)])
def test_greedy_equals_locally_dominant_ties(orc, shape):
    # All weights tie on the Laplacian with w = 1: the index tiebreak decides.
    A = W.poisson3d(*shape)
    w = np.ones(A.n)
    g = orc.match_greedy(A, w)
    ld, _ = orc.match_ld(A, w)
    assert np.array_equal(g, ld)
    _check_valid_maximal(A, g)


def test_laplacian_first_sweep_pairs_along_x(orc):
    # With all weights equal the smallest-index edge of each free vertex wins:
    # on an even x-extent every vertex pairs with its x-neighbour.
    A = W.poisson3d(8, 5, 3)
    g = orc.match_greedy(A, np.ones(A.n))
    assert np.array_equal(g, np.arange(A.n) ^ 1)


def test_anisotropy_aligned_pairs(orc):
    # Supplementary anisotropic problem: aggregates follow the strong coupling.
    A = W.poisson2d_aniso(16, 12, eps=1e-2)
    g = orc.match_greedy(A, np.ones(A.n))
    nx = 16
    for v in range(A.n):
        assert g[v] >= 0 and g[v] // nx == v // nx, "pair not along the strong (x) direction"


def _brute_max_weight(n, edges):
    best = 0.0
    for r in range(0, n // 2 + 1):
        for sub in itertools.combinations(range(len(edges)), r):
            used = set()
            ok = True
            s = 0.0
            for e in sub:
                a, b, c = edges[e]
                if a in used or b in used:
                    ok = False
                    break
                used.add(a); used.add(b); s += c
            if ok:
                best = max(best, s)
    return best


@pytest.mark.parametrize("seed", list(range(6)))
def test_half_approximation_bruteforce(orc, seed):
    # Locally-dominant matching weighs at least half the maximum (Section 3.2).
    rng = np.random.default_rng(seed)
    A = W.random_spd(8, 0.45, 50 + seed)
    w = rng.uniform(0.5, 2.0, A.n)
    c = orc.weights(A, w)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    edges = [(int(i), int(j), float(cc)) for i, j, cc in zip(rows, A.col, c) if j > i and np.isfinite(cc)]
    if len(edges) > 14:
        edges = edges[:14]
        sub = W.Csr(*_subgraph(A, edges))
        A = sub
        c = orc.weights(A, w)
    g = orc.match_greedy(A, w)
    cw = {(i, j): cc for i, j, cc in edges}
    got = sum(cw[(v, int(g[v]))] for v in range(A.n) if g[v] > v)
    opt = _brute_max_weight(A.n, edges)
    assert got >= 0.5 * opt - 1e-12


def _subgraph(A, edges):
    n = A.n
    d = np.zeros((n, n))
    dense = A.to_dense()
    for i, j, _ in edges:
        d[i, j] = dense[i, j]
        d[j, i] = dense[j, i]
    d[np.diag_indices(n)] = np.diag(dense)
    rows, cols = np.nonzero(d)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp), cols, d[rows, cols]


def _ld_rounds_equal_weights(nx, ny, nz):
    # Independent replay of the locally-dominant rounds for equal weights on
    # the 7-point grid: every free vertex points to its smallest-index free
    # neighbour (the (lo, hi) tiebreak), mutual pairs match, until no free
    # vertex has a free neighbour.
    n = nx * ny * nz
    idx = np.arange(n)
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    nbrs = [(-nx * ny, k > 0), (-nx, j > 0), (-1, i > 0), (1, i < nx - 1), (nx, j < ny - 1), (nx * ny, k < nz - 1)]
    mate = np.full(n, -1)
    rounds = 0
    while True:
        free = mate < 0
        cand = np.full(n, -1)
        for off, ok in nbrs:
            sel = ok & free & (cand < 0)
            nb = idx[sel] + off
            take = free[nb]
            cand[idx[sel][take]] = nb[take]
        c = np.where(cand >= 0, cand, idx)
        mutual = free & (cand >= 0) & (c[c] == idx) & (idx < c)
        if not mutual.any():
            return mate, rounds
        a, b = idx[mutual], c[mutual]
        mate[a], mate[b] = b, a
        rounds += 1


@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 16, 16), (10, 7, 5), (9, 4, 3)])
def test_ld_rounds_match_an_independent_replay(orc, shape):
    # pins the oracle's round count (the launch-pair GPU mode is compared
    # against it) and its matching; on N^3 the rounds form a diagonal
    # wavefront of 2.5 N - 2 rounds
    A = W.poisson3d(*shape)
    ld, rounds = orc.match_ld(A, np.ones(A.n))
    mate, r = _ld_rounds_equal_weights(*shape)
    assert rounds == r
    assert np.array_equal(ld >= 0, mate >= 0)
    assert np.array_equal(ld[mate >= 0], mate[mate >= 0])
    if shape[0] == shape[1] == shape[2]:
        assert rounds == 5 * shape[0] // 2 - 2
