"""Oracle hierarchy for a batch of independent systems (block-diagonal union).

Pins: with no edge between systems, the strict edge order of the matching
restricted to one system is that system's own order, so matching, aggregation,
Galerkin products and smoothers of the union restricted to a system's rows
equal those of the system built alone, bit for bit, and the V-cycle of the
union applied to a vector supported on one system equals that system's own
V-cycle. The size rule applies to the largest system.
"""
import numpy as np
import pytest

import oracle
from paper_2006_16147_gb300 import workloads as W


def _systems():
    return [W.poisson3d(9, 8, 7), W.poisson3d(6), W.poisson2d_aniso(20, 18, 1e-2), W.poisson3d(11, 5, 4)]


def _block(A, r0, r1):
    rp = A.row_ptr[r0:r1 + 1] - A.row_ptr[r0]
    sl = slice(A.row_ptr[r0], A.row_ptr[r1])
    return rp, A.col[sl] - r0, A.val[sl]


@pytest.fixture(scope="module")
def union():
    mats = _systems()
    A, offs = W.block_diagonal(mats)
    # no stall stop (min_ratio 0) so that every system coarsens as far as the union does
    H = oracle.Hierarchy(A, max_coarse=20, min_ratio=0.0, seg=offs)
    return mats, A, offs, H


def test_block_diagonal_generator():
    mats = _systems()
    A, offs = W.block_diagonal(mats)
    D = A.to_dense()
    for s, M in enumerate(mats):
        assert np.array_equal(D[offs[s]:offs[s + 1], offs[s]:offs[s + 1]], M.to_dense())
    mask = np.zeros_like(D, dtype=bool)
    for s in range(len(mats)):
        mask[offs[s]:offs[s + 1], offs[s]:offs[s + 1]] = True
    assert not D[~mask].any()


def test_size_rule_uses_largest_system(union):
    mats, A, offs, H = union
    sizes = H.sizes()
    # the union (total rows) stays above max_coarse long after the largest system is below it
    solo_levels = oracle.Hierarchy(max(mats, key=lambda M: M.n), max_coarse=20, min_ratio=0.0).num_levels
    assert H.num_levels == solo_levels
    assert sizes[-1][0] > 20


def test_levels_restrict_to_solo_hierarchies(union):
    mats, A, offs, H = union
    L = H.num_levels
    checked = 0
    for s, M in enumerate(mats):
        solo = oracle.Hierarchy(M, max_coarse=0, max_levels=L, min_ratio=0.0)
        if solo.num_levels != L:
            continue            # the small system stopped reducing earlier on its own
        checked += 1
        r0, r1 = offs[s], offs[s + 1]
        for l in range(L):
            ul = H.level(l)
            sl = solo.level(l)
            assert r1 - r0 == sl.n
            rp, cl, vl = _block(ul, r0, r1)
            assert np.array_equal(rp, sl.row_ptr) and np.array_equal(cl, sl.col) and np.array_equal(vl, sl.val)
            assert np.array_equal(ul.w[r0:r1], sl.w) and np.array_equal(ul.minv[r0:r1], sl.minv)
            if l < L - 1:
                nxt = H.level(l + 1)
                # offsets of the next level: the first aggregate of the system
                c0 = ul.agg[r0]
                assert np.array_equal(ul.agg[r0:r1] - c0, sl.agg)
                assert np.array_equal(ul.p[r0:r1], sl.p)
                r0, r1 = c0, c0 + solo.level(l + 1).n
                assert r1 <= nxt.n
    assert checked >= 3


def test_vcycle_is_block_diagonal(union):
    mats, A, offs, H = union
    rng = np.random.default_rng(5)
    checked = 0
    for s, M in enumerate(mats):
        solo = oracle.Hierarchy(M, max_coarse=0, max_levels=H.num_levels, min_ratio=0.0)
        if solo.num_levels != H.num_levels:
            continue
        r = np.zeros(A.n)
        rs = rng.normal(size=M.n)
        r[offs[s]:offs[s + 1]] = rs
        z = H.vcycle(r)
        assert np.array_equal(z[offs[s]:offs[s + 1]], solo.vcycle(rs))
        assert not np.delete(z, np.arange(offs[s], offs[s + 1])).any()
        checked += 1
    assert checked >= 2


def test_pcg_per_system_converges(union):
    mats, A, offs, H = union
    for s, M in enumerate(mats):
        b = np.zeros(A.n)
        bs = np.random.default_rng(s).normal(size=M.n)
        b[offs[s]:offs[s + 1]] = bs
        x, info = H.pcg(b, rtol=1e-6)
        assert info["status"] == 0
        xs = x[offs[s]:offs[s + 1]]
        assert np.linalg.norm(bs - M.scipy() @ xs) <= 1e-6 * np.linalg.norm(bs)
        assert not np.delete(x, np.arange(offs[s], offs[s + 1])).any()
