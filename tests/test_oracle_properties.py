"""Randomised properties of the oracle's hierarchy (hypothesis, CPU): on
random SPD matrices and smooth vectors of random signs, every level's
aggregates partition the rows, its prolongator has orthonormal columns whose
range holds w, its coarse matrix equals the dense Galerkin product, and the
V-cycle is symmetric positive definite (Eq. 2)."""
import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

oracle = pytest.importorskip("oracle")


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


@settings(max_examples=40, deadline=None)
@given(n=st.integers(4, 48), density=st.floats(0.05, 0.5), seed=st.integers(0, 10_000),
       sweeps=st.integers(1, 4))
def test_random_hierarchy_properties(n, density, seed, sweeps):
    A = W.random_spd(n, density, seed)
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.3, 2.0, n) * rng.choice([-1.0, 1.0], n)
    H = oracle.Hierarchy(A, w, sweeps=sweeps, max_coarse=2, max_levels=4)
    for l in range(H.num_levels - 1):
        lv = H.level(l)
        nc = H.sizes()[l + 1][0]
        counts = np.bincount(lv.agg, minlength=nc)
        assert counts.min() >= 1 and counts.sum() == lv.n and counts.max() <= 2 ** sweeps
        P = np.zeros((lv.n, nc))
        P[np.arange(lv.n), lv.agg] = lv.p
        assert np.allclose(P.T @ P, np.eye(nc), atol=1e-14)
        wl = lv.w
        assert np.allclose(P @ (P.T @ wl), wl, rtol=1e-13, atol=1e-13 * np.abs(wl).max())
        Al = W.Csr(lv.row_ptr, lv.col, lv.val).to_dense()
        C = H.level_csr(l + 1).to_dense()
        ref = P.T @ Al @ P
        assert np.abs(C - ref).max() <= 1e-12 * np.abs(ref).max()
    B = np.column_stack([H.vcycle(e) for e in np.eye(n)])
    assert np.allclose(B, B.T, atol=1e-12 * np.abs(B).max())
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


@settings(max_examples=30, deadline=None)
@given(n=st.integers(6, 40), density=st.floats(0.08, 0.5), seed=st.integers(0, 10_000))
def test_random_smoothed_hierarchy_properties(n, density, seed):
    # Pbar = (I - omega D^-1 A) P with omega = 4 / (3 max_i sum_j |a_ij| / a_ii),
    # coarse matrix Pbar^T A Pbar, V-cycle SPD
    A = W.random_spd(n, density, seed)
    H = oracle.Hierarchy(A, smooth_p=True, max_coarse=2, max_levels=3)
    for l in range(H.num_levels - 1):
        lv = H.level(l)
        nc = H.sizes()[l + 1][0]
        Al = W.Csr(lv.row_ptr, lv.col, lv.val).to_dense()
        D = np.diag(Al)
        eta = (np.abs(Al).sum(axis=1) / D).max()
        Pb, om = H.pbar(l)
        assert abs(om - 4.0 / (3.0 * eta)) <= 1e-15 * om
        P = np.zeros((lv.n, nc))
        P[np.arange(lv.n), lv.agg] = lv.p
        ref = (np.eye(lv.n) - om * Al / D[:, None]) @ P
        got = np.zeros((lv.n, nc))
        got[np.repeat(np.arange(lv.n), np.diff(Pb.row_ptr)), Pb.col] = Pb.val
        assert np.abs(got - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())
        C = H.level_csr(l + 1).to_dense()
        Cref = ref.T @ Al @ ref
        assert np.abs(C - Cref).max() <= 1e-12 * np.abs(Cref).max()
    B = np.column_stack([H.vcycle(e) for e in np.eye(n)])
    assert np.allclose(B, B.T, atol=1e-12 * np.abs(B).max())
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
