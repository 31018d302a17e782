"""Degenerate cases of the method, on the oracle: a single unknown, a matrix
without off-diagonal entries (no edges to match), and the smallest pair, whose
hierarchy has a closed form (Eq. 3 weight, Eq. 4 column, one Galerkin entry)."""
import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W

oracle = pytest.importorskip("oracle")


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def test_single_unknown_is_one_level_and_exact():
    A = W.Csr([0, 1], [0], [4.0])
    H = oracle.Hierarchy(A, max_coarse=1)
    assert H.num_levels == 1
    x, info = H.pcg(np.array([2.0]), rtol=1e-12)
    assert info["status"] == 0 and info["iterations"] <= 1
    assert x[0] == 0.5


def test_diagonal_matrix_has_no_edges_and_one_level():
    n = 50
    d = np.linspace(1.0, 3.0, n)
    A = W.Csr(np.arange(n + 1), np.arange(n), d)
    H = oracle.Hierarchy(A, max_coarse=1)
    assert H.num_levels == 1                       # nothing matched: the level is the coarsest
    b = np.arange(1.0, n + 1)
    x, info = H.pcg(b, rtol=1e-12)
    assert info["status"] == 0 and info["iterations"] <= 1
    assert np.allclose(x, b / d, rtol=1e-14, atol=0)


def test_smallest_pair_closed_form():
    # A = [[2, -1], [-1, 2]], w = (1, 2): c_01 = 1 - 2 a w0 w1 / (a00 w0^2 + a11 w1^2)
    # = 1 + 4/10 > 0, so the pair matches; the column is w / |w| and the coarse
    # matrix is p^T A p = (2 - 2*2 + 2*4) / 5 = 6/5
    A = W.Csr([0, 2, 4], [0, 1, 0, 1], [2.0, -1.0, -1.0, 2.0])
    w = np.array([1.0, 2.0])
    H = oracle.Hierarchy(A, w, max_coarse=1)
    assert H.num_levels == 2
    lv = H.level(0)
    assert lv.agg.tolist() == [0, 0]
    assert np.allclose(lv.p, w / np.sqrt(5.0), rtol=1e-15, atol=0)
    C = H.level_csr(1).to_dense()
    assert C.shape == (1, 1) and abs(C[0, 0] - 6.0 / 5.0) <= 4e-16 * 6.0 / 5.0
    x, info = H.pcg(np.array([1.0, 0.0]), rtol=1e-12)
    assert info["status"] == 0
    assert np.allclose(x, np.linalg.solve(A.to_dense(), [1.0, 0.0]), rtol=1e-12, atol=0)
