"""The synthetic input generators build the paper's model operators."""
import numpy as np

from paper_2006_16147_gb300 import workloads as W


def test_poisson_shape_and_values():
    A = W.poisson3d(32)
    assert A.n == 32768 and A.nnz == 223232
    d = A.scipy()
    assert abs(d - d.T).max() == 0
    assert np.all(d.diagonal() == 6.0)
    assert set(np.unique(A.val).tolist()) == {-1.0, 6.0}
    assert np.all(np.diff(A.col)[np.diff(np.repeat(np.arange(A.n), np.diff(A.row_ptr))) == 0] > 0)


def test_poisson_256_counts_formula():
    # nnz of the 7-point stencil on N^3 with eliminated Dirichlet nodes: 7 N^3 - 6 N^2
    for N in (5, 17, 64):
        assert W.poisson3d(N).nnz == 7 * N**3 - 6 * N**2


def test_varcoef_spd_and_seeded():
    A = W.varcoef3d(10, seed=2)
    B = W.varcoef3d(10, seed=2)
    assert np.array_equal(A.val, B.val)
    d = A.to_dense()
    assert np.allclose(d, d.T, rtol=0, atol=0)
    assert np.linalg.eigvalsh(d).min() > 0
    offd = -A.val[A.val < 0]
    assert offd.max() / offd.min() > 1e2


def test_aniso_values():
    A = W.poisson2d_aniso(8, 6, eps=1e-2)
    d = A.to_dense()
    assert np.allclose(np.diag(d), 2.02)
    assert d[0, 1] == -1.0 and d[0, 8] == -1e-2


def test_rhs_seeded():
    A = W.poisson3d(6)
    b1, x1 = W.rhs_uniform(A, 1)
    b2, x2 = W.rhs_uniform(A, 1)
    assert np.array_equal(b1, b2) and np.abs(x1).max() <= 1
    assert W.rhs_normal(10, 3, 4).shape == (10, 4)
    e = W.batch_edges(256, 5)
    assert min(e) >= 16 and max(e) <= 64 and len(e) == 256


def test_random_spd_sparse_spd_and_seeded():
    A = W.random_spd_sparse(500, 4, 3)
    B = W.random_spd_sparse(500, 4, 3)
    assert np.array_equal(A.val, B.val) and np.array_equal(A.col, B.col)
    D = A.to_dense()
    assert np.array_equal(D, D.T)
    assert np.all(np.diff(A.col[A.row_ptr[0]:A.row_ptr[1]]) > 0)
    off = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
    assert np.all(np.diag(D) > off)                   # strictly diagonally dominant => SPD
    assert np.linalg.eigvalsh(D).min() > 0


def test_with_hubs_spd_and_row_lengths():
    A = W.with_hubs(W.poisson2d_aniso(12, 10), [5, 40], 3)
    assert A.n == 122
    assert np.diff(A.row_ptr)[-2:].tolist() == [6, 41]
    D = A.to_dense()
    assert np.array_equal(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0
