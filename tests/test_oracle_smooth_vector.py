"""Oracle smooth vector (a few l1-Jacobi sweeps on A w = 0 from a sample
vector, Section 3.2) and the 3D anisotropic generator of the supplementary
anisotropic experiment.

Pins: zero sweeps return the sample; on a diagonal matrix the l1-Jacobi
diagonal is A itself, so one sweep scales w by (1 - omega); the smoother is
A-convergent, so the A-norm never grows; the sweeps damp the oscillatory
part (the Rayleigh quotient drops); and on z-aligned anisotropy
(k = (1, 1, 100)) the weighted matching pairs vertices along z only, the
aggregates the paper's figure shows.
"""
import numpy as np
import pytest

import oracle
from paper_2006_16147_gb300 import workloads as W


def test_zero_sweeps_is_identity():
    A = W.poisson3d(6)
    w0 = np.random.default_rng(0).normal(size=A.n)
    assert np.array_equal(oracle.smooth_vector(A, w0, 0), w0)


@pytest.mark.parametrize("omega", [1.0, 0.5, 2.0 / 3.0])
def test_diagonal_matrix_closed_form(omega):
    n = 50
    d = np.random.default_rng(1).uniform(0.5, 4.0, n)
    A = W.Csr(np.arange(n + 1), np.arange(n), d)
    w0 = np.random.default_rng(2).normal(size=n)
    w = oracle.smooth_vector(A, w0, 1, omega)
    assert np.allclose(w, (1.0 - omega) * w0, rtol=0, atol=4e-16 * np.abs(w0).max())


@pytest.mark.parametrize("mk", [lambda: W.poisson3d(12), lambda: W.aniso3d(10, 9, 8), lambda: W.varcoef3d(10, seed=3),
                                lambda: W.random_spd(200, 0.05, 4)])
def test_a_norm_never_grows_and_rayleigh_drops(mk):
    A = mk()
    S = A.scipy()
    w = np.random.default_rng(3).normal(size=A.n)
    norms, rq = [], []
    for k in range(6):
        Aw = S @ w
        norms.append(float(w @ Aw))
        rq.append(float(w @ Aw) / float(w @ w))
        w = oracle.smooth_vector(A, w, 1)
    assert all(norms[k + 1] <= norms[k] * (1 + 1e-12) for k in range(len(norms) - 1))
    assert rq[-1] < 0.8 * rq[0]


def test_sweeps_compose():
    A = W.poisson3d(7, 6, 5)
    w0 = np.random.default_rng(4).normal(size=A.n)
    assert np.array_equal(oracle.smooth_vector(A, oracle.smooth_vector(A, w0, 2), 3), oracle.smooth_vector(A, w0, 5))


def test_aniso3d_generator():
    A = W.aniso3d(5, 4, 3, k=(1.0, 2.0, 100.0))
    D = A.to_dense()
    assert np.allclose(D, D.T)
    nx, ny = 5, 4
    i = 1 + nx * (1 + ny * 1)                     # an interior node
    assert D[i, i] == 2 * (1.0 + 2.0 + 100.0)
    assert D[i, i - 1] == -1.0 and D[i, i - nx] == -2.0 and D[i, i - nx * ny] == -100.0


def test_z_aligned_anisotropy_matches_along_z():
    nx, ny, nz = 8, 6, 10
    A = W.aniso3d(nx, ny, nz, k=(1.0, 1.0, 100.0))
    m = oracle.match_greedy(A, np.ones(A.n))
    i = np.arange(A.n)
    paired = m >= 0
    assert paired.mean() > 0.9
    assert np.all(np.abs(m[paired] - i[paired]) == nx * ny)
