"""amg_smooth_vector against the oracle (bit for bit: the same l1-Jacobi
diagonal and the same per-row operation order), and the hierarchy and solve
built from such a vector on the 3D anisotropic problem."""
import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W

from gpu_util import dev, setup, solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("mk", [lambda: W.poisson3d(20, 17, 9), lambda: W.aniso3d(16, 12, 10), lambda: W.varcoef3d(14, seed=1),
                                lambda: W.random_spd(500, 0.02, 3)])
@pytest.mark.parametrize("sweeps,omega", [(0, 1.0), (1, 1.0), (4, 2.0 / 3.0), (7, 1.0)])
def test_smooth_vector_bit_exact(orc, mk, sweeps, omega):
    from paper_2006_16147_gb300 import amg
    A = mk()
    w0 = np.random.default_rng(5).uniform(0.5, 1.5, A.n)
    wo = orc.smooth_vector(A, w0, sweeps, omega)
    wg = amg.amg_smooth_vector(dev(A.row_ptr), dev(A.col), dev(A.val), dev(w0), sweeps, omega).cpu().numpy()
    assert np.array_equal(wo, wg)


def test_setup_and_solve_from_smooth_vector(orc):
    from paper_2006_16147_gb300 import amg
    A = W.aniso3d(24, k=(100.0, 100.0, 1.0))
    w0 = np.ones(A.n)
    w = amg.amg_smooth_vector(dev(A.row_ptr), dev(A.col), dev(A.val), dev(w0), 5).cpu().numpy()
    H = orc.Hierarchy(A, w, max_coarse=40)
    h = setup(A, w, max_coarse=40)
    info = amg.amg_hierarchy_info(h)
    assert info["n"] == [s[0] for s in H.sizes()]
    b, _ = W.rhs_uniform(A, 2)
    xo, io = H.pcg(b, rtol=1e-6)
    xg, ig = solve(h, b, rtol=1e-6)
    assert abs(ig["iterations"] - io["iterations"]) <= 1
    assert np.linalg.norm(b - A.scipy() @ xg) <= 1e-6 * np.linalg.norm(b)
    h.close()


def test_smooth_vector_errors():
    from paper_2006_16147_gb300 import amg
    A = W.poisson3d(5)
    with pytest.raises(amg.AmgError):
        amg.amg_smooth_vector(dev(A.row_ptr), dev(A.col), dev(A.val), dev(np.ones(A.n)), -1)
    with pytest.raises(amg.AmgError):
        amg.amg_smooth_vector(dev(A.row_ptr), dev(A.col), dev(A.val), dev(np.zeros(A.n)), 2)
