"""K-cycle (options.cycle = c: FCG(2) coarse corrections on coarse levels
1..c, 32 = every intermediate level) through the C ABI against the oracle's.

Bars: one application of the K-cycle preconditioner within 1e-12 relative of
the oracle's (the inner FCG dot products are summed in another order, so not
bit for bit); the flexible-CG solve within +-1 iteration and 1e-10 relative
in the solution; fewer iterations than the V-cycle; the FP32 cycle converges
to the FP64 true-residual bound.
"""
import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W

from gpu_util import assert_same_solution, dev, setup, solve, vcycle

pytestmark = pytest.mark.gpu

CASES = {
    "poisson32": (lambda: W.poisson3d(32), 200),
    "poisson_ragged": (lambda: W.poisson3d(33, 17, 9), 40),
    "aniso": (lambda: W.poisson2d_aniso(96, 80, 1e-2), 40),
    "spd_random": (lambda: W.random_spd(700, 0.01, 7), 40),
    "varcoef": (lambda: W.varcoef3d(24, seed=2), 40),
}


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("cycle", [1, 2, 32])
@pytest.mark.parametrize("name", list(CASES))
def test_kcycle_application_parity(orc, name, cycle):
    mk, mc = CASES[name]
    A = mk()
    H = orc.Hierarchy(A, max_coarse=mc, cycle=cycle)
    h = setup(A, max_coarse=mc, cycle=cycle)
    r = np.random.default_rng(3).normal(size=A.n)
    zo = H.vcycle(r)
    zg = vcycle(h, r)
    assert np.linalg.norm(zg - zo) <= 1e-12 * np.linalg.norm(zo)
    h.close()


@pytest.mark.parametrize("cycle", [1, 32])
@pytest.mark.parametrize("name", list(CASES))
def test_kcycle_fcg_parity(orc, name, cycle):
    mk, mc = CASES[name]
    A = mk()
    b, _ = W.rhs_uniform(A, 1)
    H = orc.Hierarchy(A, max_coarse=mc, cycle=cycle)
    h = setup(A, max_coarse=mc, cycle=cycle)
    xo, io = H.pcg(b, rtol=1e-6, maxit=500, flexible=True)
    xg, ig = solve(h, b, rtol=1e-6, maxit=500)
    assert io["status"] == 0 and ig["status"] == 0
    assert abs(ig["iterations"] - io["iterations"]) <= 1
    assert np.linalg.norm(b - A.scipy() @ xg) <= 1e-6 * np.linalg.norm(b)
    assert_same_solution(H, b, xg, ig, xo, io, flexible=True)
    h.close()


def test_kcycle_fewer_iterations_and_fp32():
    A = W.poisson3d(64)
    b, _ = W.rhs_uniform(A, 1)
    its = {}
    for cyc, prec in ((0, 0), (32, 0), (32, 1)):
        h = setup(A, cycle=cyc, precision=prec, krylov=1)
        x, info = solve(h, b, rtol=1e-8, maxit=500)
        assert info["status"] == 0
        assert np.linalg.norm(b - A.scipy() @ x) <= 1e-8 * np.linalg.norm(b)
        its[(cyc, prec)] = info["iterations"]
        h.close()
    assert its[(32, 0)] < its[(0, 0)]
    assert abs(its[(32, 1)] - its[(32, 0)]) <= 2


def test_kcycle_option_checks():
    import torch
    from paper_2006_16147_gb300 import amg
    A = W.poisson3d(12)
    with pytest.raises(amg.AmgError):
        setup(A, cycle=1, pre=2)
    with pytest.raises(amg.AmgError):
        setup(A, cycle=33)
    h = setup(A, cycle=1)
    B = dev(W.rhs_normal(A.n, seed=1, k=3))
    X = torch.zeros(A.n, 3, dtype=torch.float64, device="cuda:0")
    with pytest.raises(amg.AmgError):
        amg.amg_solve_batch(h, B, X)
    h.close()
    with pytest.raises(amg.AmgError):
        amg.amg_setup_many([(dev(A.row_ptr), dev(A.col), dev(A.val), dev(np.ones(A.n)))], cycle=1)
