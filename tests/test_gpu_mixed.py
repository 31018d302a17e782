"""FP32 V-cycle inside FP64 CG (AMG_FP32_VCYCLE) and flexible CG.

There is no oracle of the same mixed arithmetic: the FP32 V-cycle is compared
with the FP64 oracle's V-cycle (error reported, bounded by a multiple of FP32
rounding), and the mixed solve must still reach the requested FP64 relative
residual, with its solution compared with the FP64 oracle's.
"""
import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W

from gpu_util import assert_same_solution, setup, solve, vcycle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


CASES = {
    "poisson": lambda: W.poisson3d(33, 31, 29),
    "varcoef": lambda: W.varcoef3d(32, seed=2),
    "aniso": lambda: W.poisson2d_aniso(128, 96, 1e-2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_vcycle_error_vs_fp64_oracle(orc, name):
    A = CASES[name]()
    H = orc.Hierarchy(A)
    h = setup(A, precision=1)
    r = np.random.default_rng(7).normal(size=A.n)
    zo = H.vcycle(r)
    zg = vcycle(h, r)
    err = np.linalg.norm(zg - zo) / np.linalg.norm(zo)
    print(f"{name}: FP32 V-cycle relative error vs FP64 oracle {err:.2e}")
    assert err <= 2e-5      # about 100 x FP32 unit roundoff over the levels
    h.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("krylov", [0, 1])
@pytest.mark.parametrize("rtol", [1e-6, 1e-8])
def test_fp32_vcycle_pcg_reaches_fp64_tolerance(orc, name, krylov, rtol):
    A = CASES[name]()
    b, xs = W.rhs_uniform(A, 3)
    H = orc.Hierarchy(A)
    xo, io = H.pcg(b, rtol=rtol, flexible=bool(krylov))
    h = setup(A, precision=1, krylov=krylov)
    xg, ig = solve(h, b, rtol=rtol)
    res = np.linalg.norm(b - A.scipy() @ xg) / np.linalg.norm(b)
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    print(f"{name} krylov={krylov} rtol={rtol:g}: it {ig['iterations']} (oracle FP64 {io['iterations']}), "
          f"relres {res:.2e}, |x - x_oracle|/|x_oracle| {err:.2e}")
    assert ig["status"] == 0 and res <= rtol
    assert ig["iterations"] <= io["iterations"] + 2
    h.close()


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_flexible_cg_parity(orc, name):
    A = CASES[name]()
    b, _ = W.rhs_uniform(A, 4)
    H = orc.Hierarchy(A)
    xo, io = H.pcg(b, rtol=1e-6, flexible=True)
    h = setup(A, krylov=1)
    xg, ig = solve(h, b, rtol=1e-6)
    assert abs(ig["iterations"] - io["iterations"]) <= 1
    assert_same_solution(H, b, xg, ig, xo, io, flexible=True)
    h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_coarsest_cg_path_parity(orc, precision):
    # jump coefficients: coarsening stalls, the hierarchy stops on the ratio
    # rule; max_dense = 100 forces the CG coarsest solve on a 32^3 case
    from paper_2006_16147_gb300 import amg
    A = W.varcoef3d(32, seed=2)
    b, _ = W.rhs_uniform(A, 3)
    H = orc.Hierarchy(A, max_dense=100)
    assert H.coarse_is_cg
    h = setup(A, max_dense=100, precision=precision, krylov=1)
    info = amg.amg_hierarchy_info(h)
    assert info["coarse_solver"] == 1 and info["n"] == [s[0] for s in H.sizes()]
    r = np.random.default_rng(1).normal(size=A.n)
    zo, zg = H.vcycle(r), vcycle(h, r)
    err = np.linalg.norm(zg - zo) / np.linalg.norm(zo)
    assert err <= (1e-9 if precision == 0 else 2e-5)
    xo, io = H.pcg(b, rtol=1e-8, flexible=True)
    xg, ig = solve(h, b, rtol=1e-8)
    print(f"coarse CG precision={precision}: V-cycle err {err:.1e}, it {ig['iterations']} (oracle {io['iterations']})")
    assert ig["status"] == 0 and ig["true_relres"] <= 1e-8
    assert abs(ig["iterations"] - io["iterations"]) <= (1 if precision == 0 else 2)
    h.close()
