"""Full-size parity: the benchmark's workloads at their full sizes and in the
launch configuration bench.py times, CUDA path against the oracle on the same
inputs.

- 256^3 Poisson, FP64, default options, b = A x* with x* ~ U[-1, 1] (seed 1):
  the oracle's setup at this size takes seconds, so the whole hierarchy is
  compared bit for bit (every level's matrix, smooth vector, l1-Jacobi
  diagonal, aggregates and prolongator weights, the coarsest factor), and the
  PCG solution within 1e-10 relative with iterations within +-1.
- 256^3 jump coefficients (g ~ N(0, 2^2), seed 2; b = A x*, seed 3), FP64:
  coarsening stalls on the ratio rule with a 373,821-row coarsest level,
  solved by the CG coarsest solver, so the outer solver is flexible CG. The
  whole hierarchy bit for bit, then the FCG solution within 1e-10 of the
  oracle's (the oracle re-run for the GPU's iteration count when the counts
  differ by one).
- The served hierarchies at their served sizes: the 2D anisotropic problem
  -u_xx - 0.01 u_yy on 2048^2 and 3D Poisson 192^3: hierarchy bit for bit,
  PCG solution within 1e-10.
- 128^3 Poisson with 64 right-hand sides (seed 4), FP32 V-cycle inside FP64
  CG, autotuned: sampled columns against the oracle's FP64 PCG. Both meet
  ||b - A x|| <= e ||b||, e = 1e-6, so for SPD A each is within kappa e ||x*||
  of the solution x* and ||x - x_oracle|| <= 2 kappa e ||x_oracle|| / (1 - kappa e);
  kappa of the 7-point Laplacian on an N^3 grid is
  (6 + 6 cos(pi h)) / (6 - 6 cos(pi h)), h = 1 / (N + 1).
"""
import numpy as np
import pytest

from paper_2006_16147_gb300 import workloads as W

from gpu_util import assert_same_solution, dev, setup, solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _assert_same_hierarchy(H, h, dense_coarse=True):
    """Every level's matrix, smooth vector, l1-Jacobi diagonal, aggregates and
    prolongator weights bit for bit, and the coarsest factor when dense."""
    from paper_2006_16147_gb300 import amg
    info = amg.amg_hierarchy_info(h)
    assert info["n"] == [s[0] for s in H.sizes()]
    assert info["nnz"] == [s[1] for s in H.sizes()]
    for l in range(H.num_levels):
        ol = H.level(l)
        gl = amg.amg_export_level(h, l)
        for k in ("row_ptr", "col", "val", "w", "minv"):
            assert np.array_equal(getattr(ol, k), gl[k]), (l, k)
        if l < H.num_levels - 1:
            assert np.array_equal(ol.agg, gl["agg"]) and np.array_equal(ol.p, gl["p"]), l
        del ol, gl
    assert H.coarse_is_cg == (not dense_coarse)
    if dense_coarse:
        assert np.array_equal(H.coarse_factor(), amg.amg_coarse_factor(h))
    return info


def _pcg_parity(H, h, b, flexible=False):
    xo, io = H.pcg(b, rtol=1e-6, flexible=flexible)
    xg, ig = solve(h, b, rtol=1e-6)
    assert io["status"] == 0 and ig["status"] == 0
    assert abs(io["iterations"] - ig["iterations"]) <= 1
    assert ig["true_relres"] <= 1e-6
    assert_same_solution(H, b, xg, ig, xo, io, flexible=flexible)
    return ig, io


def test_poisson256_hierarchy_and_pcg_match_oracle(orc):
    A = W.poisson3d(256)
    b, _ = W.rhs_uniform(A, 1)
    H = orc.Hierarchy(A)
    h = setup(A)
    _assert_same_hierarchy(H, h)
    _pcg_parity(H, h, b)
    h.close()


def test_varcoef256_hierarchy_and_fcg_match_oracle(orc):
    # BASELINE config 3's matrix in FP64: the stalled coarsening and the CG
    # coarsest solver at full size
    A = W.varcoef3d(256, seed=2)
    b, _ = W.rhs_uniform(A, 3)
    H = orc.Hierarchy(A)
    h = setup(A, krylov=1)
    info = _assert_same_hierarchy(H, h, dense_coarse=False)
    assert info["coarse_solver"] == 1 and info["n"][-1] > 4096
    ig, io = _pcg_parity(H, h, b, flexible=True)
    print(f"varcoef 256^3: levels {info['n']}, FCG it {ig['iterations']} (oracle {io['iterations']})")
    h.close()


@pytest.mark.parametrize("name", ["aniso2048", "poisson192"])
def test_served_hierarchies_at_served_size_match_oracle(orc, name):
    A = W.poisson2d_aniso(2048, 2048, 1e-2) if name == "aniso2048" else W.poisson3d(192)
    b, _ = W.rhs_uniform(A, 6)
    H = orc.Hierarchy(A)
    h = setup(A)
    _assert_same_hierarchy(H, h)
    _pcg_parity(H, h, b)
    h.close()


def test_block64_poisson128_fp32_vcycle_sampled_columns(orc):
    import torch
    from paper_2006_16147_gb300 import amg
    N = 128
    A = W.poisson3d(N)
    B = W.rhs_normal(A.n, 4, 64)
    h = setup(A, precision=amg.AMG_FP32_VCYCLE, autotune=1)
    Bd = dev(B)
    Xd = dev(np.zeros_like(B))
    infos = amg.amg_solve_batch(h, Bd, Xd, rtol=1e-6, maxit=1000)
    torch.cuda.synchronize()
    X = Xd.cpu().numpy()
    h.close()
    ch = np.cos(np.pi / (N + 1))
    kappa = (6 + 6 * ch) / (6 - 6 * ch)
    H = orc.Hierarchy(A)
    As = A.scipy()
    for c in (0, 37, 63):
        assert infos[c]["true_relres"] <= 1e-6
        r = B[:, c] - As @ X[:, c]                  # recomputed here: another summation order
        assert np.linalg.norm(r) <= 1e-6 * (1 + 1e-6) * np.linalg.norm(B[:, c])
        xo, io = H.pcg(B[:, c].copy(), rtol=1e-6)
        assert io["status"] == 0
        e = 1e-6
        assert np.linalg.norm(X[:, c] - xo) <= 2 * kappa * e / (1 - kappa * e) * np.linalg.norm(xo)
