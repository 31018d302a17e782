"""Oracle smoothed prolongator Pbar = (I - omega D^-1 A) P and the general
Galerkin product Pbar^T A Pbar (Section 3.2; the paper's VA3 setting).

Pins: the two-level constant K of the paper's smoothed-aggregation table
(HGS, 16^3) from the oracle's Pbar, which the text's weight does not give;
omega = 2/3 (rule 0) and 1/2 (rule 1, the text's) on the Laplacian; the coarse
matrix against a dense numpy triple product; the V-cycle with Pbar is
symmetric positive definite, also with the paper's GPU smoother setting of
four l1-Jacobi sweeps before and after; and it needs fewer iterations than
the unsmoothed V-cycle.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_2006_16147_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_table_sm_K.txt")


def _gold():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    return {r[0]: (float(r[1]), float(r[2])) for r in rows}


def _dense_P(lv, nc):
    P = np.zeros((lv.n, nc))
    P[np.arange(lv.n), lv.agg] = lv.p
    return P


@pytest.mark.parametrize("rule,omega", [(0, 2.0 / 3.0), (1, 0.5)])
def test_omega_and_definition(rule, omega):
    # eta = ||D^-1 A||_inf = 12 / 6 on the 7-point Laplacian: rule 0 takes
    # 4 / (3 eta) = 2/3, rule 1 (the text's weight) 1 / eta = 1/2
    A = W.poisson3d(10, 9, 8)
    H = oracle.Hierarchy(A, smooth_p=True, max_coarse=40, omega_rule=rule)
    Pb, om = H.pbar(0)
    assert om == omega
    lv = H.level(0)
    nc = H.sizes()[1][0]
    Ad = A.to_dense()
    ref = (np.eye(A.n) - om * Ad / np.diag(Ad)[:, None]) @ _dense_P(lv, nc)
    got = np.zeros((A.n, nc))
    rows = np.repeat(np.arange(A.n), np.diff(Pb.row_ptr))
    got[rows, Pb.col] = Pb.val
    assert np.abs(got - ref).max() <= 1e-15


@pytest.mark.parametrize("mk", [lambda: W.poisson3d(12, 10, 9), lambda: W.aniso3d(9, 8, 7), lambda: W.random_spd(300, 0.03, 5)])
def test_galerkin_is_dense_triple_product(mk):
    A = mk()
    H = oracle.Hierarchy(A, smooth_p=True, max_coarse=20, max_levels=3)
    for l in range(H.num_levels - 1):
        lv = H.level(l)
        Al = W.Csr(lv.row_ptr, lv.col, lv.val).to_dense()
        Pb, _ = H.pbar(l)
        nc = H.sizes()[l + 1][0]
        P = np.zeros((lv.n, nc))
        rows = np.repeat(np.arange(lv.n), np.diff(Pb.row_ptr))
        P[rows, Pb.col] = Pb.val
        C = H.level_csr(l + 1).to_dense()
        ref = P.T @ Al @ P
        assert np.abs(C - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.slow
def test_paper_smoothed_K_constant():
    A = W.poisson3d(16)
    n = A.n
    H = oracle.Hierarchy(A, smooth_p=True, max_levels=2)
    Pb, om = H.pbar(0)
    nc = H.sizes()[1][0]
    assert nc == 512
    P = np.zeros((n, nc))
    P[np.repeat(np.arange(n), np.diff(Pb.row_ptr)), Pb.col] = Pb.val
    Ad = A.to_dense()
    D = np.diag(np.diag(Ad))
    S = sl.null_space(P.T @ D)
    M = np.tril(Ad)
    Mbar = M.T @ np.linalg.solve(M.T + M - Ad, M)
    SAS = S.T @ Ad @ S
    SMS = S.T @ Mbar @ S
    SMS = 0.5 * (SMS + SMS.T)
    K = 1.0 / sl.eigh(SAS, SMS, eigvals_only=True, subset_by_index=[0, 0])[0]
    k_gold, tol = _gold()["HGS"]
    assert abs(K - k_gold) <= tol
    # the text's weight 1 / eta (rule 1) does not give the table's value
    # (1.3708): the reading above rests on this difference
    H1 = oracle.Hierarchy(A, smooth_p=True, max_levels=2, omega_rule=1)
    Pb1, om1 = H1.pbar(0)
    assert om1 == 0.5
    P1 = np.zeros((n, nc))
    P1[np.repeat(np.arange(n), np.diff(Pb1.row_ptr)), Pb1.col] = Pb1.val
    S1 = sl.null_space(P1.T @ D)
    SMS1 = S1.T @ Mbar @ S1
    K1 = 1.0 / sl.eigh(S1.T @ Ad @ S1, 0.5 * (SMS1 + SMS1.T), eigvals_only=True, subset_by_index=[0, 0])[0]
    assert abs(K1 - k_gold) > 10 * tol


@pytest.mark.parametrize("rule", [0, 1])
def test_va3_four_sweeps_vcycle_spd(rule):
    # the paper's GPU setting: smoothed prolongator, l1-Jacobi 4 + 4 sweeps;
    # equal pre and post sweeps with one M make B symmetric positive definite
    A = W.poisson3d(7, 6, 5)
    H = oracle.Hierarchy(A, smooth_p=True, max_coarse=10, pre=4, post=4, omega_rule=rule)
    assert H.num_levels >= 3
    B = np.column_stack([H.vcycle(e) for e in np.eye(A.n)])
    assert np.allclose(B, B.T, atol=1e-13 * np.abs(B).max())
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    # four sweeps contract the error more than one: fewer PCG iterations
    A = W.poisson3d(24)
    b = np.random.default_rng(2).normal(size=A.n)
    its = [oracle.Hierarchy(A, smooth_p=True, pre=k, post=k, omega_rule=rule).pcg(b, rtol=1e-6)[1]["iterations"]
           for k in (1, 4)]
    assert its[1] < its[0]


def test_vcycle_spd_and_fewer_iterations():
    A = W.poisson3d(7, 6, 5)
    H = oracle.Hierarchy(A, smooth_p=True, max_coarse=10)
    assert H.num_levels >= 3
    B = np.column_stack([H.vcycle(e) for e in np.eye(A.n)])
    assert np.allclose(B, B.T, atol=1e-13 * np.abs(B).max())
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    A = W.poisson3d(32)
    b = np.random.default_rng(1).normal(size=A.n)
    its = {}
    for sp in (False, True):
        Hs = oracle.Hierarchy(A, smooth_p=sp)
        x, info = Hs.pcg(b, rtol=1e-6)
        assert info["status"] == 0
        assert np.linalg.norm(b - A.scipy() @ x) <= 1e-6 * np.linalg.norm(b)
        its[sp] = info["iterations"]
    assert its[True] < its[False]
