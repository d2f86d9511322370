"""Pins of the oracle's restarted GMRES (Algorithm 2) against library solves and exact properties."""
import numpy as np
import pytest

import oracle
from oracle import krylov as og
import synthetic as syn


def test_givens_least_squares_matches_lstsq():
    """One unrestarted cycle on a random system: gamma after the rotations gives
    exactly the least-squares residual of numpy's lstsq on the Hessenberg matrix,
    and after n steps the solution is numpy.linalg.solve's."""
    rng = np.random.default_rng(1)
    n = 24
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 8 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    hist = []
    x, info = og.gmres(lambda v: A @ v, b, tol=1e-13, m=n, max_restarts=1, history=hist)
    assert info["converged"]
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-11 * np.linalg.norm(x)
    # The Arnoldi estimate after k steps is the minimum residual over the Krylov space:
    # compare with lstsq on the Krylov basis built independently by QR of [b, Ab, ...].
    for k in (3, 7):
        xk, _ = og.gmres(lambda v: A @ v, b, tol=0.0, m=k, max_restarts=1)
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        assert np.linalg.norm(b - A @ xk) == pytest.approx(np.linalg.norm(b - A @ Q @ y), rel=1e-9)


def test_restarted_gmres_dense_random():
    """Restarted GMRES(5) on a well-conditioned system converges to numpy.linalg.solve."""
    rng = np.random.default_rng(2)
    n = 60
    A = rng.standard_normal((n, n)) / np.sqrt(n) + 3 * np.eye(n) + 1j * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n) + 0j
    x, info = og.gmres(lambda v: A @ v, b, tol=1e-11, m=5, max_restarts=200)
    assert info["converged"] and info["restarts"] > 1
    assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-9 * np.linalg.norm(x)


def test_happy_breakdown():
    """A rhs inside a 3-dimensional invariant subspace: GMRES stops after 3 steps, exact."""
    n = 30
    A = np.diag(np.arange(1.0, n + 1)).astype(complex)
    b = np.zeros(n, complex)
    b[[2, 9, 17]] = [1.0, 2.0, -1.0]
    x, info = og.gmres(lambda v: A @ v, b, tol=1e-15, m=20, max_restarts=2)
    assert info["converged"] and info["iterations"] == 3
    assert np.allclose(x, b / np.arange(1.0, n + 1))


def test_gmres_wilson_2x4_vs_dense_solve():
    """Full and odd-even solves on 2^4 (clover) match a dense LU solve."""
    dims = (2, 2, 2, 2)
    U = syn.gauge_field(dims, "exp", 0.4, seed=3)
    m0, c_sw = 0.1, 1.0
    C = oracle.clover_term(U, c_sw)
    A, Ainv = oracle.diag_blocks(U, m0, c_sw)
    D = oracle.dense_operator(U, m0, C)
    b = syn.gaussian_spinors(dims, 2, 4)
    ref = np.linalg.solve(D, b.reshape(2, -1).T).T.reshape(b.shape)
    x, infos = oracle.solve_full(U, C, m0, b, tol=1e-12, m=10, max_restarts=100)
    assert all(i["converged"] for i in infos)
    assert np.linalg.norm(x - ref) < 1e-9 * np.linalg.norm(ref)
    xe, infos = oracle.solve_eo(U, A, Ainv, b, tol=1e-12, m=10, max_restarts=100)
    assert all(i["converged"] for i in infos)
    assert np.linalg.norm(xe - ref) < 1e-9 * np.linalg.norm(ref)


def test_gmres_4x4_haar_wilson_full_eo():
    """The 4^4 Haar Wilson case (m0 = 0.1, GMRES(30), 1e-10): full and odd-even both
    reach the tolerance on the TRUE residual, agree with a dense solve, and the
    odd-even solve needs fewer iterations."""
    dims = (4, 4, 4, 4)
    U = syn.gauge_field(dims, "haar", seed=0 * 1000 + 0)
    m0 = 0.1
    b = syn.gaussian_spinors(dims, 1, 1)
    A, Ainv = oracle.diag_blocks(U, m0, 0.0)
    x, inf_full = oracle.solve_full(U, None, m0, b, tol=1e-10, m=30, max_restarts=50)
    xe, inf_eo = oracle.solve_eo(U, A, Ainv, b, tol=1e-10, m=30, max_restarts=50)
    for xx, inf in ((x, inf_full), (xe, inf_eo)):
        assert inf[0]["converged"]
        r = b - oracle.apply_D(U, xx, m0)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    D = oracle.dense_operator(U, m0)
    ref = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(x - ref) < 1e-8 * np.linalg.norm(ref)
    assert np.linalg.norm(xe - ref) < 1e-8 * np.linalg.norm(ref)
    assert inf_eo[0]["iterations"] < inf_full[0]["iterations"]
