"""Pins of the oracle's Arnoldi factorisation and harmonic Ritz values (oracle/spectrum.py).

The harmonic Ritz values are checked against their definition (the Petrov-Galerkin
condition with test space A K_m, a generalised eigenproblem solved by scipy) rather
than against the Hessenberg formula that computes them, and against the exact
spectrum where the Krylov space is invariant.
"""
import numpy as np
import pytest

import oracle
from oracle import spectrum
import synthetic as syn

scipy_linalg = pytest.importorskip("scipy.linalg")


def _random_matrix(n, seed, shift=2.0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n) + shift * np.eye(n)


def test_arnoldi_relation_and_orthonormality():
    A = _random_matrix(40, 1)
    v0 = np.random.default_rng(2).standard_normal(40) + 0j
    V, H = spectrum.arnoldi(lambda v: A @ v, v0, 12)
    assert V.shape == (13, 40) and H.shape == (13, 12)
    assert np.linalg.norm(V.conj() @ V.T - np.eye(13)) < 1e-13
    assert np.linalg.norm(A @ V[:12].T - V.T @ H) < 1e-12 * np.linalg.norm(A)
    assert np.allclose(np.tril(H, -2), 0)


def test_harmonic_ritz_values_satisfy_petrov_galerkin_definition():
    """theta with (A V y - theta V y) orthogonal to A V: eig of ((AV)^H AV, (AV)^H V)."""
    A = _random_matrix(50, 3, shift=0.3)
    v0 = np.random.default_rng(4).standard_normal(50) + 1j
    for m in (5, 11, 20):
        V, H = spectrum.arnoldi(lambda v: A @ v, v0, m)
        W = A @ V[:m].T
        ref = scipy_linalg.eigvals(W.conj().T @ W, W.conj().T @ V[:m].T)
        ref = ref[np.argsort(np.abs(ref))]
        got = spectrum.harmonic_ritz(H)
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-11)


def test_invariant_subspace_gives_exact_eigenvalues():
    """A start vector in a 4-dimensional invariant subspace: Arnoldi breaks down after 4
    steps and both Ritz and harmonic Ritz values are the 4 eigenvalues of that subspace."""
    lam = np.array([0.05 + 0.2j, 1.0, -0.7j, 3.0 - 1.0j] + list(np.linspace(5, 9, 26)))
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30)))
    A = Q @ np.diag(lam) @ Q.conj().T
    v0 = Q[:, :4] @ np.array([1.0, 2.0, -1.0, 0.5])
    V, H = spectrum.arnoldi(lambda v: A @ v, v0, 10, breakdown=1e-10)
    assert H.shape == (5, 4)
    ref = lam[:4][np.argsort(np.abs(lam[:4]))]
    assert np.allclose(spectrum.harmonic_ritz(H), ref, atol=1e-10)
    assert np.allclose(spectrum.ritz(H), ref, atol=1e-10)


def test_schur_operator_arnoldi_and_harmonic_ritz_definition():
    """The same checks with the oracle's Schur operator on 2^4 as A: the Arnoldi relation
    holds and the harmonic Ritz values satisfy the Petrov-Galerkin definition."""
    dims = (2, 2, 2, 2)
    U = syn.gauge_field(dims, "exp", 0.4, seed=6)
    A_blk, Ainv = oracle.diag_blocks(U, -0.3, 1.0)
    n_half = 8

    def S(v):
        return oracle.apply_schur(U, A_blk, Ainv, v.reshape(1, n_half, 4, 3)).ravel()

    v0 = oracle.split_parity(syn.gaussian_spinors(dims, 1, 7), 1).ravel()
    m = 16
    V, H = spectrum.arnoldi(S, v0, m)
    SV = np.stack([S(V[j]) for j in range(m)], axis=1)
    assert np.linalg.norm(SV - V.T @ H) < 1e-12 * np.linalg.norm(SV)
    ref = scipy_linalg.eigvals(SV.conj().T @ SV, SV.conj().T @ V[:m].T)
    ref = ref[np.argsort(np.abs(ref))]
    assert np.allclose(spectrum.harmonic_ritz(H), ref, rtol=1e-9, atol=1e-11)
