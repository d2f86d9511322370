"""Spectral diagnostics of the GMRES(m) iteration, plain FP64 numpy (oracle; test infrastructure only).

Algorithm 2's inner loop builds an Arnoldi factorisation A V_m = V_{m+1} Hbar_m
(Hbar_m the (m+1) x m upper Hessenberg matrix). The polynomial by which one
GMRES(m) cycle multiplies the residual vanishes at the harmonic Ritz values of
A with respect to the Krylov space K_m(A, r0): the values theta for which some
nonzero u = V_m y satisfies the Petrov-Galerkin condition

    A u - theta u  is orthogonal to  A K_m,

equivalently the eigenvalues of H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^T with
H_m the square top of Hbar_m. When the smallest harmonic Ritz values sit close
to the origin relative to the rest of the spectrum seen by the cycle, a
restarted GMRES of that length makes little progress per cycle (the residual
polynomial must be 1 at 0 and 0 near 0). These functions are used to report
that diagnostic for the large lattice; they are not part of the solver.
"""
from __future__ import annotations

import numpy as np


def arnoldi(apply_A, v0: np.ndarray, m: int, breakdown: float = 1e-14):
    """m steps of Arnoldi with modified Gram-Schmidt from v0 (flattened complex vector).

    Returns (V, Hbar): V is (k+1) x n with orthonormal rows (V[0] = v0/||v0||),
    Hbar is (k+1) x k with A V[:k]^T = V^T Hbar; k = m unless a breakdown
    (H[j+1, j] <= breakdown * ||A v_j||) stops the process early.
    """
    v0 = np.asarray(v0, dtype=np.complex128).ravel()
    n = v0.size
    V = np.zeros((m + 1, n), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    V[0] = v0 / np.linalg.norm(v0)
    k = m
    for j in range(m):
        w = np.asarray(apply_A(V[j]), dtype=np.complex128).ravel()
        w0 = float(np.linalg.norm(w))
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        h = float(np.linalg.norm(w))
        H[j + 1, j] = h
        if h <= breakdown * w0:
            k = j + 1
            break
        V[j + 1] = w / h
    return V[:k + 1], H[:k + 1, :k]


def harmonic_ritz(Hbar: np.ndarray) -> np.ndarray:
    """Harmonic Ritz values from an Arnoldi Hessenberg matrix Hbar ((k+1) x k), sorted by modulus."""
    k = Hbar.shape[1]
    Hm = Hbar[:k, :k]
    h = Hbar[k, k - 1]
    ek = np.zeros(k, dtype=np.complex128)
    ek[-1] = 1.0
    f = np.linalg.solve(Hm.conj().T, ek)
    theta = np.linalg.eigvals(Hm + (abs(h) ** 2) * np.outer(f, ek))
    return theta[np.argsort(np.abs(theta))]


def ritz(Hbar: np.ndarray) -> np.ndarray:
    """Ritz values (eigenvalues of the square top H_m), sorted by modulus."""
    k = Hbar.shape[1]
    theta = np.linalg.eigvals(Hbar[:k, :k])
    return theta[np.argsort(np.abs(theta))]
