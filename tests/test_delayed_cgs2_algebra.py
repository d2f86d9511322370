"""The delayed CGS2 Arnoldi step, restated in numpy, against the plain Arnoldi factorisation.

The GPU solver's default Gram-Schmidt keeps once-orthogonalised candidates q~_i in the basis
slots and a triangular factor T with Q~ = Q T (Q the orthonormal Arnoldi basis, never formed),
and finalises the Hessenberg column of step j from the second pass of the same step:
  z = T^{-H} (Q~^H w),  nu^2 = ||w||^2 - ||z||^2,  q~_{j+1} = (w - Q~ T^{-1} z) / nu,
  a = T^{-H} (Q~^H q~_{j+1}),  rho^2 = ||q~_{j+1}||^2 - ||a||^2,
  H[:j+1, j] = (z + nu a - H[:j+1, :j] a_j) / rho_j,  H[j+1, j] = nu rho / rho_j,
with T gaining the column [a; rho]. This file checks those recurrences (written here from the
algebra, independently of the CUDA kernels) against the Arnoldi relation A Q_k = Q_{k+1} H,
the orthonormality of Q = Q~ T^{-1}, and a modified Gram-Schmidt Arnoldi run from the same
start vector (the factorisation with a positive subdiagonal is unique), also with pass B's
projection perturbed so that the stored candidates are far from orthogonal.
"""
import numpy as np
import pytest
from scipy.linalg import solve_triangular


def arnoldi_mgs(A, r, m):
    n = r.size
    Q = np.zeros((n, m + 1), complex)
    H = np.zeros((m + 1, m), complex)
    Q[:, 0] = r / np.linalg.norm(r)
    for j in range(m):
        w = A @ Q[:, j]
        for i in range(j + 1):
            H[i, j] = np.vdot(Q[:, i], w)
            w = w - H[i, j] * Q[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        Q[:, j + 1] = w / H[j + 1, j]
    return Q, H


def arnoldi_delayed_cgs2(A, r, m, perturb=0.0, rng=None):
    """Returns (Q~, T, H): the stored candidates, their triangular factor and the Hessenberg matrix.

    perturb > 0 replaces the projection z used by pass B with z + perturb * (random): the candidates
    are then far from orthogonal to the basis (a = O(perturb)), which the recurrences must absorb
    exactly (w = Q z + nu q~_{j+1} holds for whatever z pass B used)."""
    n = r.size
    Qt = np.zeros((n, m + 1), complex)
    T = np.zeros((m + 1, m + 1), complex)
    H = np.zeros((m + 1, m), complex)
    Qt[:, 0] = r / np.linalg.norm(r)
    T[0, 0] = 1.0
    for j in range(m):
        k = j + 1
        Tk = T[:k, :k]
        w = A @ Qt[:, j]
        # pass A: projections on the stored candidates and the norm of w
        e = Qt[:, :k].conj().T @ w
        omega = np.vdot(w, w).real
        z = solve_triangular(Tk.conj().T, e, lower=True)
        nu = np.sqrt(max(omega - np.vdot(z, z).real, 1e-12 * omega))
        if perturb:
            z = z + perturb * np.linalg.norm(z) * (rng.standard_normal(k) + 1j * rng.standard_normal(k))
        g = solve_triangular(Tk, z)
        # pass B: the next candidate, its projections and norm
        w1 = w - Qt[:, :k] @ g
        Qt[:, k] = w1 / nu
        d = Qt[:, :k].conj().T @ w1
        alpha = np.vdot(w1, w1).real / nu ** 2
        a = solve_triangular(Tk.conj().T, d / nu, lower=True)
        rho = np.sqrt(max(alpha - np.vdot(a, a).real, 0.0))
        # final column j of the Hessenberg matrix
        col = z + nu * a - H[:k, :j] @ T[:j, j]
        H[:k, j] = col / T[j, j].real
        H[k, j] = nu * rho / T[j, j].real
        T[:k, k] = a
        T[k, k] = rho
    return Qt, T, H


def _matrix(kind, n, rng):
    if kind == "shifted-random":  # well conditioned, non-normal
        return np.eye(n) * 3.0 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    if kind == "graded":  # widely spread eigenvalues: the Krylov vectors align fast
        X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        lam = np.logspace(0, 6, n) * np.exp(1j * rng.uniform(0, 0.3, n))
        return X @ np.diag(lam) @ np.linalg.inv(X)
    raise ValueError(kind)


@pytest.mark.parametrize("perturb", [0.0, 1e-2])
@pytest.mark.parametrize("kind,n,m", [("shifted-random", 200, 32), ("graded", 120, 24), ("shifted-random", 40, 1)])
def test_delayed_cgs2_gives_the_arnoldi_factorisation(kind, n, m, perturb):
    rng = np.random.default_rng(n + m)
    A = _matrix(kind, n, rng)
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Qt, T, H = arnoldi_delayed_cgs2(A, r, m, perturb, np.random.default_rng(1))
    Q = solve_triangular(T.T, Qt.T, lower=True).T  # Q = Q~ T^{-1}
    scale = np.linalg.norm(A, 2)
    # orthonormal basis
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(m + 1)) < 1e-12
    # Arnoldi relation A Q_m = Q_{m+1} H
    assert np.linalg.norm(A @ Q[:, :m] - Q @ H) < 1e-11 * scale
    # T upper triangular with a positive diagonal, H upper Hessenberg with a positive subdiagonal
    assert np.allclose(np.tril(T, -1), 0) and np.all(np.diag(T).real > 0)
    assert np.allclose(np.tril(H, -2), 0) and np.all(np.diag(H, -1).real > 0)
    # the same factorisation as modified Gram-Schmidt from the same start vector (leading columns: rounding
    # differences grow with the condition of the Krylov basis further on, while both satisfy the relation)
    Qm, Hm = arnoldi_mgs(A, r, m)
    c = min(m, 8)
    assert np.linalg.norm(H[:c + 1, :c] - Hm[:c + 1, :c]) < 1e-10 * scale
    assert np.linalg.norm(Q[:, :c + 1] - Qm[:, :c + 1]) < 1e-9


def test_delayed_cgs2_gmres_update_uses_t_inverse():
    """x = Q_k y = Q~_k (T_k^{-1} y): the GMRES correction from the stored candidates."""
    rng = np.random.default_rng(7)
    n, m = 150, 20
    A = _matrix("shifted-random", n, rng)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Qt, T, H = arnoldi_delayed_cgs2(A, b, m)
    beta = np.linalg.norm(b)
    rhs = np.zeros(m + 1, complex)
    rhs[0] = beta
    y, *_ = np.linalg.lstsq(H, rhs, rcond=None)
    x = Qt[:, :m] @ solve_triangular(T[:m, :m], y)
    Qm, Hm = arnoldi_mgs(A, b, m)
    ym, *_ = np.linalg.lstsq(Hm, rhs, rcond=None)
    xm = Qm[:, :m] @ ym
    assert np.linalg.norm(x - xm) < 1e-10 * np.linalg.norm(xm)
    # the GMRES residual is the least-squares residual
    assert abs(np.linalg.norm(b - A @ x) - np.linalg.norm(rhs - H @ y)) < 1e-9 * beta


def test_dropped_correction_term_is_detected():
    """Without the -H[:, :j] a_j term the relation fails: the check has teeth (candidates made
    non-orthogonal by a perturbed pass-B projection, so that a_j is not at rounding level)."""
    rng = np.random.default_rng(3)
    n, m = 120, 16
    A = _matrix("shifted-random", n, rng)
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Qt, T, H = arnoldi_delayed_cgs2(A, r, m, 1e-2, np.random.default_rng(2))
    Q = solve_triangular(T.T, Qt.T, lower=True).T
    Hbad = H.copy()
    for j in range(1, m):  # recompute the columns without the correction
        k = j + 1
        Hbad[:k, j] = H[:k, j] + (H[:k, :j] @ T[:j, j]) / T[j, j].real
    assert np.linalg.norm(A @ Q[:, :m] - Q @ Hbad) > 1e-6 * np.linalg.norm(A, 2)
