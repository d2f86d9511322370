"""Restarted GMRES (Algorithm 2), plain FP64 numpy (oracle; test infrastructure only).

Algorithm 2 runs b right-hand sides in lockstep but each one independently
(no block Krylov space, Sec. III-A-2), so the oracle solves them one at a time
with the same steps:

* restart: r = eta - D psi, beta = ||r||, V[0] = r / beta;
* inner step j: one Arnoldi step (modified Gram-Schmidt) giving column j of
  the Hessenberg matrix H, the earlier Givens rotations applied to it, a new
  rotation that annihilates H[j+1, j], and the update of gamma;
  relnorm = |gamma[j+1]| / ||eta||;
* after the inner loop: psi += V y with y the least-squares solution of
  min || gamma - H y || (back substitution on the rotated triangle).

Readings of points the paper leaves open: the initial guess is zero unless one
is given; the inner loop stops at relnorm <= tol, at a happy breakdown
(H[j+1, j] <= 1e-14 * ||w before orthogonalisation||) or at the restart
length; a rhs is finished when the TRUE residual ||eta - D psi|| / ||eta||
recomputed at the restart is <= tol (the paper stops on the Arnoldi estimate;
the true residual is the stricter test). Givens convention, for a = H[j, j] and
h = H[j+1, j] >= 0, rho = sqrt(|a|^2 + h^2): c = |a| / rho, s = (a/|a|) h / rho
(c = 0, s = 1 when a = 0); the rotation maps (top, bottom) to
(c top + s bottom, -conj(s) top + c bottom), so gamma[j+1] = -conj(s) gamma[j]
and gamma[j] = c gamma[j].
"""
from __future__ import annotations

import numpy as np

from . import dirac


def _givens(a: complex, h: float):
    rho = np.sqrt(abs(a) ** 2 + h * h)
    if rho == 0.0:
        return 1.0, 0.0 + 0.0j, 0.0 + 0.0j
    if a == 0:
        return 0.0, 1.0 + 0.0j, complex(rho)
    phase = a / abs(a)
    return abs(a) / rho, phase * h / rho, phase * rho


def gmres(apply_A, b: np.ndarray, tol: float, m: int, max_restarts: int,
          x0: np.ndarray | None = None, norm_ref: float | None = None, history=None):
    """Solve A x = b for one rhs (flattened complex vector).

    Stops when ||b - A x|| <= tol * norm_ref (norm_ref defaults to ||b||).
    Returns (x, info) with info = {"converged", "iterations", "restarts", "relres"}.
    """
    b = np.asarray(b, dtype=np.complex128).ravel()
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    ref = float(np.linalg.norm(b)) if norm_ref is None else float(norm_ref)
    if ref == 0.0:
        return np.zeros(n, dtype=np.complex128), {"converged": True, "iterations": 0,
                                                  "restarts": 0, "relres": 0.0}
    iters = 0
    relres = None
    for restart in range(max_restarts + 1):
        r = b - apply_A(x)
        beta = float(np.linalg.norm(r))
        relres = beta / ref
        if history is not None:
            history.append(relres)
        if beta <= tol * ref:
            return x, {"converged": True, "iterations": iters, "restarts": restart, "relres": relres}
        if restart == max_restarts:
            break
        V = np.zeros((m + 1, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        gamma = np.zeros(m + 1, dtype=np.complex128)
        gamma[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = apply_A(V[j])
            w0 = float(np.linalg.norm(w))
            for i in range(j + 1):                    # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            hnext = float(np.linalg.norm(w))
            H[j + 1, j] = hnext
            for i in range(j):                        # earlier rotations
                top, bot = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * top + sn[i] * bot
                H[i + 1, j] = -np.conj(sn[i]) * top + cs[i] * bot
            c, s, r_jj = _givens(H[j, j], float(H[j + 1, j].real))
            cs[j], sn[j] = c, s
            H[j, j] = r_jj
            H[j + 1, j] = 0.0
            gamma[j + 1] = -np.conj(s) * gamma[j]
            gamma[j] = c * gamma[j]
            k = j + 1
            iters += 1
            if abs(gamma[j + 1]) <= tol * ref or hnext <= 1e-14 * w0:
                break
            V[j + 1] = w / hnext
        y = np.zeros(k, dtype=np.complex128)            # back substitution R y = gamma
        for i in range(k - 1, -1, -1):
            y[i] = (gamma[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + V[:k].T @ y
    return x, {"converged": False, "iterations": iters, "restarts": max_restarts, "relres": relres}


def solve_full(U, C, m0, b_block, tol, m=30, max_restarts=200, bc=-1.0):
    """Batched GMRES on D x = b (each rhs independently). Returns (x_block, infos)."""
    xs, infos = [], []
    for k in range(b_block.shape[0]):
        shape = b_block[k:k + 1].shape

        def A(v, shape=shape):
            return dirac.apply_D(U, v.reshape(shape), m0, C, bc).ravel()

        x, info = gmres(A, b_block[k].ravel(), tol, m, max_restarts)
        xs.append(x.reshape(b_block.shape[1:]))
        infos.append(info)
    return np.stack(xs), infos


def solve_eo(U, A_blocks, Ainv_blocks, b_block, tol, m=30, max_restarts=200, bc=-1.0):
    """Odd-even (Schur) batched GMRES on S x_o = hat b_o, then x_e reconstructed.

    The Schur solve stops at ||hat b_o - S x_o|| <= tol * ||b||, ||b|| the norm
    of the full rhs; with x_e reconstructed exactly this equals the full
    residual ||b - D x||.
    """
    dims = U.shape[:4]
    b_e = dirac.split_parity(b_block, 0)
    b_o = dirac.split_parity(b_block, 1)
    bhat = dirac.schur_prepare(U, Ainv_blocks, b_e, b_o, bc)
    xs, infos = [], []
    for k in range(b_block.shape[0]):
        shape = bhat[k:k + 1].shape

        def S(v, shape=shape):
            return dirac.apply_schur(U, A_blocks, Ainv_blocks, v.reshape(shape), bc).ravel()

        ref = float(np.linalg.norm(b_block[k]))
        x_o, info = gmres(S, bhat[k].ravel(), tol, m, max_restarts, norm_ref=ref)
        x_o = x_o.reshape(shape)
        x_e = dirac.schur_reconstruct(U, Ainv_blocks, b_e[k:k + 1], x_o, bc)
        full = dirac.embed_parity(x_e, 0, dims) + dirac.embed_parity(x_o, 1, dims)
        xs.append(full[0])
        infos.append(info)
    return np.stack(xs), infos
