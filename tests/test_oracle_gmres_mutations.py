"""The GMRES oracle's pins have teeth: plausible mistakes planted one at a time in a copy of
``oracle.krylov.gmres`` (on the CPU) each make at least one pin fail, while the unmodified copy
passes them all.

Pins (independent of the code under test): the iterate after k Arnoldi steps has the minimum
residual over the Krylov space (numpy lstsq on a QR basis of [b, Ab, ...]), n steps give
numpy.linalg.solve's solution, restarted GMRES(5) converges to it, and a right-hand side in a
3-dimensional invariant subspace ends in 3 steps with the exact solution. (A looser breakdown
threshold is not among the mistakes: it ends a cycle early, and the restart's true residual makes
the result correct, only slower.)
"""
import numpy as np
import pytest

from oracle import krylov


def _gmres(mut):
    """oracle.krylov.gmres restated with one planted mistake (``mut``)."""
    def gmres(apply_A, b, tol, m, max_restarts, x0=None, norm_ref=None, history=None):
        b = np.asarray(b, dtype=np.complex128).ravel()
        n = b.size
        x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
        ref = float(np.linalg.norm(b)) if norm_ref is None else float(norm_ref)
        iters = 0
        relres = None
        for restart in range(max_restarts + 1):
            r = b if mut == "stale_restart_residual" else b - apply_A(x)
            beta = float(np.linalg.norm(r))
            relres = beta / ref
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
                for i in range(j + 1):
                    H[i, j] = np.vdot(w, V[i]) if mut == "dot_conjugate_swapped" else np.vdot(V[i], w)
                    w = w - H[i, j] * V[i]
                hnext = float(np.linalg.norm(w))
                H[j + 1, j] = hnext
                for i in range(j):
                    top, bot = H[i, j], H[i + 1, j]
                    H[i, j] = cs[i] * top + sn[i] * bot
                    s_conj = sn[i] if mut == "rotation_missing_conjugate" else np.conj(sn[i])
                    H[i + 1, j] = -s_conj * top + cs[i] * bot
                c, s, r_jj = krylov._givens(H[j, j], float(H[j + 1, j].real))
                cs[j], sn[j] = c, s
                H[j, j] = r_jj
                H[j + 1, j] = 0.0
                gamma[j + 1] = (np.conj(s) if mut == "gamma_sign" else -np.conj(s)) * gamma[j]
                gamma[j] = c * gamma[j]
                k = j + 1
                iters += 1
                if abs(gamma[j + 1]) <= tol * ref or hnext <= 1e-14 * w0:
                    break
                V[j + 1] = w / hnext
            y = np.zeros(k, dtype=np.complex128)
            for i in range(k - 1, -1, -1):
                acc = gamma[i] if mut == "backsub_drops_coupling" else gamma[i] - np.dot(H[i, i + 1:k], y[i + 1:k])
                y[i] = acc / H[i, i]
            x = x + (V[:k].T @ y if mut != "update_transposed_basis" else V[:k].conj().T @ y)
        return x, {"converged": False, "iterations": iters, "restarts": max_restarts, "relres": relres}
    return gmres


def _pin_minimum_residual(gm):
    rng = np.random.default_rng(1)
    n = 24
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 8 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for k in (3, 7):
        xk, _ = gm(lambda v: A @ v, b, tol=0.0, m=k, max_restarts=1)
        K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        if abs(np.linalg.norm(b - A @ xk) / np.linalg.norm(b - A @ Q @ y) - 1) > 1e-9:
            return False
    x, info = gm(lambda v: A @ v, b, tol=1e-13, m=n, max_restarts=1)
    return info["converged"] and np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-11 * np.linalg.norm(x)


def _pin_restarted(gm):
    rng = np.random.default_rng(2)
    n = 60
    A = rng.standard_normal((n, n)) / np.sqrt(n) + 3 * np.eye(n) + 1j * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n) + 0j
    x, info = gm(lambda v: A @ v, b, tol=1e-11, m=5, max_restarts=200)
    return info["converged"] and np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-9 * np.linalg.norm(x)


def _pin_happy_breakdown(gm):
    n = 30
    A = np.diag(np.arange(1.0, n + 1)).astype(complex)
    b = np.zeros(n, complex)
    b[[2, 9, 17]] = [1.0, 2.0, -1.0]
    x, info = gm(lambda v: A @ v, b, tol=1e-15, m=20, max_restarts=2)
    return info["converged"] and info["iterations"] == 3 and np.allclose(x, b / np.arange(1.0, n + 1))


PINS = {"minimum_residual": _pin_minimum_residual, "restarted": _pin_restarted,
        "happy_breakdown": _pin_happy_breakdown}


def _failing(gm):
    out = []
    for name, pin in PINS.items():
        with np.errstate(all="ignore"):
            try:
                ok = pin(gm)
            except (np.linalg.LinAlgError, ZeroDivisionError, FloatingPointError, ValueError):
                ok = False
        if not ok:
            out.append(name)
    return out


def test_oracle_gmres_and_its_copy_pass_every_pin():
    assert _failing(krylov.gmres) == []
    assert _failing(_gmres("none")) == []


@pytest.mark.parametrize("mut", ["stale_restart_residual", "dot_conjugate_swapped", "rotation_missing_conjugate",
                                 "gamma_sign", "backsub_drops_coupling", "update_transposed_basis"])
def test_planted_gmres_mistake_is_caught(mut):
    assert _failing(_gmres(mut)), f"no pin catches {mut}"
