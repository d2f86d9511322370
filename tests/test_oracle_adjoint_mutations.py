"""The adjoint oracle's finite-difference pin has teeth: plausible mistakes planted one at a time in
copies of ``oracle.adjoint.hopping_gradient`` and ``clover_gradient`` (on the CPU) each break the
agreement of the gradient with central finite differences of L = sum_i Re <eta_i, D^{-1} b_i>
(dense operator built entry by entry, exact dense solves), while the unmodified copies agree.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint, dirac
import synthetic as syn

DIMS = (4, 2, 2, 4)
M0, CSW = 0.3, 1.0


def _hopping_gradient(mut):
    def grad(U, x, lam, bc=-1.0):
        g = dirac.gamma_matrices()
        one = np.eye(4, dtype=np.complex128)
        G = np.zeros(U.shape, dtype=np.complex128)
        for mu in range(4):
            pi_minus, pi_plus = (one - g[mu]) / 2, (one + g[mu]) / 2
            if mut == "swapped_projectors":
                pi_minus, pi_plus = pi_plus, pi_minus
            x_fwd = np.roll(x, 1 if mut == "wrong_roll" else -1, axis=1 + mu)
            lam_fwd = np.roll(lam, -1, axis=1 + mu)
            M = np.einsum("ntzyxsa,ntzyxsb->tzyxab", np.conj(lam), dirac._spin(pi_minus, x_fwd))
            N = np.einsum("ntzyxsa,ntzyxsb->tzyxab", np.conj(lam_fwd), dirac._spin(pi_plus, x))
            first = M if mut == "missing_conjugate" else np.conj(M)
            second = N if mut == "missing_transpose" else np.swapaxes(N, -1, -2)
            G[..., mu, :, :] = first + second
        f = np.ones(tuple(U.shape[:4]) + (4,))
        if mut != "missing_boundary_factor":
            f[-1, :, :, :, 0] = bc
        return G * f[..., None, None]
    return grad


def _clover_gradient(mut):
    def grad(U, x, lam, c_sw):
        G = np.zeros(U.shape, dtype=np.complex128)
        g = dirac.gamma_matrices()
        for mu in range(4):
            for nu in range(4):
                if mu == nu:
                    continue
                gx = dirac._spin(g[mu] @ g[nu], x)
                W = (c_sw / 32.0) * np.einsum("ntzyxsb,ntzyxsa->tzyxba", gx, np.conj(lam))
                pairs = ((mu, nu, 1.0), (nu, mu, 1.0 if mut == "second_term_sign" else -1.0))
                for (m1, n1, weight) in pairs:
                    for leaf in adjoint._LEAVES:
                        fac = [adjoint._factor(U, f, m1, n1) for f in leaf]
                        for p, f in enumerate(leaf):
                            eye = np.broadcast_to(np.eye(3, dtype=np.complex128), W.shape)
                            A = eye
                            for q in range(p):
                                A = A @ fac[q]
                            B = eye
                            for q in range(p + 1, 4):
                                B = B @ fac[q]
                            K = weight * ((A @ W @ B) if mut == "wrong_cyclic_order" else (B @ W @ A))
                            name, off, dag = f
                            rho = m1 if name == "mu" else n1
                            Ky = K
                            for nm, s in off.items():
                                Ky = np.roll(Ky, s, axis=m1 if nm == "mu" else n1)
                            if mut == "dagger_swapped":
                                dag = not dag
                            G[..., rho, :, :] += Ky if dag else dirac._dag(Ky)
        return G
    return grad


def _setup():
    U = syn.gauge_field(DIMS, "exp", 0.35, seed=31)
    b = syn.gaussian_spinors(DIMS, 2, 32)
    eta = syn.gaussian_spinors(DIMS, 2, 33)
    C = oracle.clover_term(U, CSW)
    D = oracle.dense_operator(U, M0, C)
    n = b.shape[0]
    x = np.linalg.solve(D, b.reshape(n, -1).T).T.reshape(b.shape)
    lam = np.linalg.solve(D.conj().T, eta.reshape(n, -1).T).T.reshape(eta.shape)
    return U, b, eta, x, lam


def _loss(U, b, eta):
    D = oracle.dense_operator(U, M0, oracle.clover_term(U, CSW))
    n = b.shape[0]
    x = np.linalg.solve(D, b.reshape(n, -1).T).T.reshape(b.shape)
    return adjoint.loss(x, eta)


@pytest.fixture(scope="module")
def fd_reference():
    """Central differences of L along three fixed random link directions."""
    U, b, eta, x, lam = _setup()
    rng = np.random.default_rng(5)
    h = 1e-6
    dirs = [rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape) for _ in range(3)]
    fds = [(_loss(U + h * d, b, eta) - _loss(U - h * d, b, eta)) / (2 * h) for d in dirs]
    return U, x, lam, dirs, fds


def _agrees(G, dirs, fds):
    return all(abs(fd - float(np.real(np.vdot(G, d)))) <= 2e-7 * max(1.0, abs(fd)) for d, fd in zip(dirs, fds))


def test_unmodified_copies_agree_with_finite_differences(fd_reference):
    U, x, lam, dirs, fds = fd_reference
    assert _agrees(adjoint.hopping_gradient(U, x, lam) + adjoint.clover_gradient(U, x, lam, CSW), dirs, fds)
    assert _agrees(_hopping_gradient("none")(U, x, lam) + _clover_gradient("none")(U, x, lam, CSW), dirs, fds)


@pytest.mark.parametrize("mut", ["swapped_projectors", "wrong_roll", "missing_conjugate", "missing_transpose",
                                 "missing_boundary_factor"])
def test_planted_hopping_gradient_mistake_is_caught(fd_reference, mut):
    U, x, lam, dirs, fds = fd_reference
    G = _hopping_gradient(mut)(U, x, lam) + adjoint.clover_gradient(U, x, lam, CSW)
    assert not _agrees(G, dirs, fds)


@pytest.mark.parametrize("mut", ["second_term_sign", "wrong_cyclic_order", "dagger_swapped"])
def test_planted_clover_gradient_mistake_is_caught(fd_reference, mut):
    U, x, lam, dirs, fds = fd_reference
    G = adjoint.hopping_gradient(U, x, lam) + _clover_gradient(mut)(U, x, lam, CSW)
    assert not _agrees(G, dirs, fds)
