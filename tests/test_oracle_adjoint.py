"""Pins of the oracle's adjoint (dL/db and dL/dU for L = sum_i Re <eta_i, D^{-1} b_i>).

Every gradient is checked against central finite differences of the loss computed
with the brute-force dense operator (``oracle.dense_operator``, built entry by entry)
and an exact dense solve, on lattices where x + mu and x - mu coincide (2^4) or where
the time boundary and non-cubic extents matter (4x2x2x4). The adjoint operator is
pinned by <phi, D psi> = <D^dag phi, psi>, by gamma5-hermiticity and by the dense
conjugate transpose.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint
import synthetic as syn

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _setup(dims, eps, seed, nrhs=2):
    U = syn.gauge_field(dims, "exp", eps, seed=seed)
    b = syn.gaussian_spinors(dims, nrhs, seed + 1)
    eta = syn.gaussian_spinors(dims, nrhs, seed + 2)
    return U, b, eta


def _dense_loss(U, m0, c_sw, b, eta):
    C = oracle.clover_term(U, c_sw) if c_sw else None
    D = oracle.dense_operator(U, m0, C)
    n = b.shape[0]
    x = np.linalg.solve(D, b.reshape(n, -1).T).T.reshape(b.shape)
    return adjoint.loss(x, eta)


def _dense_x_lam(U, m0, c_sw, b, eta):
    C = oracle.clover_term(U, c_sw) if c_sw else None
    D = oracle.dense_operator(U, m0, C)
    n = b.shape[0]
    x = np.linalg.solve(D, b.reshape(n, -1).T).T.reshape(b.shape)
    lam = np.linalg.solve(D.conj().T, eta.reshape(n, -1).T).T.reshape(eta.shape)
    return x, lam


@pytest.mark.parametrize("c_sw", [0.0, 1.3])
def test_adjoint_operator(c_sw):
    dims = (4, 2, 2, 4)
    U, psi, phi = _setup(dims, 0.4, 11)
    C = oracle.clover_term(U, c_sw) if c_sw else None
    m0 = -0.1
    Dpsi = oracle.apply_D(U, psi, m0, C)
    Ddphi = adjoint.apply_D_dagger(U, phi, m0, C)
    assert abs(np.vdot(phi, Dpsi) - np.vdot(Ddphi, psi)) < 1e-12 * np.linalg.norm(phi) * np.linalg.norm(Dpsi)
    # gamma5-hermiticity: D^dag = gamma5 D gamma5
    g5 = oracle.gamma5()
    g5phi = np.einsum("st,n...tc->n...sc", g5, phi)
    ref = np.einsum("st,n...tc->n...sc", g5, oracle.apply_D(U, g5phi, m0, C))
    assert np.linalg.norm(Ddphi - ref) < 1e-13 * np.linalg.norm(ref)


def test_adjoint_matches_dense_conjugate_transpose():
    dims = (2, 2, 2, 2)
    U, psi, _ = _setup(dims, 0.5, 21, nrhs=1)
    C = oracle.clover_term(U, 1.0)
    D = oracle.dense_operator(U, 0.2, C)
    got = adjoint.apply_D_dagger(U, psi, 0.2, C).reshape(-1)
    assert np.allclose(got, D.conj().T @ psi.reshape(-1), atol=1e-13)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
@pytest.mark.parametrize("c_sw", [0.0, 1.0])
def test_gradient_U_matches_finite_differences(dims, c_sw):
    """Directional derivative along random complex link perturbations (all links) and along
    single link entries (real and imaginary), hopping and clover parts together."""
    m0 = 0.3
    U, b, eta = _setup(dims, 0.35, 31)
    x, lam = _dense_x_lam(U, m0, c_sw, b, eta)
    G = adjoint.hopping_gradient(U, x, lam) + adjoint.clover_gradient(U, x, lam, c_sw)
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(2):
        dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
        fd = (_dense_loss(U + h * dU, m0, c_sw, b, eta) - _dense_loss(U - h * dU, m0, c_sw, b, eta)) / (2 * h)
        an = float(np.real(np.vdot(G, dU)))
        assert abs(fd - an) <= 2e-7 * max(1.0, abs(an)), (fd, an)
    # single entries: a time link on the last slice (boundary factor), a space link
    for idx in [(dims[0] - 1, 0, 1, 1, 0, 2, 1), (0, 1, 0, 1, 3, 0, 0), (1, 0, 1, 0, 1, 1, 2)]:
        for unit in (1.0, 1j):
            dU = np.zeros_like(U)
            dU[idx] = unit
            fd = (_dense_loss(U + h * dU, m0, c_sw, b, eta) - _dense_loss(U - h * dU, m0, c_sw, b, eta)) / (2 * h)
            an = float(np.real(np.conj(G[idx]) * unit))
            assert abs(fd - an) <= 2e-7 * max(1.0, abs(an)), (idx, unit, fd, an)


def test_clover_gradient_alone_matches_finite_differences():
    """The clover part by itself: L as a function of the links inside C only (hopping links fixed)."""
    dims = (4, 2, 2, 4)
    m0, c_sw = 0.3, 1.5
    U, b, eta = _setup(dims, 0.35, 41)
    x, lam = _dense_x_lam(U, m0, c_sw, b, eta)
    Gc = adjoint.clover_gradient(U, x, lam, c_sw)

    def L_clover_only(Uc):
        C = oracle.clover_term(Uc, c_sw)
        D = oracle.dense_operator(U, m0, C)
        n = b.shape[0]
        xx = np.linalg.solve(D, b.reshape(n, -1).T).T.reshape(b.shape)
        return adjoint.loss(xx, eta)

    rng = np.random.default_rng(9)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    h = 1e-6
    fd = (L_clover_only(U + h * dU) - L_clover_only(U - h * dU)) / (2 * h)
    an = float(np.real(np.vdot(Gc, dU)))
    assert abs(fd - an) <= 2e-7 * max(1.0, abs(an)), (fd, an)
    assert np.linalg.norm(Gc) > 1e-3 * np.linalg.norm(adjoint.hopping_gradient(U, x, lam))


def test_gradient_b_and_su3_projection():
    dims = (4, 2, 2, 4)
    m0, c_sw = 0.3, 1.0
    U, b, eta = _setup(dims, 0.35, 51)
    x, lam = _dense_x_lam(U, m0, c_sw, b, eta)
    rng = np.random.default_rng(3)
    db = rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape)
    h = 1e-6
    fd = (_dense_loss(U, m0, c_sw, b + h * db, eta) - _dense_loss(U, m0, c_sw, b - h * db, eta)) / (2 * h)
    assert abs(fd - np.real(np.vdot(lam, db))) <= 1e-8 * max(1.0, abs(fd))
    # su(3) direction on one link: U -> exp(tX) U
    G = adjoint.hopping_gradient(U, x, lam) + adjoint.clover_gradient(U, x, lam, c_sw)
    F = adjoint.su3_projection(U, G)
    assert np.allclose(F + np.conj(np.swapaxes(F, -1, -2)), 0, atol=1e-13)
    assert np.allclose(np.trace(F, axis1=-2, axis2=-1), 0, atol=1e-13)
    idx = (3, 1, 0, 1, 0)
    H = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    X = 0.5 * (H - H.conj().T)
    X -= np.trace(X) / 3 * np.eye(3)
    w, v = np.linalg.eigh(-1j * X)      # X = i v diag(w) v^dag
    def expX(t):
        return (v * np.exp(1j * t * w)) @ v.conj().T
    def L_t(t):
        Ut = U.copy()
        Ut[idx] = expX(t) @ U[idx]
        return _dense_loss(Ut, m0, c_sw, b, eta)
    fd = (L_t(h) - L_t(-h)) / (2 * h)
    assert abs(fd - np.real(np.trace(X @ F[idx]))) <= 1e-7 * max(1.0, abs(fd))


def test_gmres_gradients_match_dense():
    """The GMRES-based gradients (forward and adjoint solves) equal the dense ones."""
    dims = (4, 2, 2, 4)
    m0, c_sw = 0.3, 1.0
    U, b, eta = _setup(dims, 0.35, 61)
    x, lam, gb, G = adjoint.gradients(U, m0, c_sw, b, eta, tol=1e-13)
    xd, lamd = _dense_x_lam(U, m0, c_sw, b, eta)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert np.linalg.norm(gb - lamd) <= 1e-10 * np.linalg.norm(lamd)
    Gd = adjoint.hopping_gradient(U, xd, lamd) + adjoint.clover_gradient(U, xd, lamd, c_sw)
    assert np.linalg.norm(G - Gd) <= 1e-9 * np.linalg.norm(Gd)
