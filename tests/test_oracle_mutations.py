"""The oracle's pins have teeth: plausible mistakes planted in copies of the oracle's operator
functions (on the CPU, one at a time) each make at least one pin fail, while the unmodified
oracle passes them all.

Pins used (each independent of the code under test): the free-field plane-wave closed form
(U = 1, antiperiodic time), gamma5-hermiticity with the clover term, gauge covariance with the
clover term, the closed form of the clover term in a constant abelian field, and the dense
matrix built entry by entry with explicit loops (``oracle.dense_operator``).
"""
import numpy as np
import pytest

from oracle import dirac
from oracle.dense import dense_operator
import synthetic as syn

DIMS = (4, 2, 2, 4)


# ---------------------------------------------------------------- mutated copies of the oracle


def _hopping(mut):
    """sum_mu [pi^-_mu U_mu(x) psi(x+mu) + pi^+_mu U_mu(x-mu)^dag psi(x-mu)], with one planted mistake."""
    def hopping_sum(U, psi, bc=-1.0):
        if mut == "periodic_time":
            bc = 1.0
        g = dirac.gamma_matrices()
        one = np.eye(4, dtype=np.complex128)
        out = np.zeros_like(psi)
        for mu in range(4):
            pi_minus = (one - g[mu]) / 2
            pi_plus = (one + g[mu]) / 2
            if mut == "swapped_projectors":
                pi_minus, pi_plus = pi_plus, pi_minus
            u_here = U[..., mu, :, :]
            u_back = np.roll(u_here, +1, axis=mu)
            if mut == "back_link_at_x":
                u_back = u_here
            u_back_dag = u_back if mut == "back_link_no_dagger" else dirac._dag(u_back)
            u_fwd = np.swapaxes(u_here, -1, -2) if mut == "forward_link_transposed" else u_here
            fwd = dirac._psi_backward(psi, mu, bc) if mut == "forward_hop_backwards" else \
                dirac._psi_forward(psi, mu, bc)
            out += dirac._spin(pi_minus, dirac._colour(u_fwd, fwd))
            out += dirac._spin(pi_plus, dirac._colour(u_back_dag, dirac._psi_backward(psi, mu, bc)))
        return -out if mut == "hopping_sign" else out
    return hopping_sum


def _clover(mut):
    """C(x) = (c_sw/32) sum gamma_mu gamma_nu (x) (Q_mu,nu - Q_nu,mu), with one planted mistake."""
    def leaves(U, mu, nu):
        def at(a, *steps):
            for d, s in steps:
                a = np.roll(a, -s, axis=d)
            return a
        um, un, dag = U[..., mu, :, :], U[..., nu, :, :], dirac._dag
        leaf1 = um @ at(un, (mu, 1)) @ dag(at(um, (nu, 1))) @ dag(un)
        leaf2 = un @ dag(at(um, (mu, -1), (nu, 1))) @ dag(at(un, (mu, -1))) @ at(um, (mu, -1))
        if mut == "leaf_orientation":
            leaf2 = un @ at(um, (mu, -1), (nu, 1)) @ dag(at(un, (mu, -1))) @ at(um, (mu, -1))
        leaf3 = dag(at(um, (mu, -1))) @ dag(at(un, (mu, -1), (nu, -1))) @ at(um, (mu, -1), (nu, -1)) @ at(un, (nu, -1))
        leaf4 = dag(at(un, (nu, -1))) @ at(um, (nu, -1)) @ at(un, (nu, -1), (mu, 1)) @ dag(um)
        if mut == "three_leaves":
            return leaf1 + leaf2 + leaf3
        return leaf1 + leaf2 + leaf3 + leaf4

    def clover_term(U, c_sw):
        g = dirac.gamma_matrices()
        lat = U.shape[:4]
        C = np.zeros(lat + (12, 12), dtype=np.complex128)
        if c_sw == 0:
            return C
        norm = 16.0 if mut == "clover_norm" else 32.0
        for mu in range(4):
            for nu in range(4):
                if mu == nu:
                    continue
                F = leaves(U, mu, nu) + (1 if mut == "clover_plus" else -1) * leaves(U, nu, mu)
                C += (c_sw / norm) * np.einsum("st,...ab->...satb", g[mu] @ g[nu], F).reshape(lat + (12, 12))
        return C
    return clover_term


# ---------------------------------------------------------------- the pins


def _pin_free_field():
    U = syn.unit_gauge(DIMS)
    g = dirac.gamma_matrices()
    m0 = 0.1
    u = np.arange(12) + 1j * np.arange(12)[::-1]
    for n in [(0, 0, 0, 0), (1, 1, 0, 1)]:
        p = np.array([np.pi * (2 * n[0] + 1) / DIMS[0]] + [2 * np.pi * n[k] / DIMS[k] for k in (1, 2, 3)])
        t, z, y, x = np.indices(DIMS)
        phase = np.exp(1j * (p[0] * t + p[1] * z + p[2] * y + p[3] * x))
        Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4, dtype=complex)
        for mu in range(4):
            Dp = Dp + 1j * np.sin(p[mu]) * g[mu]
        psi = (phase[..., None] * u).reshape(DIMS + (4, 3))[None]
        expect = (phase[..., None] * (np.kron(Dp, np.eye(3)) @ u)).reshape(DIMS + (4, 3))[None]
        if np.max(np.abs(dirac.apply_D(U, psi, m0) - expect)) > 1e-12:
            return False
    return True


def _pin_gamma5_hermiticity():
    U = syn.gauge_field(DIMS, "exp", 0.4, seed=11)
    C = dirac.clover_term(U, 1.0)
    phi = syn.gaussian_spinors(DIMS, 1, 12)
    psi = syn.gaussian_spinors(DIMS, 1, 13)
    g5 = dirac.gamma5()

    def g5v(v):
        return np.einsum("st,...tc->...sc", g5, v)
    lhs = np.vdot(phi, dirac.apply_D(U, psi, -0.2, C))
    rhs = np.vdot(g5v(dirac.apply_D(U, g5v(phi), -0.2, C)), psi)
    return abs(lhs - rhs) < 1e-12 * abs(lhs)


def _pin_gauge_covariance():
    U = syn.gauge_field(DIMS, "exp", 0.5, seed=21)
    g = syn.random_gauge_transform(DIMS, 22)
    psi = syn.gaussian_spinors(DIMS, 1, 23)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ dirac._dag(np.roll(g, -1, axis=mu))

    def gmul(v):
        return np.einsum("tzyxab,ntzyxsb->ntzyxsa", g, v)
    lhs = dirac.apply_D(Ug, gmul(psi), 0.05, dirac.clover_term(Ug, 1.0))
    rhs = gmul(dirac.apply_D(U, psi, 0.05, dirac.clover_term(U, 1.0)))
    return np.max(np.abs(lhs - rhs)) < 1e-12


def _pin_abelian_clover():
    dims = (2, 2, 4, 6)
    B = 2 * np.pi / dims[3]
    U = syn.unit_gauge(dims).copy()
    x3 = np.indices(dims)[3]
    U[..., 2, 0, 0] = np.exp(1j * B * x3)
    U[..., 2, 1, 1] = np.exp(-1j * B * x3)
    g = dirac.gamma_matrices()
    expect = (1.7 / 2) * 1j * np.sin(B) * np.kron(g[3] @ g[2], np.diag([1, -1, 0]))
    return np.max(np.abs(dirac.clover_term(U, 1.7) - expect)) < 1e-13


def _pin_dense():
    U = syn.gauge_field(DIMS, "exp", 0.7, seed=41)
    C = dirac.clover_term(U, 1.0)
    D = dense_operator(U, -0.3, C)
    psi = syn.gaussian_spinors(DIMS, 1, 42)
    out = dirac.apply_D(U, psi, -0.3, C)
    return np.max(np.abs(out.reshape(-1) - D @ psi.reshape(-1))) < 1e-12


PINS = {"free_field": _pin_free_field, "gamma5_hermiticity": _pin_gamma5_hermiticity,
        "gauge_covariance": _pin_gauge_covariance, "abelian_clover": _pin_abelian_clover, "dense": _pin_dense}


def _failing_pins():
    return [name for name, pin in PINS.items() if not pin()]


def test_unmodified_oracle_passes_every_pin():
    assert _failing_pins() == []


@pytest.mark.parametrize("mut", ["periodic_time", "swapped_projectors", "back_link_at_x", "back_link_no_dagger",
                                 "forward_link_transposed", "forward_hop_backwards", "hopping_sign"])
def test_planted_hopping_mistake_is_caught(monkeypatch, mut):
    monkeypatch.setattr(dirac, "hopping_sum", _hopping(mut))
    assert _failing_pins(), f"no pin catches {mut}"


@pytest.mark.parametrize("mut", ["clover_norm", "clover_plus", "leaf_orientation", "three_leaves"])
def test_planted_clover_mistake_is_caught(monkeypatch, mut):
    monkeypatch.setattr(dirac, "clover_term", _clover(mut))
    assert _failing_pins(), f"no pin catches {mut}"


def test_mutation_copies_reproduce_the_oracle_without_a_mistake(monkeypatch):
    """The copies above differ from the oracle only by the planted mistake."""
    monkeypatch.setattr(dirac, "hopping_sum", _hopping("none"))
    monkeypatch.setattr(dirac, "clover_term", _clover("none"))
    assert _failing_pins() == []
