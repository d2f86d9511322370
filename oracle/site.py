"""The operators evaluated at single sites, plain FP64 numpy (oracle; test infrastructure only).

On lattices too large for the whole-lattice oracle to finish in a test (the
32^3 x 64 workload, 2.1 M sites), outputs are checked at sampled sites. These
functions compute one output site from the definitions of Sec. III-A-1 and the
odd-even split of Sec. III-A-2, written out term by term with explicit site
coordinates (no lattice-wide array operations), with the same readings as
``oracle.dirac``: pi^{+-}_mu = (1 +- gamma_mu)/2 in the chiral basis, mu = 0..3
= t, z, y, x, the fermion boundary factor ``bc`` on a hop across t = T-1 <-> 0,
C(x) = (c_sw/32) sum_{mu,nu} gamma_mu gamma_nu (x) (Q_mu,nu(x) - Q_nu,mu(x)) with
Q the four plaquette leaves at x, A(x) = (4 + m0) - C(x), D = A - hopping.

Inputs: U [T, Z, Y, X, 4, 3, 3]; a full-lattice spinor psi [T, Z, Y, X, 4, 3]
(one rhs) or a half-lattice odd-site block psi_o [V/2, 4, 3] listing the odd
sites in increasing site number.
"""
from __future__ import annotations

import numpy as np

from .dirac import gamma_matrices


def _dag(m):
    return np.conj(m.T)


def _shift(dims, x, mu, step):
    """Coordinates of x + step * mu-hat (periodic) and the fermion boundary crossing flag."""
    y = list(x)
    y[mu] = (x[mu] + step) % dims[mu]
    crossed = mu == 0 and ((step > 0 and x[0] == dims[0] - 1) or (step < 0 and x[0] == 0))
    return tuple(y), crossed


def _link(U, x, mu):
    return U[x[0], x[1], x[2], x[3], mu]


def leaves_at(U, x, mu, nu):
    """Q_mu,nu(x): the four oriented plaquettes in the (mu, nu) plane starting and ending at x."""
    dims = U.shape[:4]

    def at(*steps):
        y = tuple(x)
        for d, s in steps:
            y, _ = _shift(dims, y, d, s)
        return y

    um = lambda y: _link(U, y, mu)  # noqa: E731
    un = lambda y: _link(U, y, nu)  # noqa: E731
    q = um(x) @ un(at((mu, 1))) @ _dag(um(at((nu, 1)))) @ _dag(un(x))
    q = q + un(x) @ _dag(um(at((mu, -1), (nu, 1)))) @ _dag(un(at((mu, -1)))) @ um(at((mu, -1)))
    q = q + (_dag(um(at((mu, -1)))) @ _dag(un(at((mu, -1), (nu, -1))))
             @ um(at((mu, -1), (nu, -1))) @ un(at((nu, -1))))
    q = q + _dag(un(at((nu, -1)))) @ um(at((nu, -1))) @ un(at((nu, -1), (mu, 1))) @ _dag(um(x))
    return q


def site_block(U, x, m0, c_sw):
    """A(x) = (4 + m0) 1 - C(x) as a 12x12 matrix (component index 3*spin + colour)."""
    g = gamma_matrices()
    A = (4.0 + m0) * np.eye(12, dtype=np.complex128)
    if c_sw == 0:
        return A
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            F = leaves_at(U, x, mu, nu) - leaves_at(U, x, nu, mu)
            A -= (c_sw / 32.0) * np.kron(g[mu] @ g[nu], F)
    return A


def hopping_at(U, field, x, bc=-1.0):
    """sum_mu [pi^-_mu U_mu(x) f(x+mu) + pi^+_mu U_mu(x-mu)^dag f(x-mu)] at site x; field(y) -> [4, 3]."""
    dims = U.shape[:4]
    g = gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    out = np.zeros((4, 3), dtype=np.complex128)
    for mu in range(4):
        yf, cf = _shift(dims, x, mu, +1)
        yb, cb = _shift(dims, x, mu, -1)
        fwd = field(yf) * (bc if cf else 1.0)
        bwd = field(yb) * (bc if cb else 1.0)
        out += ((one - g[mu]) / 2) @ (fwd @ _link(U, x, mu).T)
        out += ((one + g[mu]) / 2) @ (bwd @ np.conj(_link(U, yb, mu)))
    return out


def apply_D_at(U, psi, x, m0, c_sw, bc=-1.0):
    """(D psi)(x) for a full-lattice spinor psi [T, Z, Y, X, 4, 3]; returns [4, 3]."""
    A = site_block(U, x, m0, c_sw)
    field = lambda y: psi[y]  # noqa: E731
    return (A @ psi[x].reshape(12)).reshape(4, 3) - hopping_at(U, field, x, bc)


def half_index(dims, x):
    """Position of site x in a half-lattice block of its parity (sites in increasing site number)."""
    T, Z, Y, X = dims
    lex = ((x[0] * Z + x[1]) * Y + x[2]) * X + x[3]
    return lex // 2


def apply_schur_at(U, psi_o, x, m0, c_sw, bc=-1.0):
    """(S psi_o)(x) = A(x) psi_o(x) - (D_oe A_ee^{-1} D_eo psi_o)(x) at an odd site x; returns [4, 3]."""
    dims = U.shape[:4]
    assert sum(x) % 2 == 1, "the Schur system lives on the odd sites"

    def odd(y):
        return psi_o[half_index(dims, y)]

    def t_even(y):
        # t(y) = A(y)^{-1} (D_eo psi_o)(y), (D_eo psi_o)(y) = -hopping of the odd field at even y
        d = -hopping_at(U, odd, y, bc)
        return np.linalg.solve(site_block(U, y, m0, c_sw), d.reshape(12)).reshape(4, 3)

    A = site_block(U, x, m0, c_sw)
    return (A @ odd(x).reshape(12)).reshape(4, 3) + hopping_at(U, t_even, x, bc)
