"""Wilson(-clover) Dirac operator, plain FP64 numpy (oracle; test infrastructure only).

Follows Sec. III-A-1 (the unnumbered definitions of D_W and D = D_W - C,
Algorithm 1's terms and the storage description) and Sec. III-A-2 (odd-even
preconditioning). Readings of points the paper leaves open:

* pi^{+-}_mu = (1 +- gamma_mu)/2 (projectors, so idempotent), lattice spacing 1.
* chiral gamma basis: gamma_mu = [[0, P_mu], [P_mu^dag, 0]] with P_t = 1 and
  P_k = i sigma_k; gamma5 = gamma_x gamma_y gamma_z gamma_t = diag(-1,-1,+1,+1).
  In this basis the clover term is block-diagonal with two Hermitian 6x6
  blocks (the paper's "42 complex" per site).
* directions mu = 0, 1, 2, 3 are t, z, y, x; time is antiperiodic for the
  fermion field (factor ``bc`` on a hop across t = T-1 <-> 0), space periodic.
* clover: C(x) = (c_sw/32) sum_{mu,nu} (gamma_mu gamma_nu) (x) (Q_mu,nu(x) - Q_nu,mu(x)),
  Q_mu,nu the sum of the four oriented plaquettes in the (mu, nu) plane that
  start and end at x; D = D_W - C.
* odd-even: even sites have (t+z+y+x) even; the Schur system lives on the odd
  sites, S = A_oo - D_oe A_ee^{-1} D_eo with A = (4 + m0) - C the site-diagonal
  part and D_eo / D_oe the hopping part restricted by parity.

Array shapes: gauge U [T, Z, Y, X, 4, 3, 3]; spinor block psi
[nrhs, T, Z, Y, X, 4, 3]; site matrices [T, Z, Y, X, 12, 12] with component
index 3*spin + colour; a half-lattice block [nrhs, V/2, 4, 3] lists the sites
of one parity in increasing site number.
"""
from __future__ import annotations

import numpy as np

_SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def _chiral(p: np.ndarray) -> np.ndarray:
    g = np.zeros((4, 4), dtype=np.complex128)
    g[0:2, 2:4] = p
    g[2:4, 0:2] = p.conj().T
    return g


def gamma_matrices() -> np.ndarray:
    """gamma_mu for mu = 0 (t), 1 (z), 2 (y), 3 (x); shape [4, 4, 4]."""
    g_t = _chiral(np.eye(2, dtype=np.complex128))
    g_x = _chiral(1j * _SIGMA[0])
    g_y = _chiral(1j * _SIGMA[1])
    g_z = _chiral(1j * _SIGMA[2])
    return np.stack([g_t, g_z, g_y, g_x])


def gamma5() -> np.ndarray:
    g = gamma_matrices()
    return g[3] @ g[2] @ g[1] @ g[0]


def _dag(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def _spin(p: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(p (x) 1_colour) psi for a 4x4 spin matrix p."""
    return np.einsum("st,...tc->...sc", p, psi)


def _colour(u: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(1_spin (x) u(x)) psi(x) for a site field of 3x3 matrices u [T, Z, Y, X, 3, 3]."""
    return np.einsum("tzyxab,ntzyxsb->ntzyxsa", u, psi)


def _psi_forward(psi: np.ndarray, mu: int, bc: float) -> np.ndarray:
    """psi(x + mu-hat), with the time boundary factor on the wrap t = T-1 -> 0."""
    out = np.roll(psi, -1, axis=1 + mu)
    if mu == 0 and bc != 1:
        out[:, -1] *= bc
    return out


def _psi_backward(psi: np.ndarray, mu: int, bc: float) -> np.ndarray:
    """psi(x - mu-hat), with the time boundary factor on the wrap t = 0 -> T-1."""
    out = np.roll(psi, +1, axis=1 + mu)
    if mu == 0 and bc != 1:
        out[:, 0] *= bc
    return out


def hopping_sum(U: np.ndarray, psi: np.ndarray, bc: float = -1.0) -> np.ndarray:
    """sum_mu [pi^-_mu (x) U_mu(x) psi(x+mu) + pi^+_mu (x) U_mu(x-mu)^dag psi(x-mu)] (Sec. III-A-1)."""
    g = gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    out = np.zeros_like(psi)
    for mu in range(4):
        pi_minus = (one - g[mu]) / 2
        pi_plus = (one + g[mu]) / 2
        u_here = U[..., mu, :, :]
        u_back_dag = _dag(np.roll(u_here, +1, axis=mu))
        out += _spin(pi_minus, _colour(u_here, _psi_forward(psi, mu, bc)))
        out += _spin(pi_plus, _colour(u_back_dag, _psi_backward(psi, mu, bc)))
    return out


def site_matrix_apply(M: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 12x12 matrix per site, M [T, Z, Y, X, 12, 12], to psi [n, T, Z, Y, X, 4, 3]."""
    flat = psi.reshape(psi.shape[:5] + (12,))
    out = np.einsum("tzyxij,ntzyxj->ntzyxi", M, flat)
    return out.reshape(psi.shape)


def plaquette_leaves(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Q_mu,nu(x): the four plaquettes in the (mu, nu) plane starting and ending at x."""
    def at(a, *steps):
        # a(x + sum of steps), steps given as (direction, +-1)
        for d, s in steps:
            a = np.roll(a, -s, axis=d)
        return a

    um = U[..., mu, :, :]
    un = U[..., nu, :, :]
    leaf1 = um @ at(un, (mu, 1)) @ _dag(at(um, (nu, 1))) @ _dag(un)
    leaf2 = un @ _dag(at(um, (mu, -1), (nu, 1))) @ _dag(at(un, (mu, -1))) @ at(um, (mu, -1))
    leaf3 = (_dag(at(um, (mu, -1))) @ _dag(at(un, (mu, -1), (nu, -1)))
             @ at(um, (mu, -1), (nu, -1)) @ at(un, (nu, -1)))
    leaf4 = _dag(at(un, (nu, -1))) @ at(um, (nu, -1)) @ at(un, (nu, -1), (mu, 1)) @ _dag(um)
    return leaf1 + leaf2 + leaf3 + leaf4


def clover_term(U: np.ndarray, c_sw: float) -> np.ndarray:
    """C(x) = (c_sw/32) sum_{mu,nu} gamma_mu gamma_nu (x) (Q_mu,nu - Q_nu,mu); [T, Z, Y, X, 12, 12]."""
    g = gamma_matrices()
    lat = U.shape[:4]
    C = np.zeros(lat + (12, 12), dtype=np.complex128)
    if c_sw == 0:
        return C
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            F = plaquette_leaves(U, mu, nu) - plaquette_leaves(U, nu, mu)
            gg = g[mu] @ g[nu]
            C += (c_sw / 32.0) * np.einsum("st,...ab->...satb", gg, F).reshape(lat + (12, 12))
    return C


def diag_blocks(U: np.ndarray, m0: float, c_sw: float):
    """Site-diagonal part A(x) = (4 + m0) 1 - C(x) and its inverse, each [T, Z, Y, X, 12, 12]."""
    C = clover_term(U, c_sw)
    A = (4.0 + m0) * np.eye(12, dtype=np.complex128) - C
    return A, np.linalg.inv(A)


def apply_D(U: np.ndarray, psi: np.ndarray, m0: float, C: np.ndarray | None = None,
            bc: float = -1.0) -> np.ndarray:
    """D psi = (4 + m0) psi - C psi - hopping (Sec. III-A-1, a = 1)."""
    out = (4.0 + m0) * psi - hopping_sum(U, psi, bc)
    if C is not None:
        out = out - site_matrix_apply(C, psi)
    return out


# ---------------------------------------------------------------- odd-even (Sec. III-A-2)

def parity_mask(dims) -> np.ndarray:
    t, z, y, x = np.indices(tuple(int(d) for d in dims))
    return (t + z + y + x) % 2


def split_parity(psi: np.ndarray, p: int) -> np.ndarray:
    """Sites of parity p of psi [n, T, Z, Y, X, 4, 3] -> [n, V/2, 4, 3], in site order."""
    mask = parity_mask(psi.shape[1:5]) == p
    return psi[:, mask]


def embed_parity(half: np.ndarray, p: int, dims) -> np.ndarray:
    """Inverse of split_parity: a full-lattice block that is zero off parity p."""
    dims = tuple(int(d) for d in dims)
    full = np.zeros((half.shape[0],) + dims + (4, 3), dtype=np.complex128)
    full[:, parity_mask(dims) == p] = half
    return full


def _hop_part(U, psi_full, bc):
    """The hopping part of D (everything but the site-diagonal term)."""
    return -hopping_sum(U, psi_full, bc)


def apply_D_eo(U, psi_o, bc=-1.0):
    """D_eo psi_o: hopping from odd sites, evaluated on even sites."""
    dims = U.shape[:4]
    return split_parity(_hop_part(U, embed_parity(psi_o, 1, dims), bc), 0)


def apply_D_oe(U, psi_e, bc=-1.0):
    """D_oe psi_e: hopping from even sites, evaluated on odd sites."""
    dims = U.shape[:4]
    return split_parity(_hop_part(U, embed_parity(psi_e, 0, dims), bc), 1)


def _apply_blocks_half(M, half, p):
    """Apply the per-site 12x12 blocks of parity p to a half-lattice block."""
    mask = parity_mask(M.shape[:4]) == p
    Mp = M[mask]                                  # [V/2, 12, 12]
    flat = half.reshape(half.shape[0], half.shape[1], 12)
    return np.einsum("vij,nvj->nvi", Mp, flat).reshape(half.shape)


def apply_Aee_inv(Ainv, psi_e):
    return _apply_blocks_half(Ainv, psi_e, 0)


def apply_Aoo(A, psi_o):
    return _apply_blocks_half(A, psi_o, 1)


def apply_schur(U, A, Ainv, psi_o, bc=-1.0):
    """S psi_o = A_oo psi_o - D_oe A_ee^{-1} D_eo psi_o."""
    t_e = apply_Aee_inv(Ainv, apply_D_eo(U, psi_o, bc))
    return apply_Aoo(A, psi_o) - apply_D_oe(U, t_e, bc)


def schur_prepare(U, Ainv, b_e, b_o, bc=-1.0):
    """hat b_o = b_o - D_oe A_ee^{-1} b_e."""
    return b_o - apply_D_oe(U, apply_Aee_inv(Ainv, b_e), bc)


def schur_reconstruct(U, Ainv, b_e, x_o, bc=-1.0):
    """x_e = A_ee^{-1} (b_e - D_eo x_o)."""
    return apply_Aee_inv(Ainv, b_e - apply_D_eo(U, x_o, bc))
