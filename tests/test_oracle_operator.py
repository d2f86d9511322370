"""Pins of the oracle's Dirac operator against facts fixed by the paper and by the mathematics.

Each test states what it pins and which plausible mistake it catches. None
compares the oracle with itself: closed forms, invariants with an independent
transform, and a brute-force dense matrix built with explicit loops.
"""
import numpy as np
import pytest

import oracle
from oracle import dirac
import synthetic as syn


def _rand_field(dims, seed, kind="exp", eps=0.3):
    return syn.gauge_field(dims, kind=kind, eps=eps, seed=seed)


# ------------------------------------------------------------------ gamma basis

def test_clifford_algebra_and_gamma5():
    """{gamma_mu, gamma_nu} = 2 delta, Hermitian; gamma5 diagonal (chiral basis)."""
    g = oracle.gamma_matrices()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))
    g5 = oracle.gamma5()
    assert np.allclose(g5, np.diag([-1, -1, 1, 1]))
    for mu in range(4):
        assert np.allclose(g5 @ g[mu], -g[mu] @ g5)
    one = np.eye(4)
    for mu in range(4):
        pm, pp = (one - g[mu]) / 2, (one + g[mu]) / 2
        assert np.allclose(pm @ pm, pm) and np.allclose(pp @ pp, pp)
        assert np.allclose(pm @ pp, 0)
        assert np.linalg.matrix_rank(pm) == 2          # 6 of 12 components survive


# ------------------------------------------------------------------ free field

def _plane_wave(dims, n, u):
    """psi(x) = exp(i p.x) u with p_t antiperiodic, p_space periodic; u a 12-vector."""
    T = dims[0]
    p = np.array([np.pi * (2 * n[0] + 1) / T] + [2 * np.pi * n[k] / dims[k] for k in (1, 2, 3)])
    t, z, y, x = np.indices(dims)
    phase = np.exp(1j * (p[0] * t + p[1] * z + p[2] * y + p[3] * x))
    return p, (phase[..., None] * u[None, None, None, None, :]).reshape(dims + (4, 3))[None]


def _symbol(p, m0):
    """D(p) = m0 + sum(1 - cos p) + i sum gamma_mu sin p_mu, times 1_colour."""
    g = oracle.gamma_matrices()
    Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4, dtype=complex)
    for mu in range(4):
        Dp = Dp + 1j * np.sin(p[mu]) * g[mu]
    return np.kron(Dp, np.eye(3))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 2, 4, 6)])
def test_free_field_plane_wave(dims):
    """U = 1: D e^{ipx} u = e^{ipx} D(p) u (pins projector signs, hop directions, BC)."""
    U = syn.unit_gauge(dims)
    rng = np.random.default_rng(5)
    m0 = 0.1
    for n in [(0, 0, 0, 0), (1, 1, 0, 1), (dims[0] // 2 - 1, 1, 1, 2)]:
        u = rng.standard_normal(12) + 1j * rng.standard_normal(12)
        p, psi = _plane_wave(dims, n, u)
        out = oracle.apply_D(U, psi, m0)
        expect = _plane_wave(dims, n, _symbol(p, m0) @ u)[1]
        assert np.max(np.abs(out - expect)) < 1e-13


def test_free_field_plane_wave_16x32():
    """Same closed form on the 16^3 x 32 lattice of the operator sweep."""
    dims = (32, 16, 16, 16)
    U = syn.unit_gauge(dims)
    u = np.arange(12) + 1j * np.arange(12)[::-1]
    p, psi = _plane_wave(dims, (3, 1, 2, 5), u)
    out = oracle.apply_D(U, psi, -0.2)
    expect = _plane_wave(dims, (3, 1, 2, 5), _symbol(p, -0.2) @ u)[1]
    assert np.max(np.abs(out - expect)) < 1e-12


def test_free_field_spectrum_dense():
    """Dense D at U = 1 on 2^4: eigenvalues m0 + sum(1-cos p) +- i sqrt(sum sin^2 p), 6-fold each."""
    dims = (2, 2, 2, 2)
    m0 = 0.3
    D = oracle.dense_operator(syn.unit_gauge(dims), m0)
    ev = np.sort_complex(np.round(np.linalg.eigvals(D), 10))
    expect = []
    for nt in range(2):
        for nz in range(2):
            for ny in range(2):
                for nx in range(2):
                    p = np.array([np.pi * (2 * nt + 1) / 2, np.pi * nz, np.pi * ny, np.pi * nx])
                    re = m0 + np.sum(1 - np.cos(p))
                    im = np.sqrt(np.sum(np.sin(p) ** 2))
                    expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    expect = np.sort_complex(np.round(np.array(expect), 10))
    assert np.max(np.abs(ev - expect)) < 1e-9


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("c_sw", [0.0, 1.0])
def test_gamma5_hermiticity(c_sw):
    """<phi, D psi> = <gamma5 D gamma5 phi, psi> (pins U vs U^dag and the clover Hermiticity)."""
    dims = (4, 4, 4, 4)
    U = _rand_field(dims, 11)
    C = oracle.clover_term(U, c_sw)
    phi = syn.gaussian_spinors(dims, 1, 12)
    psi = syn.gaussian_spinors(dims, 1, 13)
    g5 = oracle.gamma5()

    def g5v(v):
        return np.einsum("st,...tc->...sc", g5, v)

    lhs = np.vdot(phi, oracle.apply_D(U, psi, -0.2, C))
    rhs = np.vdot(g5v(oracle.apply_D(U, g5v(phi), -0.2, C)), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _gauge_transform(U, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x + mu)^dag."""
    Ug = np.empty_like(U)
    for mu in range(4):
        g_next = np.roll(g, -1, axis=mu)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_next, -1, -2))
    return Ug


def test_gauge_covariance_with_clover():
    """D[U^g](g psi) = g D[U] psi (pins link placement x vs x-mu and the leaf products)."""
    dims = (4, 4, 4, 4)
    U = _rand_field(dims, 21, eps=0.5)
    g = syn.random_gauge_transform(dims, 22)
    psi = syn.gaussian_spinors(dims, 2, 23)
    Ug = _gauge_transform(U, g)

    def gmul(v):
        return np.einsum("tzyxab,ntzyxsb->ntzyxsa", g, v)

    lhs = oracle.apply_D(Ug, gmul(psi), 0.05, oracle.clover_term(Ug, 1.0))
    rhs = gmul(oracle.apply_D(U, psi, 0.05, oracle.clover_term(U, 1.0)))
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_clover_hermitian_chiral_blocks_and_free():
    """C Hermitian, commutes with gamma5 (two 6x6 blocks, 42 complex per site), C = 0 at U = 1."""
    dims = (4, 4, 4, 4)
    C = oracle.clover_term(_rand_field(dims, 31, eps=0.6), 1.3)
    assert np.max(np.abs(C - np.conj(np.swapaxes(C, -1, -2)))) < 1e-14
    G5 = np.kron(oracle.gamma5(), np.eye(3))
    assert np.max(np.abs(C @ G5 - G5 @ C)) < 1e-14
    assert np.max(np.abs(C[..., 0:6, 6:12])) < 1e-14
    assert np.max(np.abs(C)) > 0.1
    assert np.max(np.abs(oracle.clover_term(syn.unit_gauge(dims), 1.0))) == 0.0


def test_clover_abelian_closed_form():
    """Constant abelian field in the (x, y) plane: C has a closed form.

    U_y(x) = diag(e^{iB x3}, e^{-iB x3}, 1), every other link 1, B = 2 pi / X.
    Every plaquette in the (x, y) plane is diag(e^{iB}, e^{-iB}, 1), so
    Q_xy = 4 diag(e^{iB}, e^{-iB}, 1), Q_yx = Q_xy^dag and
    C = (c_sw/32)[g_x g_y (Q_xy - Q_yx) + g_y g_x (Q_yx - Q_xy)]
      = (c_sw/2) i sin(B) g_x g_y (x) diag(1, -1, 0).
    Also D's diagonal block is (4 + m0) - C (the sign of D = D_W - C).
    Catches a swapped leaf orientation, a wrong 1/32 and a wrong sign of C.
    """
    dims = (2, 2, 4, 6)
    X = dims[3]
    B = 2 * np.pi / X
    U = syn.unit_gauge(dims).copy()
    x3 = np.indices(dims)[3]
    U[..., 2, 0, 0] = np.exp(1j * B * x3)
    U[..., 2, 1, 1] = np.exp(-1j * B * x3)
    c_sw = 1.7
    g = oracle.gamma_matrices()
    expect = (c_sw / 2) * 1j * np.sin(B) * np.kron(g[3] @ g[2], np.diag([1, -1, 0]))
    C = oracle.clover_term(U, c_sw)
    assert np.max(np.abs(C - expect)) < 1e-13
    m0 = -0.1
    D = oracle.dense_operator(U, m0, C)
    blk = D[0:12, 0:12]
    assert np.max(np.abs(blk - ((4 + m0) * np.eye(12) - expect))) < 1e-13


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_dense_brute_force_matches_apply(dims):
    """apply_D equals the dense matrix built entry by entry (2^4: both hops on one site add)."""
    U = _rand_field(dims, 41, eps=0.7)
    C = oracle.clover_term(U, 1.0)
    D = oracle.dense_operator(U, -0.3, C)
    psi = syn.gaussian_spinors(dims, 3, 42)
    out = oracle.apply_D(U, psi, -0.3, C)
    ref = (D @ psi.reshape(3, -1).T).T.reshape(psi.shape)
    assert np.max(np.abs(out - ref)) < 1e-13


def test_dense_schur_complement_and_determinant():
    """S = D_oo - D_oe D_ee^{-1} D_eo from dense blocks; det D = det D_ee det S on 2^4."""
    dims = (2, 2, 2, 2)
    U = _rand_field(dims, 51, eps=0.8)
    m0, c_sw = 0.2, 1.0
    A, Ainv = oracle.diag_blocks(U, m0, c_sw)
    C = oracle.clover_term(U, c_sw)
    D = oracle.dense_operator(U, m0, C)
    par = oracle.parity_mask(dims).ravel()
    idx_e = np.concatenate([np.arange(12 * s, 12 * s + 12) for s in np.where(par == 0)[0]])
    idx_o = np.concatenate([np.arange(12 * s, 12 * s + 12) for s in np.where(par == 1)[0]])
    Dee, Deo = D[np.ix_(idx_e, idx_e)], D[np.ix_(idx_e, idx_o)]
    Doe, Doo = D[np.ix_(idx_o, idx_e)], D[np.ix_(idx_o, idx_o)]
    S_dense = Doo - Doe @ np.linalg.solve(Dee, Deo)
    psi_o = syn.gaussian_spinors((1, 1, 1, 8), 2, 52).reshape(2, 8, 4, 3)
    out = oracle.apply_schur(U, A, Ainv, psi_o)
    ref = (S_dense @ psi_o.reshape(2, -1).T).T.reshape(psi_o.shape)
    assert np.max(np.abs(out - ref)) < 1e-12
    lhs = np.linalg.slogdet(D)
    r1, r2 = np.linalg.slogdet(Dee), np.linalg.slogdet(S_dense)
    assert abs(lhs[1] - (r1[1] + r2[1])) < 1e-10
    assert abs(lhs[0] - r1[0] * r2[0]) < 1e-10


def test_schur_prepare_reconstruct_identity():
    """With x_e reconstructed, ||b - D x|| equals ||hat b_o - S x_o|| for any x_o."""
    dims = (4, 4, 2, 2)
    U = _rand_field(dims, 61, eps=0.4)
    m0, c_sw = 0.1, 1.0
    A, Ainv = oracle.diag_blocks(U, m0, c_sw)
    C = oracle.clover_term(U, c_sw)
    b = syn.gaussian_spinors(dims, 2, 62)
    b_e, b_o = oracle.split_parity(b, 0), oracle.split_parity(b, 1)
    x_o = oracle.split_parity(syn.gaussian_spinors(dims, 2, 63), 1)
    x_e = oracle.schur_reconstruct(U, Ainv, b_e, x_o)
    x = oracle.embed_parity(x_e, 0, dims) + oracle.embed_parity(x_o, 1, dims)
    r_full = b - oracle.apply_D(U, x, m0, C)
    assert np.max(np.abs(oracle.split_parity(r_full, 0))) < 1e-12
    bhat = oracle.schur_prepare(U, Ainv, b_e, b_o)
    r_schur = bhat - oracle.apply_schur(U, A, Ainv, x_o)
    assert np.max(np.abs(oracle.split_parity(r_full, 1) - r_schur)) < 1e-12


def test_clover_inverse_blocks():
    """A A^{-1} = 1 per site and A^{-1} keeps the chiral block structure."""
    U = _rand_field((4, 2, 2, 2), 71, eps=0.5)
    A, Ainv = oracle.diag_blocks(U, -0.2, 1.0)
    assert np.max(np.abs(A @ Ainv - np.eye(12))) < 1e-13
    assert np.max(np.abs(Ainv[..., 0:6, 6:12])) < 1e-15
