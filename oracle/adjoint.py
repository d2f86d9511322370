"""Adjoint of the batched solve, plain FP64 numpy (oracle; test infrastructure only).

The paper has no adjoint; this is the task's differentiable-solve extension. For
x_i = D^{-1} b_i and a loss L = sum_i Re <eta_i, x_i> (<a, b> = a^H b):

* dL/db_i = lambda_i = D^{-dagger} eta_i, one solve with the adjoint operator.
* dL = -Re <lambda, (dD) x>, so the gradient with respect to the gauge links
  comes from the derivative of D (Sec. III-A-1 definitions) in each link:
  the hopping terms pi^- U_mu(x) psi(x+mu) and pi^+ U_mu(x-mu)^dag psi(x-mu),
  and the clover term through the plaquette leaves of Q_mu,nu.

Gradient convention (the one PyTorch uses for complex tensors and a real loss):
a complex array G with dL = Re sum conj(G) * dU for every perturbation dU of the
link entries, treated as independent complex numbers. The su(3) projection
F = TA(U G^dag) (TA = traceless anti-Hermitian part) gives the derivative along
U -> exp(t X) U for X in su(3): dL/dt = Re tr(X F).

Shapes as in ``dirac``: U [T, Z, Y, X, 4, 3, 3]; spinor blocks [n, T, Z, Y, X, 4, 3].
"""
from __future__ import annotations

import numpy as np

from . import dirac
from . import krylov


def hopping_sum_dagger(U: np.ndarray, psi: np.ndarray, bc: float = -1.0) -> np.ndarray:
    """Adjoint of ``dirac.hopping_sum``: the adjoint of pi^- U_mu(x) psi(x+mu) is
    pi^- U_mu(y-mu)^dag phi(y-mu), that of pi^+ U_mu(x-mu)^dag psi(x-mu) is
    pi^+ U_mu(y) phi(y+mu) (the projectors are Hermitian, the boundary factor real)."""
    g = dirac.gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    out = np.zeros_like(psi)
    for mu in range(4):
        pi_minus = (one - g[mu]) / 2
        pi_plus = (one + g[mu]) / 2
        u_here = U[..., mu, :, :]
        u_back_dag = dirac._dag(np.roll(u_here, +1, axis=mu))
        out += dirac._spin(pi_minus, dirac._colour(u_back_dag, dirac._psi_backward(psi, mu, bc)))
        out += dirac._spin(pi_plus, dirac._colour(u_here, dirac._psi_forward(psi, mu, bc)))
    return out


def apply_D_dagger(U: np.ndarray, psi: np.ndarray, m0: float, C: np.ndarray | None = None,
                   bc: float = -1.0) -> np.ndarray:
    """D^dagger psi = (4 + m0) psi - C psi - H^dagger psi (C(x) is Hermitian)."""
    out = (4.0 + m0) * psi - hopping_sum_dagger(U, psi, bc)
    if C is not None:
        out = out - dirac.site_matrix_apply(C, psi)
    return out


def solve_dagger(U, C, m0, eta_block, tol, m=30, max_restarts=400, bc=-1.0):
    """GMRES on D^dagger lambda = eta for each rhs (the adjoint solve)."""
    out = []
    for k in range(eta_block.shape[0]):
        shape = eta_block[k:k + 1].shape

        def A(v, shape=shape):
            return apply_D_dagger(U, v.reshape(shape), m0, C, bc).ravel()

        lam, info = krylov.gmres(A, eta_block[k].ravel(), tol, m, max_restarts)
        if not info["converged"]:
            raise RuntimeError(f"adjoint solve of rhs {k} did not converge: {info}")
        out.append(lam.reshape(eta_block.shape[1:]))
    return np.stack(out)


def loss(x: np.ndarray, eta: np.ndarray) -> float:
    """L = sum_i Re <eta_i, x_i>."""
    return float(np.real(np.vdot(eta.ravel(), x.ravel())))


def _link_bc(dims, bc: float) -> np.ndarray:
    """Factor [T, Z, Y, X, 4] multiplying U_mu(y) in the hopping terms: bc on the time links
    of the last time slice (the hop across t = T-1 <-> 0), 1 elsewhere."""
    f = np.ones(tuple(dims) + (4,))
    f[-1, :, :, :, 0] = bc
    return f


def hopping_gradient(U: np.ndarray, x: np.ndarray, lam: np.ndarray, bc: float = -1.0) -> np.ndarray:
    """dL/dU from the hopping terms of D (summed over rhs); G [T, Z, Y, X, 4, 3, 3].

    D x contains -pi^- (b U_mu(y)) x(y+mu) at y and -pi^+ (b U_mu(y))^dag x(y) at y+mu, with
    b the link's boundary factor, and dL = -Re <lambda, (dD) x>:
      from the first term  dL = Re sum_ab b dU_ab M_ab,   M_ab = sum_s conj(lam_sa(y)) (pi^- x(y+mu))_sb
      from the second      dL = Re sum_ab b conj(dU_ba) N_ab, N_ab = sum_s conj(lam_sa(y+mu)) (pi^+ x(y))_sb
    so G_mu(y) = b (conj(M) + N^T)."""
    g = dirac.gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    dims = U.shape[:4]
    G = np.zeros(U.shape, dtype=np.complex128)
    for mu in range(4):
        pi_minus = (one - g[mu]) / 2
        pi_plus = (one + g[mu]) / 2
        # neighbours without the boundary factor (it is carried by b)
        x_fwd = np.roll(x, -1, axis=1 + mu)
        lam_fwd = np.roll(lam, -1, axis=1 + mu)
        px = dirac._spin(pi_minus, x_fwd)
        M = np.einsum("ntzyxsa,ntzyxsb->tzyxab", np.conj(lam), px)
        qx = dirac._spin(pi_plus, x)
        N = np.einsum("ntzyxsa,ntzyxsb->tzyxab", np.conj(lam_fwd), qx)
        G[..., mu, :, :] = np.conj(M) + np.swapaxes(N, -1, -2)
    return G * _link_bc(dims, bc)[..., None, None]


# The four leaves of Q_mu,nu(x) (the oracle's ``dirac.plaquette_leaves``) as link factors:
# (direction: "mu" or "nu", site offset {"mu": +-1, "nu": +-1}, daggered).
_LEAVES = (
    (("mu", {}, False), ("nu", {"mu": 1}, False), ("mu", {"nu": 1}, True), ("nu", {}, True)),
    (("nu", {}, False), ("mu", {"mu": -1, "nu": 1}, True), ("nu", {"mu": -1}, True), ("mu", {"mu": -1}, False)),
    (("mu", {"mu": -1}, True), ("nu", {"mu": -1, "nu": -1}, True), ("mu", {"mu": -1, "nu": -1}, False),
     ("nu", {"nu": -1}, False)),
    (("nu", {"nu": -1}, True), ("mu", {"nu": -1}, False), ("nu", {"nu": -1, "mu": 1}, False), ("mu", {}, True)),
)


def _shifted(a: np.ndarray, offset: dict, mu: int, nu: int) -> np.ndarray:
    """a(x + offset) for a site field a [T, Z, Y, X, ...]."""
    for name, s in offset.items():
        a = np.roll(a, -s, axis=mu if name == "mu" else nu)
    return a


def _factor(U, f, mu, nu):
    name, off, dag = f
    u = _shifted(U[..., mu if name == "mu" else nu, :, :], off, mu, nu)
    return dirac._dag(u) if dag else u


def clover_gradient(U: np.ndarray, x: np.ndarray, lam: np.ndarray, c_sw: float) -> np.ndarray:
    """dL/dU from the clover term (summed over rhs); G [T, Z, Y, X, 4, 3, 3].

    D = ... - C with C(x) = (c_sw/32) sum_{mu != nu} gamma_mu gamma_nu (x) (Q_mu,nu - Q_nu,mu), so
    dL = -Re <lambda, (dD) x> = Re sum_x lambda(x)^H dC(x) x(x)
       = (c_sw/32) Re sum_x sum_{mu != nu} tr[(dQ_mu,nu(x) - dQ_nu,mu(x)) W_mu,nu(x)],
    W_mu,nu(x) = sum_i sum_s (gamma_mu gamma_nu x_i(x))_s lambda_i(x)_s^H (a colour matrix).
    For a leaf A F B with the factor F = U_rho(y) (or its adjoint) the term tr(A dF B W) = tr(dF K),
    K = B W A, gives G_rho(y) += K^dag (or K)."""
    G = np.zeros(U.shape, dtype=np.complex128)
    if c_sw == 0:
        return G
    g = dirac.gamma_matrices()
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            gx = dirac._spin(g[mu] @ g[nu], x)
            W = (c_sw / 32.0) * np.einsum("ntzyxsb,ntzyxsa->tzyxba", gx, np.conj(lam))
            for (m1, n1, weight) in ((mu, nu, 1.0), (nu, mu, -1.0)):   # Q_mu,nu and -Q_nu,mu
                for leaf in _LEAVES:
                    fac = [_factor(U, f, m1, n1) for f in leaf]
                    for p, f in enumerate(leaf):
                        eye = np.broadcast_to(np.eye(3, dtype=np.complex128), W.shape)
                        A = eye
                        for q in range(p):
                            A = A @ fac[q]
                        B = eye
                        for q in range(p + 1, 4):
                            B = B @ fac[q]
                        K = weight * (B @ W @ A)
                        name, off, dag = f
                        rho = m1 if name == "mu" else n1
                        # the factor sits at y = x + off: move K from x to y
                        Ky = K
                        for nm, s in off.items():
                            Ky = np.roll(Ky, s, axis=m1 if nm == "mu" else n1)
                        G[..., rho, :, :] += Ky if dag else dirac._dag(Ky)
    return G


def gradients(U, m0, c_sw, b, eta, tol=1e-13, m=40, max_restarts=400, bc=-1.0):
    """(x, lambda, dL/db, dL/dU) for L = sum_i Re <eta_i, D^{-1} b_i>, by FP64 GMRES solves."""
    C = dirac.clover_term(U, c_sw) if c_sw else None
    x, infos = krylov.solve_full(U, C, m0, b, tol, m, max_restarts, bc)
    if not all(i["converged"] for i in infos):
        raise RuntimeError("forward solve did not converge")
    lam = solve_dagger(U, C, m0, eta, tol, m, max_restarts, bc)
    G = hopping_gradient(U, x, lam, bc) + clover_gradient(U, x, lam, c_sw)
    return x, lam, lam.copy(), G


def su3_projection(U: np.ndarray, G: np.ndarray) -> np.ndarray:
    """F = TA(U G^dag), the traceless anti-Hermitian part: for U -> exp(t X) U, X in su(3),
    dL/dt = Re tr(X F)."""
    A = U @ dirac._dag(G)
    ah = 0.5 * (A - dirac._dag(A))
    tr = np.trace(ah, axis1=-2, axis2=-1)[..., None, None]
    return ah - tr / 3.0 * np.eye(3)
