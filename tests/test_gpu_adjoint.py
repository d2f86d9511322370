"""GPU adjoint (dagger solve, force kernel, autograd solve) checked against the FP64 oracle
and against central finite differences of the loss L = sum_i Re <eta_i, D^{-1} b_i>."""
import numpy as np
import pytest

import oracle
from oracle import adjoint
import synthetic as syn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_05816_gb300 as lq  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2601_05816_gb300 import _build
    _build.build()
    lq.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("op", [lq.OP_FULL, lq.OP_SCHUR])
@pytest.mark.parametrize("precision", [lq.C128, lq.C64])
def test_dagger_solve(op, precision):
    """D^dagger x = b solved through gamma5 D^{-1} gamma5: the oracle's adjoint operator gives the residual."""
    dims = (8, 4, 4, 8)
    m0, c_sw = -0.1, 1.0
    U = syn.gauge_field(dims, "exp", 0.3, seed=701)
    b = syn.gaussian_spinors(dims, 3, 702)
    lat = lq.Lattice(dims)
    lat.set_gauge(dev(U))
    lat.set_clover(m0, c_sw)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    res = lat.solve(dev(b), x, 3, op=op, precision=precision, tol=1e-10, dagger=True)
    torch.cuda.synchronize()
    assert res.status == lq.OK
    C = oracle.clover_term(U, c_sw)
    xs = x.cpu().numpy()
    r = b - adjoint.apply_D_dagger(U, xs, m0, C)
    rel = [np.linalg.norm(r[k]) / np.linalg.norm(b[k]) for k in range(3)]
    assert max(rel) <= 1e-10, rel
    # D x = b is a different system
    r2 = b - oracle.apply_D(U, xs, m0, C)
    assert min(np.linalg.norm(r2[k]) / np.linalg.norm(b[k]) for k in range(3)) > 1e-3
    lat.close()


@pytest.mark.parametrize("dims,c_sw", [((4, 4, 4, 4), 1.0), ((4, 2, 6, 4), 1.7), ((2, 2, 2, 2), 1.0),
                                       ((4, 4, 4, 4), 0.0)])
def test_force_kernel_matches_oracle(dims, c_sw):
    """lqcd_force on the oracle's x and lambda equals the oracle's dL/dU element-wise (FP64)."""
    m0 = 0.2
    U = syn.gauge_field(dims, "exp", 0.4, seed=711)
    x = syn.gaussian_spinors(dims, 3, 712)
    lam = syn.gaussian_spinors(dims, 3, 713)
    G_ref = adjoint.hopping_gradient(U, x, lam) + adjoint.clover_gradient(U, x, lam, c_sw)
    lat = lq.Lattice(dims)
    lat.set_gauge(dev(U))
    lat.set_clover(m0, c_sw)
    G = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
    lat.force(3, dev(x), dev(lam), G)
    torch.cuda.synchronize()
    Gg = G.cpu().numpy()
    assert np.max(np.abs(Gg - G_ref)) <= 1e-12 * np.max(np.abs(G_ref))
    lat.close()


def test_autograd_matches_oracle_gradients():
    """End to end: the autograd solve's dL/db and dL/dU equal the oracle's (4^4, clover, 2 rhs)."""
    dims = (4, 4, 4, 4)
    m0, c_sw = 0.1, 1.0
    U = syn.gauge_field(dims, "exp", 0.3, seed=721)
    b = syn.gaussian_spinors(dims, 2, 722)
    eta = syn.gaussian_spinors(dims, 2, 723)
    _, _, gb_ref, gU_ref = adjoint.gradients(U, m0, c_sw, b, eta, tol=1e-13)
    lat = lq.Lattice(dims)
    Ut = dev(U).requires_grad_(True)
    bt = dev(b).requires_grad_(True)
    x = lq.solve_differentiable(lat, Ut, bt, m0, c_sw, precision=lq.C128, tol=1e-13, op=lq.OP_SCHUR)
    L = (torch.conj(dev(eta)) * x).real.sum()
    L.backward()
    assert np.linalg.norm(bt.grad.cpu().numpy() - gb_ref) <= 1e-10 * np.linalg.norm(gb_ref)
    assert np.linalg.norm(Ut.grad.cpu().numpy() - gU_ref) <= 1e-10 * np.linalg.norm(gU_ref)
    lat.close()


def test_autograd_finite_differences_16x4():
    """16^4 Wilson-clover, 8 rhs: gradients from FP32-inner / FP64-refined solves (tol 1e-10) against central
    finite differences (h = 1e-6) of L computed with FP64 solves to 1e-14, along random directions in b and U."""
    dims = (16, 16, 16, 16)
    m0, c_sw, nrhs = -0.05, 1.0, 8
    U = syn.gauge_field(dims, "exp", 0.3, seed=4001)
    b = syn.gaussian_spinors(dims, nrhs, 4002)
    eta = syn.gaussian_spinors(dims, nrhs, 4003)
    lat = lq.Lattice(dims)
    Ut = dev(U).requires_grad_(True)
    bt = dev(b).requires_grad_(True)
    etat = dev(eta)
    x = lq.solve_differentiable(lat, Ut, bt, m0, c_sw, precision=lq.C64, tol=1e-10, op=lq.OP_SCHUR)
    L = (torch.conj(etat) * x).real.sum()
    L.backward()
    gb, gU = bt.grad, Ut.grad

    def loss(Uv, bv):
        lat.set_gauge(Uv)
        lat.set_clover(m0, c_sw)
        xx = torch.zeros_like(bv)
        r = lat.solve(bv, xx, nrhs, precision=lq.C128, tol=1e-14, op=lq.OP_SCHUR, max_restarts=2000)
        assert r.status == lq.OK, r
        return float((torch.conj(etat) * xx).real.sum())

    g = torch.Generator(device="cuda").manual_seed(3)
    h = 1e-6
    Ud, bd = Ut.detach(), bt.detach()
    db = torch.randn(b.shape, dtype=torch.complex128, device="cuda", generator=g)
    fd_b = (loss(Ud, bd + h * db) - loss(Ud, bd - h * db)) / (2 * h)
    an_b = float((torch.conj(gb) * db).real.sum())
    assert abs(fd_b - an_b) <= 1e-6 * abs(an_b), (fd_b, an_b)
    dU = torch.randn(U.shape, dtype=torch.complex128, device="cuda", generator=g)
    fd_U = (loss(Ud + h * dU, bd) - loss(Ud - h * dU, bd)) / (2 * h)
    an_U = float((torch.conj(gU) * dU).real.sum())
    assert abs(fd_U - an_U) <= 1e-6 * abs(an_U), (fd_U, an_U)
    lat.close()
