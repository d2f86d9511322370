"""GPU batched GMRES (through lqcd_solve) checked against the FP64 oracle.

A solve is accepted when the ORACLE's operator applied to the GPU solution
gives ||b - D x|| / ||b|| <= tol for every rhs (the solution itself is unique,
the iterates are not: the GPU uses CGS2 where the oracle uses MGS). The GPU
solution is also compared with the oracle's solve; their difference is bounded
by about cond(D) * tol, checked loosely.
"""
import numpy as np
import pytest

import oracle
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


def oracle_relres(U, m0, c_sw, b, x):
    C = oracle.clover_term(U, c_sw) if c_sw else None
    r = b - oracle.apply_D(U, x, m0, C)
    return np.array([np.linalg.norm(r[k]) / np.linalg.norm(b[k]) for k in range(b.shape[0])])


@pytest.mark.parametrize("op", [lq.OP_FULL, lq.OP_SCHUR])
@pytest.mark.parametrize("precision", [lq.C128, lq.C64])
def test_haar_4x4_wilson_solve(op, precision):
    """4^4, Wilson, m0 = 0.1, Haar links, one rhs, GMRES(30) to 1e-10, full and odd-even."""
    dims = (4, 4, 4, 4)
    U = syn.gauge_field(dims, "haar", seed=0)
    b = syn.gaussian_spinors(dims, 1, 1)
    lat = lq.Lattice(dims)
    lat.set_gauge(U)
    lat.set_clover(0.1, 0.0)
    x = np.zeros_like(b)
    res = lat.solve(b, x, 1, op=op, precision=precision, restart_len=30, tol=1e-10, use_graph=False)
    assert res.status == lq.OK
    rel = oracle_relres(U, 0.1, 0.0, b, x)
    assert np.all(rel <= 1e-10), rel
    assert res.relres_max <= 1e-10
    xo, _ = oracle.solve_full(U, None, 0.1, b, tol=1e-12, m=30, max_restarts=50)
    assert np.linalg.norm(x - xo) <= 1e-7 * np.linalg.norm(xo)
    lat.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_clover_multi_rhs_eo_mixed(use_graph):
    """8^4 Wilson-clover (eps 0.3, m0 = -0.2), 5 rhs (odd count), mixed precision, odd-even."""
    dims = (8, 8, 8, 8)
    m0, c_sw = -0.2, 1.0
    U = syn.gauge_field(dims, "exp", 0.3, seed=1001)
    b = syn.gaussian_spinors(dims, 5, 1002)
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    res = lat.solve(torch.from_numpy(b).cuda(), x, 5, op=lq.OP_SCHUR, precision=lq.C64, restart_len=32,
                    tol=1e-10, use_graph=use_graph)
    torch.cuda.synchronize()
    assert res.status == lq.OK, res
    rel = oracle_relres(U, m0, c_sw, b, x.cpu().numpy())
    assert np.all(rel <= 1e-10), rel
    assert np.allclose(rel, res.relres_per_rhs, rtol=1e-3, atol=1e-13)
    lat.close()


def test_fp64_and_mixed_agree_and_eo_needs_fewer_iterations():
    dims = (8, 4, 4, 8)
    m0, c_sw = 0.0, 1.0
    U = syn.gauge_field(dims, "exp", 0.3, seed=77)
    b = syn.gaussian_spinors(dims, 2, 78)
    lat = lq.Lattice(dims)
    lat.set_gauge(U)
    lat.set_clover(m0, c_sw)
    out = {}
    for op in (lq.OP_FULL, lq.OP_SCHUR):
        for prec in (lq.C128, lq.C64):
            x = np.zeros_like(b)
            res = lat.solve(b, x, 2, op=op, precision=prec, restart_len=16, tol=1e-10)
            assert res.status == lq.OK
            assert np.all(oracle_relres(U, m0, c_sw, b, x) <= 1e-10)
            # FP64 Arnoldi recomputes the FP64 residual at every restart; the mixed solve
            # only after each inner solve (nested refinement)
            if prec == lq.C128:
                assert res.outer_steps == res.restarts + 1
            else:
                assert 2 <= res.outer_steps <= res.restarts + 1
            out[(op, prec)] = (x, res)
    xs = [v[0] for v in out.values()]
    for x in xs[1:]:
        assert np.linalg.norm(x - xs[0]) <= 1e-7 * np.linalg.norm(xs[0])
    assert out[(lq.OP_SCHUR, lq.C128)][1].iterations < out[(lq.OP_FULL, lq.C128)][1].iterations
    lat.close()


def test_initial_guess_and_zero_rhs():
    """x0 = the solution converges with no iteration; a zero rhs gives x = 0."""
    dims = (4, 4, 4, 4)
    U = syn.gauge_field(dims, "exp", 0.3, seed=5)
    lat = lq.Lattice(dims)
    lat.set_gauge(U)
    lat.set_clover(0.1, 1.0)
    b = syn.gaussian_spinors(dims, 2, 6)
    b[1] = 0
    x = np.zeros_like(b)
    res = lat.solve(b, x, 2, op=lq.OP_SCHUR, precision=lq.C128, restart_len=20, tol=1e-11)
    assert res.status == lq.OK and np.all(x[1] == 0)
    x2 = x.copy()
    res2 = lat.solve(b, x2, 2, op=lq.OP_SCHUR, precision=lq.C128, restart_len=20, tol=1e-10, x0_given=True)
    assert res2.status == lq.OK and res2.iterations == 0 and res2.restarts == 0
    lat.close()


def test_not_converged_and_nonfinite_status():
    dims = (4, 4, 4, 4)
    U = syn.gauge_field(dims, "exp", 0.3, seed=5)
    lat = lq.Lattice(dims)
    lat.set_gauge(U)
    lat.set_clover(-0.2, 1.0)
    b = syn.gaussian_spinors(dims, 1, 6)
    x = np.zeros_like(b)
    res = lat.solve(b, x, 1, op=lq.OP_FULL, precision=lq.C128, restart_len=2, max_restarts=1, tol=1e-12)
    assert res.status == lq.NOT_CONVERGED and res.relres_max > 1e-12
    b[0, 0, 0, 0, 0, 0, 0] = np.nan
    with pytest.raises(lq.LqcdError) as ei:
        lat.solve(b, x, 1, op=lq.OP_FULL, precision=lq.C128)
    assert ei.value.status == lq.ERR_NONFINITE
    lat.close()


@pytest.mark.parametrize("op", [lq.OP_SCHUR, lq.OP_FULL])
def test_bf16_basis_solve(op):
    """FP32 Arnoldi with the basis stored in BF16 inside FP64 restarts still reaches 1e-10."""
    dims = (8, 8, 8, 8)
    m0, c_sw = -0.2, 1.0
    U = syn.gauge_field(dims, "exp", 0.3, seed=1001)
    b = syn.gaussian_spinors(dims, 4, 1003)
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    x = np.zeros_like(b)
    res = lat.solve(b, x, 4, op=op, precision=lq.BF16S, restart_len=32, tol=1e-10)
    assert res.status == lq.OK, res
    rel = oracle_relres(U, m0, c_sw, b, x)
    assert np.all(rel <= 1e-10), rel
    lat.close()


def test_uneven_multi_lattice_batch_solve():
    """Three lattices of different size, mass, gauge roughness and rhs count solved as one batch:
    every rhs meets tol with the oracle's operator, the per-lattice results equal the single
    solves' to rounding, and the lattices needing fewer restarts retire first."""
    specs = [((4, 4, 4, 4), 0.2, 0.05, 2), ((8, 8, 8, 8), 0.3, -0.15, 4), ((8, 4, 4, 8), 0.4, 0.0, 3)]
    lats, Us, bs, xs = [], [], [], []
    for k, (dims, eps, m0, nr) in enumerate(specs):
        U = syn.gauge_field(dims, "exp", eps, seed=3000 + k)
        lat = lq.Lattice(dims)
        lat.set_gauge(torch.from_numpy(U).cuda())
        lat.set_clover(m0, 1.0)
        lats.append(lat)
        Us.append(U)
        bs.append(torch.from_numpy(syn.gaussian_spinors(dims, nr, 3100 + k)).cuda())
        xs.append(torch.zeros_like(bs[-1]))
    res = lq.solve_batch(lats, bs, xs, [s[3] for s in specs], op=lq.OP_SCHUR, precision=lq.C64, restart_len=16,
                         tol=1e-10)
    torch.cuda.synchronize()
    for k, (dims, eps, m0, nr) in enumerate(specs):
        assert res[k].status == lq.OK, res[k]
        rel = oracle_relres(Us[k], m0, 1.0, bs[k].cpu().numpy(), xs[k].cpu().numpy())
        assert np.all(rel <= 1e-10), (k, rel)
        x1 = torch.zeros_like(bs[k])
        r1 = lats[k].solve(bs[k], x1, nr, op=lq.OP_SCHUR, precision=lq.C64, restart_len=16, tol=1e-10)
        torch.cuda.synchronize()
        assert r1.iterations == res[k].iterations and r1.restarts == res[k].restarts
        assert torch.allclose(x1, xs[k], rtol=0, atol=1e-12 * float(x1.abs().max()))
    assert len({r.restarts for r in res}) > 1      # uneven: the lattices retire at different rounds
    for lat in lats:
        lat.close()


@pytest.mark.parametrize("nrhs,precision,restart_len", [(64, lq.C64, 8), (40, lq.BF16S, 12), (1, lq.BF16S, 20),
                                                         (3, lq.C64, 64), (2, lq.C128, 1)])
def test_solver_size_limits(nrhs, precision, restart_len):
    """Largest rhs block (64: two rhs per lane in the streaming Gram-Schmidt kernel), BF16 with an even nrhs > 32,
    the largest restart length (64 basis vectors: the register-tiled kernel above 32) and GMRES(1)."""
    dims = (4, 4, 4, 4)
    m0, c_sw = 0.3, 1.0
    U = syn.gauge_field(dims, "exp", 0.2, seed=801)
    b = syn.gaussian_spinors(dims, nrhs, 802)
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    res = lat.solve(torch.from_numpy(b).cuda(), x, nrhs, op=lq.OP_SCHUR, precision=precision,
                    restart_len=restart_len, tol=1e-10, max_restarts=2000)
    torch.cuda.synchronize()
    assert res.status == lq.OK, res
    rel = oracle_relres(U, m0, c_sw, b, x.cpu().numpy())
    assert np.all(rel <= 1e-10), rel
    lat.close()


@pytest.fixture(scope="module")
def bench_problem():
    """The bench workload's inputs and the oracle's clover term (computed once)."""
    dims = (32, 16, 16, 16)
    U = syn.gauge_field(dims, "exp", 0.3, seed=1000)
    b = syn.gaussian_spinors(dims, 16, 1001)
    return dims, U, b, oracle.clover_term(U, 1.0)


@pytest.mark.parametrize("precision", [lq.C64, lq.BF16S])
def test_bench_configuration_solve_sampled(precision, bench_problem):
    """The bench's timed solve (16^3 x 32, clover, exp(i 0.3 H), m0 = -0.2, 16 rhs, odd-even GMRES(32) in FP64
    refinement, tol 1e-10, CUDA graphs): the oracle's residual of rhs 0 and 15 of the GPU solution is <= 1e-10."""
    dims, U, b, C = bench_problem
    m0, c_sw, nrhs = -0.2, 1.0, 16
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    res = lat.solve(torch.from_numpy(b).cuda(), x, nrhs, op=lq.OP_SCHUR, precision=precision, restart_len=32,
                    tol=1e-10, max_restarts=500, use_graph=True)
    torch.cuda.synchronize()
    assert res.status == lq.OK, res
    xs = x.cpu().numpy()
    lat.close()
    for k in (0, nrhs - 1):
        r = b[k:k + 1] - oracle.apply_D(U, xs[k:k + 1], m0, C)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b[k]), k


@pytest.mark.parametrize("precision,op", [(lq.C64, lq.OP_SCHUR), (lq.BF16S, lq.OP_SCHUR), (lq.C64, lq.OP_FULL)])
def test_gram_schmidt_modes_agree(precision, op):
    """CGS1, CGS2 and the delayed CGS2 (two basis passes per step) all reach the tolerance with the oracle's
    operator; the delayed variant builds the same Krylov basis as CGS2, so its iteration count stays close."""
    dims = (8, 8, 8, 8)
    m0, c_sw = -0.2, 1.0
    U = syn.gauge_field(dims, "exp", 0.3, seed=1001)
    b = syn.gaussian_spinors(dims, 6, 1005)
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    its = {}
    for reorth in ((0, 1, 2) if precision == lq.C64 else (1, 2)):
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        res = lat.solve(torch.from_numpy(b).cuda(), x, 6, op=op, precision=precision, restart_len=32, tol=1e-10,
                        reorth=reorth)
        torch.cuda.synchronize()
        assert res.status == lq.OK, (reorth, res)
        rel = oracle_relres(U, m0, c_sw, b, x.cpu().numpy())
        assert np.all(rel <= 1e-10), (reorth, rel)
        its[reorth] = res.iterations
        assert res.ortho == reorth, (reorth, res.ortho)
    assert abs(its[2] - its[1]) <= max(4, its[1] // 10), its
    lat.close()


@pytest.mark.gpu
def test_delayed_gram_schmidt_selection():
    """reorth = 2 runs the delayed CGS2 where its kernels apply (FP32 / BF16 basis, restart length <= 32,
    nrhs <= 32 or even nrhs <= 64) and CGS2 otherwise; every case converges."""
    dims = (4, 4, 4, 4)
    m0, c_sw = 0.1, 1.0
    U = syn.gauge_field(dims, "exp", 0.3, seed=1201)
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    cases = [  # (nrhs, precision, restart_len, expected Gram-Schmidt)
        (4, lq.C64, 32, 2), (4, lq.BF16S, 32, 2), (40, lq.C64, 16, 2), (33, lq.C64, 16, 1),
        (40, lq.BF16S, 16, 2), (4, lq.C64, 40, 1), (4, lq.C128, 16, 1), (3, lq.C64, 1, 2)]
    for nrhs, prec, m, expect in cases:
        b = syn.gaussian_spinors(dims, nrhs, 1202 + nrhs)
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        res = lat.solve(torch.from_numpy(b).cuda(), x, nrhs, op=lq.OP_SCHUR, precision=prec, restart_len=m,
                        tol=1e-10, max_restarts=2000, reorth=2)
        torch.cuda.synchronize()
        assert res.status == lq.OK, (nrhs, prec, m, res)
        assert res.ortho == expect, (nrhs, prec, m, res.ortho)
        rel = oracle_relres(U, m0, c_sw, b, x.cpu().numpy())
        assert np.all(rel <= 1e-10), (nrhs, prec, m, rel.max())
    lat.close()


def _plane_wave(dims, n, u, bc=-1):
    """psi(x) = exp(i p.x) u with p_mu = 2 pi n_mu / L_mu in space and pi (2 n_0 + 1) / T in time (an
    antiperiodic momentum), u a 4x3 spin-colour vector: at U = 1 an eigenvector of the free operator's
    translation part, so D psi lies in the span of exp(i p.x) times the spin space."""
    t, z, y, x = np.indices(dims)
    p = [np.pi * (2 * n[0] + (1 if bc == -1 else 0)) / dims[0]] + [2 * np.pi * n[k] / dims[k] for k in (1, 2, 3)]
    phase = np.exp(1j * (p[0] * t + p[1] * z + p[2] * y + p[3] * x))
    return phase[..., None, None] * u[None, None, None, None]


@pytest.mark.parametrize("precision", [lq.C64, lq.BF16S, lq.C128])
@pytest.mark.parametrize("op", [lq.OP_SCHUR, lq.OP_FULL])
@pytest.mark.parametrize("reorth", [2, 1])
def test_near_breakdown_plane_wave_solve(precision, op, reorth):
    """Free field (U = 1): a rhs made of plane waves spans a Krylov space of dimension <= 2 per momentum
    (the free operator restricted to one momentum has two distinct eigenvalues, m0 + sum(1 - cos p) +- i|sin p|,
    and the Schur complement is a function of it there), so the Arnoldi process hits a (near) happy breakdown
    after two steps per momentum: h_{j+1,j} and, in the delayed CGS2, nu^2 = ||w||^2 - ||z||^2 cancel to
    rounding. The solve must still reach 1e-10 with the oracle's operator, without non-finite values; the FP64
    solve stops at the breakdown, the mixed-precision solves refine the FP32 rounding noise afterwards."""
    dims = (8, 4, 4, 8)
    m0 = 0.1
    U = syn.unit_gauge(dims)
    rng = np.random.default_rng(77)
    u1 = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    u2 = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    b = np.stack([_plane_wave(dims, (1, 0, 1, 2), u1),
                  _plane_wave(dims, (0, 1, 0, 1), u1) + 0.5 * _plane_wave(dims, (2, 1, 3, 0), u2)])
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, 1.0)        # C(x) = 0 at U = 1
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    prec_reorth = 1 if (precision == lq.BF16S and reorth == 0) else reorth
    res = lat.solve(torch.from_numpy(b).cuda(), x, 2, op=op, precision=precision, restart_len=32, tol=1e-10,
                    reorth=prec_reorth, max_restarts=200)
    torch.cuda.synchronize()
    assert res.status == lq.OK, res
    xs = x.cpu().numpy()
    assert np.all(np.isfinite(xs))
    rel = oracle_relres(U, m0, 0.0, b, xs)
    assert np.all(rel <= 1e-10), rel
    if precision == lq.C128:
        # exact arithmetic would need 2 and 4 steps; the FP64 solve stops at the breakdown
        assert res.iters_per_rhs[0] <= 3 and res.iters_per_rhs[1] <= 6, res.iters_per_rhs
    else:
        assert res.iterations <= 64, res.iters_per_rhs
    lat.close()


@pytest.mark.parametrize("precision", [lq.C64, lq.C128])
@pytest.mark.parametrize("op", [lq.OP_SCHUR, lq.OP_FULL])
def test_retirement_compacts_the_active_rhs(precision, op):
    """Eight rhs of uneven difficulty: rhs 0-1 start at the oracle's solution (retired at the first
    restart), rhs 2-3 near it (relative error 1e-6: they retire after a few cycles), rhs 4-7 from zero.
    With compaction the retired rhs leave the block (the operator then runs on fewer rhs, so its
    algorithmic bytes per launch fall); every rhs still meets the tolerance with the oracle's operator,
    the immediately retired ones keep their initial guess exactly (its odd half for odd-even), and the
    solutions agree with those of the solve without compaction."""
    dims = (8, 4, 4, 8)
    m0, c_sw, nrhs = -0.1, 1.0, 8
    U = syn.gauge_field(dims, "exp", 0.3, seed=1301)
    b = syn.gaussian_spinors(dims, nrhs, 1302)
    A, Ainv = oracle.diag_blocks(U, m0, c_sw)
    xo, _ = oracle.solve_eo(U, A, Ainv, b[:4], tol=1e-13, m=40, max_restarts=200)
    rng = np.random.default_rng(1303)
    x0 = np.zeros_like(b)
    x0[:2] = xo[:2]
    noise = rng.standard_normal(xo[2:4].shape) + 1j * rng.standard_normal(xo[2:4].shape)
    x0[2:4] = xo[2:4] + 1e-6 * noise * (np.linalg.norm(xo[2:4]) / np.linalg.norm(noise))
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    out = {}
    for compact in (True, False):
        x = torch.from_numpy(x0.copy()).cuda()
        res = lat.solve(torch.from_numpy(b).cuda(), x, nrhs, op=op, precision=precision, restart_len=16,
                        tol=1e-10, x0_given=True, profile=True, compact=compact, max_restarts=400)
        torch.cuda.synchronize()
        assert res.status == lq.OK, (compact, res)
        xs = x.cpu().numpy()
        rel = oracle_relres(U, m0, c_sw, b, xs)
        assert np.all(rel <= 1e-10), (compact, rel)
        out[compact] = (res, xs)
    rc, xc = out[True]
    rn, xn = out[False]
    # immediately retired rhs: untouched (odd-even: the even half is reconstructed from the odd one at the end)
    if op == lq.OP_SCHUR:
        assert np.array_equal(oracle.split_parity(xc[:2], 1), oracle.split_parity(x0[:2], 1))
    else:
        assert np.array_equal(xc[:2], x0[:2])
    # fewer iterations for the rhs that started near the solution
    assert max(rc.iters_per_rhs[:4]) < min(rc.iters_per_rhs[4:]), rc.iters_per_rhs
    # bytes per operator launch fall once rhs retire (the non-compacting solve keeps all 8)
    assert rc.op_bytes / rc.op_launches < rn.op_bytes / rn.op_launches
    for k in range(nrhs):
        assert np.linalg.norm(xc[k] - xn[k]) <= 1e-6 * np.linalg.norm(xn[k]), k
    lat.close()


@pytest.mark.parametrize("precision", [lq.C64, lq.BF16S])
def test_mixed_solve_with_bf16_links(precision):
    """The FP32 inner operator on BF16 two-row links (an O(2^-9) perturbation of D): the FP64
    refinement on the exact links still brings every rhs to 1e-10 with the oracle's operator."""
    dims = (8, 8, 8, 8)
    m0, c_sw = -0.2, 1.0
    U = syn.gauge_field(dims, "exp", 0.3, seed=1001)
    b = syn.gaussian_spinors(dims, 4, 1401)
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    lat.set_link_storage(lq.LINKS_BF16)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    res = lat.solve(torch.from_numpy(b).cuda(), x, 4, op=lq.OP_SCHUR, precision=precision, restart_len=32,
                    tol=1e-10, max_restarts=400)
    torch.cuda.synchronize()
    assert res.status == lq.OK, res
    rel = oracle_relres(U, m0, c_sw, b, x.cpu().numpy())
    assert np.all(rel <= 1e-10), rel
    lat.close()


@pytest.mark.parametrize("nrhs", [1, 2, 6, 16])
@pytest.mark.parametrize("op", [lq.OP_SCHUR, lq.OP_FULL])
def test_block_gmres_solve(nrhs, op):
    """Block GMRES (one Krylov space shared by all rhs, FP32 inner cycles in FP64 refinement): every rhs
    meets 1e-10 with the oracle's operator, the solution agrees with the batched solver's, and the block
    space of dimension m * nrhs needs no more Arnoldi steps per rhs than the independent spaces."""
    dims = (8, 8, 8, 8)
    m0, c_sw = -0.2, 1.0
    U = syn.gauge_field(dims, "exp", 0.3, seed=1001)
    b = syn.gaussian_spinors(dims, nrhs, 1501 + nrhs)
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    xb = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    rb = lat.solve(torch.from_numpy(b).cuda(), xb, nrhs, op=op, precision=lq.C64, restart_len=32, tol=1e-10,
                   block=True, max_restarts=400)
    xn = torch.zeros_like(xb)
    rn = lat.solve(torch.from_numpy(b).cuda(), xn, nrhs, op=op, precision=lq.C64, restart_len=32, tol=1e-10,
                   max_restarts=400)
    torch.cuda.synchronize()
    assert rb.status == lq.OK and rn.status == lq.OK, (rb, rn)
    xs = xb.cpu().numpy()
    rel = oracle_relres(U, m0, c_sw, b, xs)
    assert np.all(rel <= 1e-10), rel
    assert np.allclose(rel, rb.relres_per_rhs, rtol=1e-3, atol=1e-13)
    xr = xn.cpu().numpy()
    for k in range(nrhs):
        assert np.linalg.norm(xs[k] - xr[k]) <= 1e-6 * np.linalg.norm(xr[k]), k
    assert rb.iterations <= rn.iterations + 8, (rb.iterations, rn.iterations)
    lat.close()


def test_block_gmres_argument_checks():
    dims = (4, 4, 4, 4)
    lat = lq.Lattice(dims)
    lat.set_gauge(syn.gauge_field(dims, "exp", 0.3, seed=3))
    lat.set_clover(0.1, 1.0)
    b = syn.gaussian_spinors(dims, 17, 4)
    with pytest.raises(lq.LqcdError):   # at most 16 rhs per block
        lat.solve(b, np.zeros_like(b), 17, precision=lq.C64, block=True)
    with pytest.raises(lq.LqcdError):   # FP32 inner cycles only
        lat.solve(b[:2], np.zeros_like(b[:2]), 2, precision=lq.C128, block=True)
    lat.close()
