"""GPU parity of the operator path (through the C ABI) against the FP64 oracle.

Tolerances (norm-wise relative, per rhs): FP64 1e-12 (the applies are exact
linear algebra; the two sides differ only in summation order, ~1e-15);
FP32 5e-6: inputs rounded to FP32 (relative 6e-8) and about a hundred
accumulated products per output component give an expected relative error of
~1e-6 for Gaussian inputs, so 5e-6 leaves a factor of a few.
Layout conversion is bit-exact.
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


TOL = {lq.C128: 1e-12, lq.C64: 5e-6}

_CACHE = {}


def setup(dims, kind, eps, m0, c_sw, seed):
    key = (dims, kind, eps, m0, c_sw, seed)
    if key not in _CACHE:
        U = syn.gauge_field(dims, kind, eps, seed=seed)
        lat = lq.Lattice(dims, time_bc=-1)
        lat.set_gauge(torch.from_numpy(U).cuda())
        lat.set_clover(m0, c_sw)
        C = oracle.clover_term(U, c_sw)
        A, Ainv = oracle.diag_blocks(U, m0, c_sw)
        _CACHE[key] = (lat, U, C, A, Ainv)
    return _CACHE[key]


def dev(a, dtype):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dtype == lq.C128 else t.to(torch.complex64)).cuda()


def relerr(got, ref):
    got = np.asarray(got, dtype=np.complex128).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return max(np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k]) for k in range(ref.shape[0]))


CASES = [
    # dims, gauge kind, eps, m0, c_sw
    ((4, 4, 4, 4), "exp", 0.3, -0.2, 1.0),
    ((4, 4, 4, 4), "haar", 0.0, 0.1, 0.0),
    ((8, 2, 6, 4), "exp", 0.5, 0.05, 1.3),     # non-cubic: catches stride mistakes
    ((2, 2, 2, 2), "exp", 0.7, 0.2, 1.0),      # both hops on one site; site tile capped at 8
]


@pytest.mark.parametrize("case", CASES)
def test_site_blocks_match_oracle(case):
    dims, kind, eps, m0, c_sw = case
    lat, U, C, A, Ainv = setup(dims, kind, eps, m0, c_sw, 101)
    V = lat.V
    out = torch.empty((V, 12, 12), dtype=torch.complex128, device="cuda")
    for which, ref in ((0, A), (1, Ainv)):
        lat.export_blocks(which, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(ref.shape)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("dtype", [lq.C64, lq.C128])
@pytest.mark.parametrize("nrhs", [1, 3, 12, 16])
@pytest.mark.parametrize("sites", [lq.SITES_FULL, lq.SITES_ODD])
def test_pack_unpack_roundtrip_bit_exact(dtype, nrhs, sites):
    lat, *_ = setup((8, 2, 6, 4), "exp", 0.5, 0.05, 1.3, 101)
    n_sites = lat.V if sites == lq.SITES_FULL else lat.V // 2
    g = torch.Generator(device="cpu").manual_seed(nrhs)
    src = torch.randn((nrhs, n_sites, 4, 3), dtype=torch.complex128, generator=g)
    src = src if dtype == lq.C128 else src.to(torch.complex64)
    src = src.cuda()
    packed = lat.packed_empty(dtype, sites, nrhs)
    back = torch.empty_like(src)
    lat.pack(sites, nrhs, src, packed)
    lat.unpack(sites, nrhs, packed, back)
    torch.cuda.synchronize()
    assert torch.equal(src, back)
    # spot-check the packed position of (site i, component c, rhs r)
    S = lat.site_tile(nrhs)
    p = packed.cpu()
    s = src.cpu().reshape(nrhs, n_sites, 12)
    for (i, c, r) in [(0, 0, 0), (n_sites - 1, 11, nrhs - 1), (n_sites // 3, 5, nrhs // 2)]:
        if sites == lq.SITES_FULL:
            t, z, y, x = np.unravel_index(i, lat.dims)
            par = (t + z + y + x) % 2
            e = par * (lat.V // 2) + i // 2
        else:
            e = i
        idx = ((e // S) * 12 + c) * S * nrhs + (e % S) * nrhs + r
        assert p[idx] == s[r, i, c]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("dtype", [lq.C128, lq.C64])
@pytest.mark.parametrize("nrhs", [1, 2, 3, 13, 16])
def test_full_operator(case, dtype, nrhs):
    dims, kind, eps, m0, c_sw = case
    lat, U, C, A, Ainv = setup(dims, kind, eps, m0, c_sw, 101)
    psi = syn.gaussian_spinors(dims, nrhs, 200 + nrhs)
    ref = oracle.apply_D(U, psi, m0, C if c_sw else None)
    d_in = dev(psi, dtype)
    d_out = torch.empty_like(d_in)
    lat.apply(lq.OP_FULL, nrhs, d_in, d_out)
    torch.cuda.synchronize()
    assert relerr(d_out.cpu().numpy(), ref) < TOL[dtype]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("dtype", [lq.C128, lq.C64])
@pytest.mark.parametrize("nrhs", [1, 4, 12, 13])
def test_schur_operator(case, dtype, nrhs):
    dims, kind, eps, m0, c_sw = case
    lat, U, C, A, Ainv = setup(dims, kind, eps, m0, c_sw, 101)
    psi_o = oracle.split_parity(syn.gaussian_spinors(dims, nrhs, 300 + nrhs), 1)
    ref = oracle.apply_schur(U, A, Ainv, psi_o)
    d_in = dev(psi_o, dtype)
    d_out = torch.empty_like(d_in)
    lat.apply(lq.OP_SCHUR, nrhs, d_in, d_out)
    torch.cuda.synchronize()
    assert relerr(d_out.cpu().numpy(), ref) < TOL[dtype]


@pytest.mark.parametrize("case", CASES[:3])
@pytest.mark.parametrize("dtype", [lq.C128, lq.C64])
def test_schur_prepare_reconstruct(case, dtype):
    dims, kind, eps, m0, c_sw = case
    lat, U, C, A, Ainv = setup(dims, kind, eps, m0, c_sw, 101)
    nrhs = 3
    b = syn.gaussian_spinors(dims, nrhs, 400)
    x_o = oracle.split_parity(syn.gaussian_spinors(dims, nrhs, 401), 1)
    b_e, b_o = oracle.split_parity(b, 0), oracle.split_parity(b, 1)
    ref_bhat = oracle.schur_prepare(U, Ainv, b_e, b_o)
    ref_xe = oracle.schur_reconstruct(U, Ainv, b_e, x_o)
    bp = lat.packed_empty(dtype, lq.SITES_FULL, nrhs)
    lat.pack(lq.SITES_FULL, nrhs, dev(b, dtype), bp)
    bhat_p = lat.packed_empty(dtype, lq.SITES_ODD, nrhs)
    lat.schur_prepare(nrhs, bp, bhat_p)
    bhat = torch.empty((nrhs, lat.V // 2, 4, 3), dtype=bp.dtype, device="cuda")
    lat.unpack(lq.SITES_ODD, nrhs, bhat_p, bhat)
    xo_p = lat.packed_empty(dtype, lq.SITES_ODD, nrhs)
    lat.pack(lq.SITES_ODD, nrhs, dev(x_o, dtype), xo_p)
    x_p = lat.packed_empty(dtype, lq.SITES_FULL, nrhs)
    lat.schur_reconstruct(nrhs, bp, xo_p, x_p)
    x = torch.empty((nrhs, lat.V, 4, 3), dtype=bp.dtype, device="cuda")
    lat.unpack(lq.SITES_FULL, nrhs, x_p, x)
    torch.cuda.synchronize()
    assert relerr(bhat.cpu().numpy(), ref_bhat) < TOL[dtype]
    xfull = x.cpu().numpy().reshape((nrhs,) + dims + (4, 3))
    assert relerr(oracle.split_parity(xfull, 0), ref_xe) < TOL[dtype]
    assert np.array_equal(oracle.split_parity(xfull, 1).astype(np.complex128),
                          x_o.astype(xfull.dtype).astype(np.complex128))


@pytest.mark.parametrize("dtype", [lq.C128, lq.C64])
@pytest.mark.parametrize("nvec,nrhs,reorth", [(1, 1, True), (5, 3, True), (17, 12, False), (32, 16, True),
                                               (40, 16, True), (9, 40, True), (20, 2, True), (12, 6, True),
                                               (33, 64, True), (32, 64, True), (24, 40, False), (7, 5, True),
                                               (17, 1, True), (3, 31, True)])
def test_orthogonalise_matches_projection(dtype, nvec, nrhs, reorth):
    """h = V^H w and w' = (1 - V V^H) w per rhs for an orthonormal basis (numpy QR)."""
    lat, *_ = setup((4, 4, 4, 4), "exp", 0.3, -0.2, 1.0, 101)
    n_sites = lat.V // 2
    rng = np.random.default_rng(nvec * 100 + nrhs)
    N = n_sites * 12
    Vb = np.empty((nvec, nrhs, N), complex)
    for r in range(nrhs):
        Z = rng.standard_normal((N, nvec)) + 1j * rng.standard_normal((N, nvec))
        Q, _ = np.linalg.qr(Z)
        Vb[:, r, :] = Q.T
    w = rng.standard_normal((nrhs, N)) + 1j * rng.standard_normal((nrhs, N))
    if dtype == lq.C64:   # reference on the FP32-rounded inputs
        Vb = Vb.astype(np.complex64).astype(complex)
        w = w.astype(np.complex64).astype(complex)
    h_ref = np.einsum("irn,rn->ir", Vb.conj(), w)
    w_ref = w - np.einsum("irn,ir->rn", Vb, h_ref)
    basis = torch.cat([lat.packed_empty(dtype, lq.SITES_ODD, nrhs) for _ in range(nvec)])
    nb = basis.numel() // nvec
    for i in range(nvec):
        lat.pack(lq.SITES_ODD, nrhs, dev(Vb[i].reshape(nrhs, n_sites, 4, 3), dtype), basis[i * nb:(i + 1) * nb])
    wp = lat.packed_empty(dtype, lq.SITES_ODD, nrhs)
    lat.pack(lq.SITES_ODD, nrhs, dev(w.reshape(nrhs, n_sites, 4, 3), dtype), wp)
    h = torch.empty((nvec, nrhs), dtype=torch.complex128, device="cuda")
    hn = torch.empty(nrhs, dtype=torch.float64, device="cuda")
    lat.orthogonalise(lq.SITES_ODD, nrhs, nvec, basis, wp, h, hn, reorth=reorth)
    wout = torch.empty((nrhs, n_sites, 4, 3), dtype=wp.dtype, device="cuda")
    lat.unpack(lq.SITES_ODD, nrhs, wp, wout)
    torch.cuda.synchronize()
    tol = 1e-12 if dtype == lq.C128 else 2e-5
    assert np.max(np.abs(h.cpu().numpy() - h_ref)) < tol * np.max(np.abs(h_ref)) * 10
    got_w = wout.cpu().numpy().reshape(nrhs, N)
    assert relerr(got_w, w_ref) < (1e-12 if dtype == lq.C128 else 1e-5)
    assert np.allclose(hn.cpu().numpy(), np.linalg.norm(got_w, axis=1), rtol=1e-6 if dtype == lq.C64 else 1e-12)


@pytest.mark.parametrize("dtype", [lq.C64, lq.C128])
@pytest.mark.parametrize("nrhs", [16, 64])
def test_operator_sweep_lattice_sampled_rhs(dtype, nrhs):
    """16^3 x 32, Wilson-clover, nrhs = 16 and 64 in the launch configuration the bench's operator
    sweep times (the autotuner's choice for that nrhs); the first and last rhs checked against the
    oracle (rhs are independent)."""
    dims = (32, 16, 16, 16)
    m0, c_sw = -0.2, 1.0
    U = syn.gauge_field(dims, "exp", 0.3, seed=1 * 1000 + 1)
    lat = lq.Lattice(dims, time_bc=-1)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    lat.tune(dtype, nrhs, reps=2)
    psi = syn.gaussian_spinors(dims, nrhs, 1 * 1000 + 2)
    psi_o = oracle.split_parity(psi, 1)
    sample = [0, nrhs - 1]
    A, Ainv = oracle.diag_blocks(U, m0, c_sw)
    ref_s = oracle.apply_schur(U, A, Ainv, psi_o[sample])
    ref_f = oracle.apply_D(U, psi[sample], m0, oracle.clover_term(U, c_sw))
    for op, src, ref, sites in ((lq.OP_SCHUR, psi_o, ref_s, lq.SITES_ODD), (lq.OP_FULL, psi, ref_f, lq.SITES_FULL)):
        d_in = dev(src, dtype)
        pin = lat.packed_empty(dtype, sites, nrhs)
        pout = lat.packed_empty(dtype, sites, nrhs)
        lat.pack(sites, nrhs, d_in, pin)
        lat.apply_packed(op, nrhs, pin, pout)
        out = torch.empty_like(d_in)
        lat.unpack(sites, nrhs, pout, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()[sample]
        assert relerr(got, ref) < TOL[dtype], (op, lat.kernel_variant(dtype, nrhs, op))
    lat.close()


def _sample_sites(dims, parity, n, seed):
    """n sites of the given parity: the lattice corners and both time boundaries, then random ones."""
    rng = np.random.default_rng(seed)
    T, Z, Y, X = dims
    fixed = [(0, 0, 0, 1), (T - 1, Z - 1, Y - 1, X - 2), (T - 1, 0, 0, 0), (0, Z - 1, Y - 1, X - 1),
             (T - 1, Z - 1, 0, 1), (0, 0, Y - 1, 0)]
    out = [x for x in fixed if sum(x) % 2 == parity]
    while len(out) < n:
        x = tuple(int(rng.integers(0, d)) for d in dims)
        if sum(x) % 2 == parity and x not in out:
            out.append(x)
    return out


_LARGE = {}


def _large_inputs(dims, nrhs):
    """Gauge field and sources of the 32^3 x 64 workload (generated once per module: ~2 minutes)."""
    if dims not in _LARGE:
        _LARGE.clear()
        _LARGE[dims] = (syn.gauge_field(dims, "exp", 0.25, seed=2 * 1000 + 0),
                        syn.gaussian_spinors(dims, nrhs, 2 * 1000 + 1))
    return _LARGE[dims]


@pytest.mark.parametrize("dtype", [lq.C64, lq.C128])
def test_operator_32x64_lattice_sampled_sites(dtype):
    """The 32^3 x 64 Wilson-clover lattice of the large GMRES workload (eps 0.25, m0 = -0.3, 12 rhs),
    2.1 M sites, in the tuned launch configuration: Schur and full applies at sampled sites (corners, both
    time boundaries, random sites) and the first and last rhs, each output site computed one by one by the
    per-site oracle. Rules out a size-dependent indexing fault (site numbers, packed offsets and link
    offsets beyond 2^31 bytes)."""
    from oracle import site
    dims = (64, 32, 32, 32)
    m0, c_sw, nrhs = -0.3, 1.0, 12
    U, psi = _large_inputs(dims, nrhs)
    lat = lq.Lattice(dims, time_bc=-1)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(m0, c_sw)
    lat.tune(dtype, nrhs, reps=1)
    tol = 1e-12 if dtype == lq.C128 else 5e-6
    # Schur operator on the odd sites
    psi_o = oracle.split_parity(psi, 1)
    d_in = dev(psi_o, dtype)
    d_out = torch.empty_like(d_in)
    lat.apply(lq.OP_SCHUR, nrhs, d_in, d_out)
    got = d_out.cpu().numpy()
    del d_in, d_out
    for x in _sample_sites(dims, 1, 24, 5):
        k = site.half_index(dims, x)
        for r in (0, nrhs - 1):
            ref = site.apply_schur_at(U, psi_o[r], x, m0, c_sw)
            assert np.linalg.norm(got[r, k] - ref) <= tol * np.linalg.norm(ref), (x, r)
    del psi_o, got
    # full operator on all sites
    d_in = dev(psi, dtype)
    d_out = torch.empty_like(d_in)
    lat.apply(lq.OP_FULL, nrhs, d_in, d_out)
    got = d_out.cpu().numpy()
    del d_in, d_out
    for parity in (0, 1):
        for x in _sample_sites(dims, parity, 12, 6 + parity):
            for r in (0, nrhs - 1):
                ref = site.apply_D_at(U, psi[r], x, m0, c_sw)
                assert np.linalg.norm(got[(r,) + x] - ref) <= tol * np.linalg.norm(ref), (x, r)
    lat.close()


@pytest.mark.parametrize("dtype", [lq.C64, lq.C128])
@pytest.mark.parametrize("nrhs", [32, 64])
@pytest.mark.parametrize("case", [CASES[0], CASES[2]])
def test_large_nrhs_every_kernel_variant(dtype, nrhs, case):
    """nrhs 32 and 64 (two rhs per lane and the variants compiled for those counts): every launch
    variant that fits, full and Schur operator, element-wise per rhs against the oracle."""
    dims, kind, eps, m0, c_sw = case
    lat, U, C, A, Ainv = setup(dims, kind, eps, m0, c_sw, 101)
    lib = lq.load()
    psi = syn.gaussian_spinors(dims, nrhs, 700 + nrhs)
    psi_o = oracle.split_parity(psi, 1)
    ref_f = oracle.apply_D(U, psi, m0, C if c_sw else None)
    ref_s = oracle.apply_schur(U, A, Ainv, psi_o)
    ran = 0
    for v in range(lib.lqcd_kernel_variant_count(dtype)):
        for op, src, ref in ((lq.OP_FULL, psi, ref_f), (lq.OP_SCHUR, psi_o, ref_s)):
            try:
                lat.set_kernel_variant(dtype, nrhs, op, v)
            except lq.LqcdError:
                continue
            d_in = dev(src, dtype)
            d_out = torch.empty_like(d_in)
            lat.apply(op, nrhs, d_in, d_out)
            torch.cuda.synchronize()
            assert relerr(d_out.cpu().numpy(), ref) < TOL[dtype], (v, op)
            ran += 1
    for op in (lq.OP_FULL, lq.OP_SCHUR):
        lat.set_kernel_variant(dtype, nrhs, op, -1)
    assert ran >= 4


@pytest.mark.parametrize("dtype", [lq.C64, lq.C128])
def test_every_kernel_variant_and_tuner(dtype):
    """Every launch variant of the hopping kernel gives the oracle's answer, and
    the autotuner leaves a valid choice that persists through a JSON cache."""
    dims, kind, eps, m0, c_sw = CASES[0]
    lat, U, C, A, Ainv = setup(dims, kind, eps, m0, c_sw, 101)
    lib = lq.load()
    for nrhs in (4, 6, 16):   # 16: also the variants compiled for 16 rhs
        psi = syn.gaussian_spinors(dims, nrhs, 500 + nrhs)
        psi_o = oracle.split_parity(psi, 1)
        ref_f = oracle.apply_D(U, psi, m0, C)
        ref_s = oracle.apply_schur(U, A, Ainv, psi_o)
        for v in range(lib.lqcd_kernel_variant_count(dtype)):
            for op, src, ref in ((lq.OP_FULL, psi, ref_f), (lq.OP_SCHUR, psi_o, ref_s)):
                try:
                    lat.set_kernel_variant(dtype, nrhs, op, v)
                except lq.LqcdError:
                    continue      # variant does not fit nrhs
                d_in = dev(src, dtype)
                d_out = torch.empty_like(d_in)
                lat.apply(op, nrhs, d_in, d_out)
                torch.cuda.synchronize()
                assert relerr(d_out.cpu().numpy(), ref) < TOL[dtype], (v, op, nrhs)
        times = lat.tune(dtype, nrhs, reps=3)
        for op in (lq.OP_FULL, lq.OP_SCHUR):
            chosen = lat.kernel_variant(dtype, nrhs, op)
            col = 0 if op == lq.OP_FULL else 1
            ok = [t[col] for t in times if t[col] == t[col]]
            assert times[chosen][col] == min(ok)
        d_in = dev(psi_o, dtype)
        d_out = torch.empty_like(d_in)
        lat.apply(lq.OP_SCHUR, nrhs, d_in, d_out)
        torch.cuda.synchronize()
        assert relerr(d_out.cpu().numpy(), ref_s) < TOL[dtype]
    import json, os, tempfile
    path = os.path.join(tempfile.mkdtemp(), "tune.json")
    keys = [(dtype, 4, lq.OP_SCHUR), (dtype, 6, lq.OP_FULL)]
    lat.save_tuning(path, keys)
    saved = json.load(open(path))["variants"]
    for (d, n, o) in keys:
        lat.set_kernel_variant(d, n, o, -1)
    assert lat.load_tuning(path)
    for (d, n, o) in keys:
        assert lat.kernel_variant(d, n, o) == saved[f"{d},{n},{o}"]


@pytest.mark.parametrize("nrhs", [16, 32])
def test_blocked_row_variants(nrhs):
    """The variants that give each CTA a block of target rows (t, z0 .. z0 + rz - 1, y0, y0 + 1) and walk the
    directions x, y, z, t: on a lattice whose shape lets every such launch take the blocked mapping (whole
    x rows per CTA, z blocks tiling Z), the Schur operator and both single-parity hopping passes agree with
    the oracle element-wise; the full operator (both parities, linear mapping) too."""
    dims = (4, 8, 4, 8)       # T, Z, Y, X: X/2 = 4 targets per row
    lat, U, C, A, Ainv = setup(dims, "exp", 0.4, -0.1, 1.0, 303)
    lib = lq.load()
    T, Z, Y, X = dims
    psi = syn.gaussian_spinors(dims, nrhs, 900 + nrhs)
    psi_o = oracle.split_parity(psi, 1)
    ref_f = oracle.apply_D(U, psi, -0.1, C)
    ref_s = oracle.apply_schur(U, A, Ainv, psi_o)
    ran = 0
    for v in range(lib.lqcd_kernel_variant_count(lq.C64)):
        info = lat.kernel_variant_info(lq.C64, v)
        if info["order"] != 1:
            continue
        lanes = nrhs // info["nr"]
        targets = info["threads"] // lanes
        rows = targets // (X // 2)
        # the precondition of the blocked mapping holds on this lattice
        assert targets % (X // 2) == 0 and rows % 2 == 0 and Z % (rows // 2) == 0
        for op, src, ref in ((lq.OP_FULL, psi, ref_f), (lq.OP_SCHUR, psi_o, ref_s)):
            try:
                lat.set_kernel_variant(lq.C64, nrhs, op, v)
            except lq.LqcdError:
                continue
            d_in = dev(src, lq.C64)
            d_out = torch.empty_like(d_in)
            lat.apply(op, nrhs, d_in, d_out)
            torch.cuda.synchronize()
            assert relerr(d_out.cpu().numpy(), ref) < TOL[lq.C64], (v, op)
            ran += 1
    for op in (lq.OP_FULL, lq.OP_SCHUR):
        lat.set_kernel_variant(lq.C64, nrhs, op, -1)
    assert ran >= (6 if nrhs == 16 else 2)


def _bf16_round(a):
    """Round a complex array to BF16 real and imaginary parts (round to nearest even), back to complex128."""
    t = torch.from_numpy(np.ascontiguousarray(a)).to(torch.complex64)
    r = torch.view_as_real(t).to(torch.bfloat16).to(torch.float32)
    return torch.view_as_complex(r.contiguous()).numpy().astype(np.complex128)


@pytest.mark.parametrize("nrhs", [1, 6, 16])
@pytest.mark.parametrize("sites", [lq.SITES_FULL, lq.SITES_ODD])
def test_bf16_pack_roundtrip_rounds_like_torch(nrhs, sites):
    lat, *_ = setup((8, 2, 6, 4), "exp", 0.5, 0.05, 1.3, 101)
    n_sites = lat.V if sites == lq.SITES_FULL else lat.V // 2
    g = torch.Generator(device="cpu").manual_seed(7 + nrhs)
    src = torch.randn((nrhs, n_sites, 4, 3), dtype=torch.complex64, generator=g)
    packed = lat.packed_empty(lq.BF16S, sites, nrhs)
    back = torch.empty_like(src).cuda()
    lat.pack(sites, nrhs, src.cuda(), packed, dtype=lq.BF16S)
    lat.unpack(sites, nrhs, packed, back, dtype=lq.BF16S)
    torch.cuda.synchronize()
    expect = _bf16_round(src.numpy()).astype(np.complex64)
    assert np.array_equal(back.cpu().numpy(), expect)


@pytest.mark.parametrize("case", CASES[:3])
@pytest.mark.parametrize("op", [lq.OP_FULL, lq.OP_SCHUR])
@pytest.mark.parametrize("nrhs", [3, 16])
def test_bf16_storage_operator(case, op, nrhs):
    """BF16-stored input, FP32 arithmetic: equals the oracle applied to the BF16-rounded input."""
    dims, kind, eps, m0, c_sw = case
    lat, U, C, A, Ainv = setup(dims, kind, eps, m0, c_sw, 101)
    psi = syn.gaussian_spinors(dims, nrhs, 600 + nrhs)
    src = psi if op == lq.OP_FULL else oracle.split_parity(psi, 1)
    src_r = _bf16_round(src)
    ref = (oracle.apply_D(U, src_r, m0, C if c_sw else None) if op == lq.OP_FULL
           else oracle.apply_schur(U, A, Ainv, src_r))
    d_in = torch.from_numpy(np.ascontiguousarray(src)).to(torch.complex64).cuda()
    d_out = torch.empty_like(d_in)
    lat.apply(op, nrhs, d_in, d_out, dtype=lq.BF16S)
    torch.cuda.synchronize()
    assert relerr(d_out.cpu().numpy(), ref) < TOL[lq.C64]


@pytest.mark.parametrize("nvec,nrhs", [(5, 3), (17, 12), (32, 16), (3, 2), (12, 6), (9, 40), (33, 64), (24, 64),
                                       (1, 1), (23, 7)])
def test_orthogonalise_bf16_basis(nvec, nrhs):
    """BF16-stored basis, complex64 w: h = V^H w and w' = (1 - V V^H) w with V the BF16-rounded basis."""
    lat, *_ = setup((4, 4, 4, 4), "exp", 0.3, -0.2, 1.0, 101)
    n_sites = lat.V // 2
    rng = np.random.default_rng(nvec * 7 + nrhs)
    N = n_sites * 12
    Vb = np.empty((nvec, nrhs, N), complex)
    for r in range(nrhs):
        Z = rng.standard_normal((N, nvec)) + 1j * rng.standard_normal((N, nvec))
        Q, _ = np.linalg.qr(Z)
        Vb[:, r, :] = Q.T
    Vb = _bf16_round(Vb)
    w = (rng.standard_normal((nrhs, N)) + 1j * rng.standard_normal((nrhs, N))).astype(np.complex64).astype(complex)
    # the projection with a not exactly orthonormal basis, as the kernels compute it (CGS2)
    h1 = np.einsum("irn,rn->ir", Vb.conj(), w)
    w1 = w - np.einsum("irn,ir->rn", Vb, h1)
    h2 = np.einsum("irn,rn->ir", Vb.conj(), w1)
    w2 = w1 - np.einsum("irn,ir->rn", Vb, h2)
    basis = torch.cat([lat.packed_empty(lq.BF16S, lq.SITES_ODD, nrhs) for _ in range(nvec)])
    nb = basis.numel() // nvec
    for i in range(nvec):
        src = torch.from_numpy(Vb[i].reshape(nrhs, n_sites, 4, 3)).to(torch.complex64).cuda()
        lat.pack(lq.SITES_ODD, nrhs, src, basis[i * nb:(i + 1) * nb], dtype=lq.BF16S)
    wp = lat.packed_empty(lq.C64, lq.SITES_ODD, nrhs)
    lat.pack(lq.SITES_ODD, nrhs, dev(w.reshape(nrhs, n_sites, 4, 3), lq.C64), wp)
    h = torch.empty((nvec, nrhs), dtype=torch.complex128, device="cuda")
    hn = torch.empty(nrhs, dtype=torch.float64, device="cuda")
    lat.orthogonalise(lq.SITES_ODD, nrhs, nvec, basis, wp, h, hn, reorth=True, dtype=lq.BF16S)
    wout = torch.empty((nrhs, n_sites, 4, 3), dtype=torch.complex64, device="cuda")
    lat.unpack(lq.SITES_ODD, nrhs, wp, wout)
    torch.cuda.synchronize()
    assert np.max(np.abs(h.cpu().numpy() - (h1 + h2))) < 2e-5 * np.max(np.abs(h1))
    assert relerr(wout.cpu().numpy().reshape(nrhs, N), w2) < 1e-5


def _bf16_link_rows(U):
    """The links the BF16 two-row storage represents: rows 0 and 1 of every U_mu(x) rounded to
    BF16 (through FP32, as the library rounds its FP32 copy), row 2 rebuilt as conj(row0 x row1)
    in FP64 (an SU(3) matrix's third row)."""
    Ur = _bf16_round(U)
    Ur[..., 2, :] = np.conj(np.cross(Ur[..., 0, :], Ur[..., 1, :]))
    return Ur


@pytest.mark.parametrize("case", CASES[:3])
@pytest.mark.parametrize("op", [lq.OP_FULL, lq.OP_SCHUR])
@pytest.mark.parametrize("nrhs", [1, 3, 4, 16])
def test_bf16_link_storage_operator(case, op, nrhs):
    """The FP32 operator with BF16 two-row link storage equals the oracle's operator on the links it
    represents (hopping term on the rounded links, clover blocks from the exact ones), to the FP32
    tolerance; and it differs from the FP32-link operator (the rounding is real)."""
    dims, kind, eps, m0, c_sw = case
    lat, U, C, A, Ainv = setup(dims, kind, eps, m0, c_sw, 101)
    Ur = _bf16_link_rows(U)
    psi = syn.gaussian_spinors(dims, nrhs, 800 + nrhs)
    src = psi if op == lq.OP_FULL else oracle.split_parity(psi, 1)
    ref = (oracle.apply_D(Ur, src, m0, C if c_sw else None) if op == lq.OP_FULL
           else oracle.apply_schur(Ur, A, Ainv, src))
    exact = (oracle.apply_D(U, src, m0, C if c_sw else None) if op == lq.OP_FULL
             else oracle.apply_schur(U, A, Ainv, src))
    d_in = dev(src, lq.C64)
    d_out = torch.empty_like(d_in)
    lat.set_link_storage(lq.LINKS_BF16)
    try:
        assert lat.link_storage() == lq.LINKS_BF16
        lat.apply(op, nrhs, d_in, d_out)
        torch.cuda.synchronize()
    finally:
        lat.set_link_storage(lq.LINKS_FP32)
    got = d_out.cpu().numpy()
    assert relerr(got, ref) < TOL[lq.C64]
    assert relerr(got, exact) > 1e-4


@pytest.mark.parametrize("nrhs", [4, 16])
def test_bf16_spinors_and_links_operator(nrhs):
    """BF16-stored input and BF16 two-row links together (the operator of the BF16-basis solve with
    BF16 links): the oracle on the rounded input and the rounded links."""
    dims, kind, eps, m0, c_sw = CASES[0]
    lat, U, C, A, Ainv = setup(dims, kind, eps, m0, c_sw, 101)
    Ur = _bf16_link_rows(U)
    psi_o = oracle.split_parity(syn.gaussian_spinors(dims, nrhs, 900 + nrhs), 1)
    ref = oracle.apply_schur(Ur, A, Ainv, _bf16_round(psi_o))
    d_in = torch.from_numpy(np.ascontiguousarray(psi_o)).to(torch.complex64).cuda()
    d_out = torch.empty_like(d_in)
    lat.set_link_storage(lq.LINKS_BF16)
    try:
        lat.apply(lq.OP_SCHUR, nrhs, d_in, d_out, dtype=lq.BF16S)
        torch.cuda.synchronize()
    finally:
        lat.set_link_storage(lq.LINKS_FP32)
    assert relerr(d_out.cpu().numpy(), ref) < TOL[lq.C64]


def test_two_row_variants_read_fewer_link_bytes():
    """The autotuner's two-row FP32 link variants report 12 reals per link, the others 18."""
    lat, *_ = setup(*CASES[0][:5], 101)
    lib = lq.load()
    reals = [lat.variant_link_reals(lq.C64, v) for v in range(lib.lqcd_kernel_variant_count(lq.C64))]
    assert set(reals) == {12, 18} and reals.count(12) >= 4
    assert all(lat.variant_link_reals(lq.C128, v) == 18 for v in range(lib.lqcd_kernel_variant_count(lq.C128)))


@pytest.mark.parametrize("dtype", [lq.C64, lq.C128])
@pytest.mark.parametrize("nrhs", [100, 256])
def test_maximum_and_ragged_large_nrhs(dtype, nrhs):
    """The largest rhs count an apply takes (256) and a large count that is no power of two (100): the
    default launch and the tuned one, full and Schur, against the oracle."""
    dims, kind, eps, m0, c_sw = CASES[0]
    lat, U, C, A, Ainv = setup(dims, kind, eps, m0, c_sw, 101)
    psi = syn.gaussian_spinors(dims, nrhs, 1000 + nrhs)
    psi_o = oracle.split_parity(psi, 1)
    ref_f = oracle.apply_D(U, psi, m0, C)
    ref_s = oracle.apply_schur(U, A, Ainv, psi_o)
    for tuned in (False, True):
        if tuned:
            lat.tune(dtype, nrhs, reps=1)
        for op, src, ref in ((lq.OP_FULL, psi, ref_f), (lq.OP_SCHUR, psi_o, ref_s)):
            d_in = dev(src, dtype)
            d_out = torch.empty_like(d_in)
            lat.apply(op, nrhs, d_in, d_out)
            torch.cuda.synchronize()
            assert relerr(d_out.cpu().numpy(), ref) < TOL[dtype], (op, tuned, lat.kernel_variant(dtype, nrhs, op))
    for op in (lq.OP_FULL, lq.OP_SCHUR):
        lat.set_kernel_variant(dtype, nrhs, op, -1)
