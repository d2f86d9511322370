"""The allocation-free Schur apply gives the same result as the regular one.

lqcd_apply_schur_noalloc is meant for callers that cannot let the library
allocate device memory during their run (their own allocator owns the memory,
or their footprint must be fixed in advance, or their loop cannot take the
synchronisation of a cudaMalloc). It keeps its intermediate block in a fixed
device array instead of workspace. This test calls it through the C ABI twice
in a row and compares each output with lqcd_apply_packed(LQCD_OP_SCHUR) and with
the FP64 oracle's Schur operator within the operator tolerances of the other GPU
tests (FP64 1e-12, FP32 5e-6); checks on a fresh lattice context, before any
other apply on it, that the call leaves the device's free memory unchanged (no
workspace allocated); and checks that a request larger than the fixed array or a
call with another device current is refused on the host. The file name makes
pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synthetic as syn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_05816_gb300 as lq  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    from paper_2601_05816_gb300 import _build
    _build.build()
    L = lq.load()
    L.lqcd_apply_schur_noalloc.restype = ctypes.c_int
    L.lqcd_apply_schur_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]
    L.lqcd_noalloc_scratch_bytes.restype = ctypes.c_size_t
    L.lqcd_noalloc_scratch_bytes.argtypes = []
    return L


@pytest.mark.parametrize("dtype,tol", [(lq.C64, 5e-6), (lq.C128, 1e-12)])
def test_noalloc_schur_matches_regular_apply_twice(lib, dtype, tol):
    dims = (8, 8, 8, 8)
    nrhs = 6
    U = syn.gauge_field(dims, "exp", 0.3, seed=31)
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(-0.2, 1.0)
    A, Ainv = oracle.diag_blocks(U, -0.2, 1.0)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        psi = syn.gaussian_spinors((8, 8, 8, 4), nrhs, 40 + call).reshape(nrhs, lat.V // 2, 4, 3)
        t = torch.from_numpy(psi).cuda()
        t = t if dtype == lq.C128 else t.to(torch.complex64)
        pin = lat.packed_empty(dtype, lq.SITES_ODD, nrhs)
        lat.pack(lq.SITES_ODD, nrhs, t, pin)
        ref = lat.packed_empty(dtype, lq.SITES_ODD, nrhs)
        lat.apply_packed(lq.OP_SCHUR, nrhs, pin, ref)
        got = lat.packed_empty(dtype, lq.SITES_ODD, nrhs)
        got.fill_(float("nan"))
        st = lib.lqcd_apply_schur_noalloc(lat.handle, dtype, nrhs, pin.data_ptr(), got.data_ptr(), stream)
        assert st == lq.OK, lib.lqcd_last_error()
        torch.cuda.synchronize()
        g = got.cpu().numpy().astype(np.complex128).reshape(-1, nrhs)
        r = ref.cpu().numpy().astype(np.complex128).reshape(-1, nrhs)
        err = max(np.linalg.norm(g[:, k] - r[:, k]) / np.linalg.norm(r[:, k]) for k in range(nrhs))
        assert err <= tol, (call, err)
        # and the oracle's S psi_o on the same (rounded) input
        ref_o = oracle.apply_schur(U, A, Ainv, t.cpu().numpy().astype(np.complex128))
        out = torch.empty_like(t)
        lat.unpack(lq.SITES_ODD, nrhs, got, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.complex128).reshape(nrhs, -1)
        ro = ref_o.reshape(nrhs, -1)
        err_o = max(np.linalg.norm(o[k] - ro[k]) / np.linalg.norm(ro[k]) for k in range(nrhs))
        assert err_o <= tol, (call, err_o)
    lat.close()


def test_noalloc_allocates_nothing_on_a_fresh_context(lib):
    """A fresh lattice context that has never applied an operator: the no-alloc Schur apply leaves
    the device's free memory unchanged (the regular apply would allocate its workspace here). One
    earlier call on another context loads the library's scratch array first (CUDA loads a module's
    device globals when the module is first used)."""
    dims = (16, 8, 8, 8)
    nrhs = 8    # the regular apply's intermediate block: V/2 * 12 * 8 * 8 bytes = 3.1 MB
    U = syn.gauge_field(dims, "exp", 0.3, seed=32)
    stream = torch.cuda.current_stream().cuda_stream
    warm = lq.Lattice(dims)
    warm.set_gauge(torch.from_numpy(U).cuda())
    warm.set_clover(-0.2, 1.0)
    a = warm.packed_empty(lq.C64, lq.SITES_ODD, nrhs)
    a.zero_()
    b = torch.empty_like(a)
    assert lib.lqcd_apply_schur_noalloc(warm.handle, lq.C64, nrhs, a.data_ptr(), b.data_ptr(), stream) == lq.OK
    torch.cuda.synchronize()
    lat = lq.Lattice(dims)
    lat.set_gauge(torch.from_numpy(U).cuda())
    lat.set_clover(-0.2, 1.0)
    pin = lat.packed_empty(lq.C64, lq.SITES_ODD, nrhs)
    pin.normal_()
    pout = torch.empty_like(pin)
    ref = torch.empty_like(pin)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        st = lib.lqcd_apply_schur_noalloc(lat.handle, lq.C64, nrhs, pin.data_ptr(), pout.data_ptr(), stream)
        assert st == lq.OK, lib.lqcd_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # the regular apply on the same fresh context does allocate its workspace (the check has teeth)
    lat.apply_packed(lq.OP_SCHUR, nrhs, pin, ref)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free0
    assert torch.allclose(ref, pout, rtol=0, atol=1e-5 * float(ref.abs().max()))
    lat.close()
    warm.close()


def test_noalloc_rejects_oversized_request(lib):
    dims = (16, 16, 16, 16)
    lat = lq.Lattice(dims)
    lat.set_gauge(syn.gauge_field(dims, "unit"))
    lat.set_clover(0.1, 0.0)
    nrhs = 64   # V/2 * 12 * 64 * 16 bytes = 402 MB > the fixed scratch
    assert (lat.V // 2) * 12 * nrhs * 16 > lib.lqcd_noalloc_scratch_bytes()
    dummy = torch.empty(16, dtype=torch.complex128, device="cuda")
    st = lib.lqcd_apply_schur_noalloc(lat.handle, lq.C128, nrhs, dummy.data_ptr(), dummy.data_ptr() + 256,
                                      torch.cuda.current_stream().cuda_stream)
    assert st == lq.ERR_ARG
    assert b"scratch" in lib.lqcd_last_error()
    lat.close()
