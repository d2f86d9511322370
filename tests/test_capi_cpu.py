"""CPU checks of the C ABI library: it builds for sm_103a, loads, exports every
symbol declared in include/lqcd.h, and rejects bad arguments on the host
(no CUDA compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_05816_gb300 import _build
    import paper_2601_05816_gb300 as lq
    _build.build()
    return lq.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for need in ("lqcd_create", "lqcd_free", "lqcd_set_gauge", "lqcd_set_clover", "lqcd_apply",
                 "lqcd_apply_packed", "lqcd_solve", "lqcd_schur_prepare", "lqcd_schur_reconstruct",
                 "lqcd_orthogonalise", "lqcd_pack", "lqcd_unpack"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, f"liblqcd.so lacks {missing}"


def test_host_side_argument_errors(lib):
    import paper_2601_05816_gb300 as lq
    h = ctypes.c_void_p()
    odd = (ctypes.c_int * 4)(4, 4, 3, 4)
    assert lib.lqcd_create(odd, -1, ctypes.byref(h)) == lq.ERR_ARG
    assert b"not even" in lib.lqcd_last_error()
    assert lib.lqcd_create((ctypes.c_int * 4)(4, 4, 4, 4), 0, ctypes.byref(h)) == lq.ERR_ARG
    assert lib.lqcd_create((ctypes.c_int * 4)(4, 4, 4, 4), -1, ctypes.byref(h)) == lq.OK
    # operator use before the gauge field is set is refused on the host
    buf = ctypes.c_void_p(16)
    assert lib.lqcd_apply_packed(h, lq.OP_FULL, lq.C64, 4, buf, buf, None) == lq.ERR_STATE
    assert lib.lqcd_set_clover(h, 0.1, 1.0, None) == lq.ERR_STATE
    assert lib.lqcd_packed_bytes(h, lq.C64, lq.SITES_ODD, 3) == 128 * 12 * 3 * 8
    assert lib.lqcd_packed_bytes(h, 7, lq.SITES_ODD, 3) == 0
    assert lib.lqcd_site_tile(h, 1) == 16 and lib.lqcd_site_tile(h, 12) == 2 and lib.lqcd_site_tile(h, 16) == 1
    assert lib.lqcd_status_string(lq.ERR_SINGULAR) == b"singular site block"
    # force: bad sizes and null pointers are argument errors, a missing gauge field a state error
    assert lib.lqcd_force(h, 0, buf, buf, buf, None) == lq.ERR_ARG
    assert lib.lqcd_force(h, 2, None, buf, buf, None) == lq.ERR_ARG
    assert lib.lqcd_force(h, 2, buf, buf, buf, None) == lq.ERR_STATE
    # Gram-Schmidt step: basis sizes 1..64, BF16 storage needs nrhs <= 32 or even nrhs <= 64
    hv = ctypes.c_void_p(32)
    assert lib.lqcd_orthogonalise(h, lq.C64, lq.SITES_ODD, 4, 0, buf, buf, hv, hv, 1, None) == lq.ERR_ARG
    assert lib.lqcd_orthogonalise(h, lq.C64, lq.SITES_ODD, 4, 65, buf, buf, hv, hv, 1, None) == lq.ERR_ARG
    assert lib.lqcd_orthogonalise(h, lq.BF16S, lq.SITES_ODD, 33, 4, buf, buf, hv, hv, 1, None) == lq.ERR_ARG
    assert lib.lqcd_orthogonalise(h, lq.BF16S, lq.SITES_ODD, 66, 4, buf, buf, hv, hv, 1, None) == lq.ERR_ARG
    # batch: empty batch, a lattice listed twice
    ctxs = (ctypes.c_void_p * 2)(h.value, h.value)
    params = (lq.SolveParams * 2)()
    nr = (ctypes.c_int * 2)(1, 1)
    ptrs = (ctypes.c_void_p * 2)(16, 16)
    assert lib.lqcd_solve_batch(0, ctxs, params, nr, ptrs, ptrs, None, None) == lq.ERR_ARG
    assert lib.lqcd_solve_batch(2, ctxs, params, nr, ptrs, ptrs, None, None) == lq.ERR_ARG
    assert b"twice" in lib.lqcd_last_error()
    assert lib.lqcd_free(h) == lq.OK
    assert lib.lqcd_free(None) == lq.OK


def test_link_storage_variant_query_and_probe_arguments(lib):
    """The link-storage switch, the variant link query and the FMA probe check their arguments on the host."""
    import paper_2601_05816_gb300 as lq
    h = ctypes.c_void_p()
    assert lib.lqcd_create((ctypes.c_int * 4)(4, 4, 4, 4), -1, ctypes.byref(h)) == lq.OK
    assert lib.lqcd_get_link_storage(h) == lq.LINKS_FP32
    assert lib.lqcd_set_link_storage(h, 7) == lq.ERR_ARG
    assert lib.lqcd_set_link_storage(h, lq.LINKS_BF16) == lq.OK
    assert lib.lqcd_get_link_storage(h) == lq.LINKS_BF16
    assert lib.lqcd_set_link_storage(None, lq.LINKS_BF16) == lq.ERR_ARG
    assert lib.lqcd_get_link_storage(None) == -1
    n32 = lib.lqcd_kernel_variant_count(lq.C64)
    reals = [lib.lqcd_kernel_variant_link_reals(lq.C64, v) for v in range(n32)]
    assert set(reals) == {12, 18}
    assert lib.lqcd_kernel_variant_link_reals(lq.C64, n32) == -1
    assert lib.lqcd_kernel_variant_link_reals(9, 0) == -1
    assert lib.lqcd_fma_peak(1, None, None) == lq.ERR_ARG
    # the shape query agrees with the link query and marks the blocked-row variants
    shapes = [lq.variant_shape(lq.C64, v) for v in range(n32)]
    assert [sh["link_reals"] for sh in shapes] == reals
    blocked = [sh for sh in shapes if sh["order"] == 1]
    assert blocked and all(sh["ring_warps"] == 0 and sh["stages"] == 0 and sh["nrhs_fixed"] > 0 for sh in blocked)
    assert all(sh["order"] == 0 for sh in (lq.variant_shape(lq.C128, v)
                                           for v in range(lib.lqcd_kernel_variant_count(lq.C128))))
    assert lib.lqcd_kernel_variant_shape(lq.C64, n32, (ctypes.c_int * 11)()) == lq.ERR_ARG
    piped = [sh for sh in shapes if sh["pipe"] > 0]
    assert piped and all(sh["nrhs_fixed"] in (16, 32, 64) and sh["nr"] == 2 for sh in piped)
    assert lib.lqcd_kernel_variant_shape(lq.C64, 0, None) == lq.ERR_ARG
    # block GMRES on a batch is refused before any device work
    ctxs = (ctypes.c_void_p * 1)(h.value)
    params = (lq.SolveParams * 1)()
    params[0].block = 1
    nr = (ctypes.c_int * 1)(2)
    ptrs = (ctypes.c_void_p * 1)(16)
    assert lib.lqcd_solve_batch(1, ctxs, params, nr, ptrs, ptrs, None, None) == lq.ERR_ARG
    assert b"block" in lib.lqcd_last_error()
    assert lib.lqcd_free(h) == lq.OK
