"""Python binding of liblqcd.so: the GB300 multi-rhs Wilson(-clover) operator and batched GMRES.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/lqcd.h``. PyTorch provides device
memory and the current CUDA stream; tensors are passed by ``data_ptr()``.
There is no CPU fallback: if the library is missing or cannot be loaded the
calls raise ``LqcdError``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblqcd.so")

# status codes and enums (include/lqcd.h)
OK, NOT_CONVERGED = 0, 1
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_SINGULAR, ERR_STATE = -1, -2, -3, -4, -5, -6
C64, C128, BF16S = 1, 2, 3
OP_FULL, OP_SCHUR = 0, 1
LINKS_FP32, LINKS_BF16 = 0, 1
SITES_FULL, SITES_EVEN, SITES_ODD = 0, 1, 2

_lib = None


class LqcdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


class SolveParams(ctypes.Structure):
    _fields_ = [
        ("op", ctypes.c_int), ("precision", ctypes.c_int), ("restart_len", ctypes.c_int),
        ("max_restarts", ctypes.c_int), ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
        ("x0_given", ctypes.c_int), ("use_graph", ctypes.c_int), ("reorth", ctypes.c_int),
        ("profile", ctypes.c_int), ("dagger", ctypes.c_int), ("compact", ctypes.c_int),
        ("block", ctypes.c_int),
    ]


class SolveStats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("restarts", ctypes.c_int), ("iterations", ctypes.c_int),
        ("seconds", ctypes.c_double), ("relres_max", ctypes.c_double),
        ("op_ms", ctypes.c_double), ("op_launches", ctypes.c_int), ("op_bytes", ctypes.c_double),
        ("ortho_ms", ctypes.c_double), ("ortho_launches", ctypes.c_int), ("ortho_bytes", ctypes.c_double),
        ("kernel_launches", ctypes.c_longlong),
        ("iters_per_rhs", ctypes.POINTER(ctypes.c_int)),
        ("relres_per_rhs", ctypes.POINTER(ctypes.c_double)),
        ("outer_steps", ctypes.c_int), ("ortho", ctypes.c_int),
    ]


_VP, _I, _D, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_SIGS = {
    "lqcd_status_string": (ctypes.c_char_p, [_I]),
    "lqcd_last_error": (ctypes.c_char_p, []),
    "lqcd_create": (_I, [ctypes.POINTER(ctypes.c_int), _I, ctypes.POINTER(_VP)]),
    "lqcd_free": (_I, [_VP]),
    "lqcd_set_gauge": (_I, [_VP, _VP, _VP]),
    "lqcd_set_clover": (_I, [_VP, _D, _D, _VP]),
    "lqcd_export_blocks": (_I, [_VP, _I, _VP, _VP]),
    "lqcd_site_tile": (_I, [_VP, _I]),
    "lqcd_packed_bytes": (_SZ, [_VP, _I, _I, _I]),
    "lqcd_pack": (_I, [_VP, _I, _I, _I, _VP, _VP, _VP]),
    "lqcd_unpack": (_I, [_VP, _I, _I, _I, _VP, _VP, _VP]),
    "lqcd_apply_packed": (_I, [_VP, _I, _I, _I, _VP, _VP, _VP]),
    "lqcd_apply": (_I, [_VP, _I, _I, _I, _VP, _VP, _VP]),
    "lqcd_schur_prepare": (_I, [_VP, _I, _I, _VP, _VP, _VP]),
    "lqcd_schur_reconstruct": (_I, [_VP, _I, _I, _VP, _VP, _VP, _VP]),
    "lqcd_orthogonalise": (_I, [_VP, _I, _I, _I, _I, _VP, _VP, _VP, _VP, _I, _VP]),
    "lqcd_solve": (_I, [_VP, ctypes.POINTER(SolveParams), _I, _VP, _VP, ctypes.POINTER(SolveStats), _VP]),
    "lqcd_force": (_I, [_VP, _I, _VP, _VP, _VP, _VP]),
    "lqcd_tune": (_I, [_VP, _I, _I, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), _VP]),
    "lqcd_solve_batch": (_I, [_I, ctypes.POINTER(_VP), ctypes.POINTER(SolveParams), ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(SolveStats), _VP]),
    "lqcd_kernel_variant_count": (_I, [_I]),
    "lqcd_get_kernel_variant": (_I, [_VP, _I, _I, _I]),
    "lqcd_set_kernel_variant": (_I, [_VP, _I, _I, _I, _I]),
    "lqcd_set_link_storage": (_I, [_VP, _I]),
    "lqcd_fma_peak": (_I, [_I, ctypes.POINTER(ctypes.c_double), _VP]),
    "lqcd_kernel_variant_link_reals": (_I, [_I, _I]),
    "lqcd_kernel_variant_shape": (_I, [_I, _I, ctypes.POINTER(ctypes.c_int)]),
    "lqcd_get_link_storage": (_I, [_VP]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblqcd.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LqcdError(ERR_STATE, f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, what: str) -> int:
    if status < 0:
        msg = load().lqcd_last_error().decode(errors="replace")
        raise LqcdError(status, f"{what}: {msg}")
    return status


def _stream(stream=None) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t) -> int:
    import torch
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise LqcdError(ERR_ARG, "tensor must be contiguous")
        return int(t.data_ptr())
    import numpy as np
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise LqcdError(ERR_ARG, "array must be C-contiguous")
        return int(t.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(t)}")


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.complex64:
        return C64
    if t.dtype == torch.complex128:
        return C128
    raise LqcdError(ERR_ARG, f"unsupported dtype {t.dtype}")


@dataclass
class SolveResult:
    status: int
    restarts: int
    iterations: int
    seconds: float
    relres_max: float
    op_ms: float
    op_launches: int
    op_bytes: float
    ortho_ms: float
    ortho_launches: int
    ortho_bytes: float
    kernel_launches: int
    iters_per_rhs: list
    relres_per_rhs: list
    outer_steps: int = 0
    ortho: int = -1      # Gram-Schmidt that ran: 0 CGS1, 1 CGS2, 2 delayed CGS2


class Lattice:
    """A lattice context: gauge field, clover blocks and library workspace.

    dims = (T, Z, Y, X), all even; time_bc = -1 (antiperiodic) or +1.
    """

    def __init__(self, dims, time_bc: int = -1):
        lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.V = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        arr = (ctypes.c_int * 4)(*self.dims)
        h = ctypes.c_void_p()
        _check(lib.lqcd_create(arr, int(time_bc), ctypes.byref(h)), "lqcd_create")
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lqcd_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_gauge(self, U, stream=None):
        """U: complex128 [V][4][3][3] (any shape with that memory layout), torch CUDA tensor or numpy."""
        _check(self._lib.lqcd_set_gauge(self._h, _ptr(U), _stream(stream)), "lqcd_set_gauge")

    def set_clover(self, m0: float, c_sw: float, stream=None):
        _check(self._lib.lqcd_set_clover(self._h, float(m0), float(c_sw), _stream(stream)), "lqcd_set_clover")

    def export_blocks(self, which: int, out, stream=None):
        _check(self._lib.lqcd_export_blocks(self._h, int(which), _ptr(out), _stream(stream)),
               "lqcd_export_blocks")

    def site_tile(self, nrhs: int) -> int:
        return int(self._lib.lqcd_site_tile(self._h, int(nrhs)))

    def packed_bytes(self, dtype: int, sites: int, nrhs: int) -> int:
        return int(self._lib.lqcd_packed_bytes(self._h, int(dtype), int(sites), int(nrhs)))

    def packed_empty(self, dtype: int, sites: int, nrhs: int):
        """Device buffer for a packed block: complex128 / complex64, or int32 words holding BF16 pairs."""
        import torch
        if dtype == BF16S:
            return torch.empty(self.packed_bytes(dtype, sites, nrhs) // 4, dtype=torch.int32, device="cuda")
        n = self.packed_bytes(dtype, sites, nrhs) // (16 if dtype == C128 else 8)
        return torch.empty(n, dtype=torch.complex128 if dtype == C128 else torch.complex64, device="cuda")

    def pack(self, sites: int, nrhs: int, src, dst, stream=None, dtype=None):
        d = _dtype_code(src) if dtype is None else int(dtype)
        _check(self._lib.lqcd_pack(self._h, d, int(sites), int(nrhs), _ptr(src), _ptr(dst), _stream(stream)),
               "lqcd_pack")

    def unpack(self, sites: int, nrhs: int, src, dst, stream=None, dtype=None):
        d = _dtype_code(dst) if dtype is None else int(dtype)
        _check(self._lib.lqcd_unpack(self._h, d, int(sites), int(nrhs), _ptr(src), _ptr(dst), _stream(stream)),
               "lqcd_unpack")

    def apply_packed(self, op: int, nrhs: int, src, dst, stream=None, dtype=None):
        d = _dtype_code(src) if dtype is None else int(dtype)
        _check(self._lib.lqcd_apply_packed(self._h, int(op), d, int(nrhs), _ptr(src), _ptr(dst), _stream(stream)),
               "lqcd_apply_packed")

    def apply(self, op: int, nrhs: int, src, dst, stream=None, dtype=None):
        d = _dtype_code(src) if dtype is None else int(dtype)
        _check(self._lib.lqcd_apply(self._h, int(op), d, int(nrhs), _ptr(src), _ptr(dst), _stream(stream)),
               "lqcd_apply")

    def schur_prepare(self, nrhs: int, b_full, bhat_o, stream=None):
        _check(self._lib.lqcd_schur_prepare(self._h, _dtype_code(b_full), int(nrhs), _ptr(b_full), _ptr(bhat_o),
                                            _stream(stream)), "lqcd_schur_prepare")

    def schur_reconstruct(self, nrhs: int, b_full, x_o, x_full, stream=None):
        _check(self._lib.lqcd_schur_reconstruct(self._h, _dtype_code(b_full), int(nrhs), _ptr(b_full), _ptr(x_o),
                                                _ptr(x_full), _stream(stream)), "lqcd_schur_reconstruct")

    def orthogonalise(self, sites: int, nrhs: int, nvec: int, basis, w, h, hnorm, reorth: bool = True,
                      stream=None, dtype=None):
        d = _dtype_code(w) if dtype is None else int(dtype)
        _check(self._lib.lqcd_orthogonalise(self._h, d, int(sites), int(nrhs), int(nvec),
                                            _ptr(basis), _ptr(w), _ptr(h), _ptr(hnorm), int(bool(reorth)),
                                            _stream(stream)), "lqcd_orthogonalise")

    def tune(self, dtype: int, nrhs: int, reps: int = 5, stream=None):
        """Autotune the hopping-kernel variant for (dtype, nrhs); returns [(full_ms, schur_ms)] per variant."""
        times = (ctypes.c_double * 256)()
        n = ctypes.c_int(0)
        _check(self._lib.lqcd_tune(self._h, int(dtype), int(nrhs), int(reps), times, ctypes.byref(n),
                                   _stream(stream)), "lqcd_tune")
        return [(times[2 * v], times[2 * v + 1]) for v in range(n.value)]

    def variant_link_reals(self, dtype: int, variant: int) -> int:
        """Reals per link read by a hopping-kernel launch variant (18, or 12 with the third row rebuilt)."""
        return int(self._lib.lqcd_kernel_variant_link_reals(int(dtype), int(variant)))

    def kernel_variant_info(self, dtype: int, variant: int) -> dict:
        """Launch shape of a hopping-kernel variant (rhs per thread, threads, ..., blocked row order)."""
        return variant_shape(dtype, variant)

    def kernel_variant(self, dtype: int, nrhs: int, op: int) -> int:
        return int(self._lib.lqcd_get_kernel_variant(self._h, int(dtype), int(nrhs), int(op)))

    def set_kernel_variant(self, dtype: int, nrhs: int, op: int, variant: int):
        _check(self._lib.lqcd_set_kernel_variant(self._h, int(dtype), int(nrhs), int(op), int(variant)),
               "lqcd_set_kernel_variant")

    def set_link_storage(self, fmt: int):
        """Link storage of the FP32 operator: LINKS_FP32 (default) or LINKS_BF16 (two rows in BF16)."""
        _check(self._lib.lqcd_set_link_storage(self._h, int(fmt)), "lqcd_set_link_storage")

    def link_storage(self) -> int:
        return int(self._lib.lqcd_get_link_storage(self._h))

    def save_tuning(self, path: str, keys):
        """Write the chosen variants for keys = [(dtype, nrhs, op), ...] to a JSON cache."""
        import json
        data = {f"{d},{n},{o}": self.kernel_variant(d, n, o) for (d, n, o) in keys}
        with open(path, "w") as f:
            json.dump({"dims": list(self.dims), "variants": data}, f, indent=1)

    def load_tuning(self, path: str) -> bool:
        """Restore variants from a JSON cache written for the same lattice; False if absent or for other dims."""
        import json
        if not os.path.exists(path):
            return False
        with open(path) as f:
            data = json.load(f)
        if tuple(data.get("dims", ())) != self.dims:
            return False
        for key, v in data["variants"].items():
            d, n, o = (int(t) for t in key.split(","))
            self.set_kernel_variant(d, n, o, int(v))
        return True

    def solve(self, b, x, nrhs: int, *, op: int = OP_SCHUR, precision: int = C64, restart_len: int = 32,
              max_restarts: int = 200, tol: float = 1e-10, inner_tol: float = 0.0, x0_given: bool = False,
              use_graph: bool = True, reorth: int = 2, profile: bool = False, dagger: bool = False,
              compact: bool = True, block: bool = False, stream=None) -> SolveResult:
        """Batched GMRES on D x = b (dagger: D^dagger x = b); b and x complex128 canonical [nrhs][V][4][3],
        host (numpy) or device."""
        p = SolveParams(op, precision, restart_len, max_restarts, tol, inner_tol, int(x0_given), int(use_graph),
                        int(reorth), int(profile), int(dagger), int(compact), int(block))
        # reorth: 0 CGS1, 1 CGS2, 2 delayed CGS2; block: block GMRES inner solver
        its = (ctypes.c_int * nrhs)()
        rel = (ctypes.c_double * nrhs)()
        st = SolveStats()
        st.iters_per_rhs = ctypes.cast(its, ctypes.POINTER(ctypes.c_int))
        st.relres_per_rhs = ctypes.cast(rel, ctypes.POINTER(ctypes.c_double))
        status = _check(self._lib.lqcd_solve(self._h, ctypes.byref(p), int(nrhs), _ptr(b), _ptr(x),
                                             ctypes.byref(st), _stream(stream)), "lqcd_solve")
        return SolveResult(status, st.restarts, st.iterations, st.seconds, st.relres_max, st.op_ms,
                           st.op_launches, st.op_bytes, st.ortho_ms, st.ortho_launches, st.ortho_bytes,
                           st.kernel_launches, list(its), list(rel), st.outer_steps, st.ortho)


    def force(self, nrhs: int, x, lam, grad_U, stream=None) -> None:
        """dL/dU for L = sum_i Re <eta_i, x_i>, x = D^{-1} b, lam = D^{-dagger} eta (lqcd_force): device complex128
        x, lam [nrhs][V][4][3] and grad_U [V][4][3][3] (overwritten)."""
        _check(self._lib.lqcd_force(self._h, int(nrhs), _ptr(x), _ptr(lam), _ptr(grad_U), _stream(stream)),
               "lqcd_force")


def fma_peak(f64: bool, stream=None) -> float:
    """Measured SIMT FMA rate of the current GPU in TFLOP/s (lqcd_fma_peak): FP64 or FP32."""
    v = ctypes.c_double(0.0)
    _check(load().lqcd_fma_peak(int(bool(f64)), ctypes.byref(v), _stream(stream)), "lqcd_fma_peak")
    return float(v.value)


_SHAPE_KEYS = ("nr", "threads", "min_ctas", "stages", "nrhs_fixed", "prefetch", "ring_warps", "ring_slots",
               "link_reals", "order", "pipe")


def variant_shape(dtype: int, variant: int) -> dict:
    """Launch shape of a hopping-kernel variant (lqcd_kernel_variant_shape), keyed by field name."""
    shape = (ctypes.c_int * 11)()
    _check(load().lqcd_kernel_variant_shape(int(dtype), int(variant), shape), "lqcd_kernel_variant_shape")
    return dict(zip(_SHAPE_KEYS, (int(x) for x in shape)))


def solve_batch(lattices, bs, xs, nrhs, *, op: int = OP_SCHUR, precision: int = C64, restart_len: int = 32,
                max_restarts: int = 200, tol=1e-10, inner_tol: float = 0.0, use_graph: bool = True,
                reorth: int = 2, compact: bool = True, stream=None):
    """Batched GMRES over several lattices of uneven size (lqcd_solve_batch); returns one SolveResult each.

    tol may be one value or one per lattice; b and x complex128 canonical per lattice (host or device).
    """
    lib = load()
    n = len(lattices)
    tols = list(tol) if isinstance(tol, (list, tuple)) else [tol] * n
    ctxs = (ctypes.c_void_p * n)(*[lat.handle.value for lat in lattices])
    params = (SolveParams * n)(*[SolveParams(op, precision, restart_len, max_restarts, tols[i], inner_tol, 0,
                                             int(use_graph), int(reorth), 0, 0, int(compact), 0) for i in range(n)])
    nr = (ctypes.c_int * n)(*[int(v) for v in nrhs])
    bp = (ctypes.c_void_p * n)(*[_ptr(v) for v in bs])
    xp = (ctypes.c_void_p * n)(*[_ptr(v) for v in xs])
    stats = (SolveStats * n)()
    per_its = [(ctypes.c_int * int(v))() for v in nrhs]
    per_rel = [(ctypes.c_double * int(v))() for v in nrhs]
    for i in range(n):
        stats[i].iters_per_rhs = ctypes.cast(per_its[i], ctypes.POINTER(ctypes.c_int))
        stats[i].relres_per_rhs = ctypes.cast(per_rel[i], ctypes.POINTER(ctypes.c_double))
    _check(lib.lqcd_solve_batch(n, ctxs, params, nr, bp, xp, stats, _stream(stream)), "lqcd_solve_batch")
    out = []
    for i in range(n):
        st = stats[i]
        out.append(SolveResult(st.status, st.restarts, st.iterations, st.seconds, st.relres_max, st.op_ms,
                               st.op_launches, st.op_bytes, st.ortho_ms, st.ortho_launches, st.ortho_bytes,
                               st.kernel_launches, list(per_its[i]), list(per_rel[i]), st.outer_steps,
                               st.ortho))
    return out


def _autograd_function():
    import torch

    class DiracSolve(torch.autograd.Function):
        """x = D[U]^{-1} b for a block of rhs, differentiable in b and U.

        Backward: the adjoint solve lam = D^{-dagger} g (g the incoming gradient of x; the
        Krylov basis is recomputed, not stored), dL/db = lam and dL/dU from lqcd_force."""

        @staticmethod
        def forward(ctx, b, U, lattice, m0, c_sw, kw):
            lattice.set_gauge(U.detach().contiguous())
            lattice.set_clover(m0, c_sw)
            x = torch.zeros_like(b)
            res = lattice.solve(b.detach().contiguous(), x, b.shape[0], **kw)
            if res.status != OK:
                raise LqcdError(res.status, f"forward solve did not converge: {res}")
            ctx.lattice, ctx.m0, ctx.c_sw, ctx.kw = lattice, m0, c_sw, kw
            ctx.save_for_backward(U, x)
            return x

        @staticmethod
        def backward(ctx, gx):
            U, x = ctx.saved_tensors
            lat = ctx.lattice
            lat.set_gauge(U.detach().contiguous())
            lat.set_clover(ctx.m0, ctx.c_sw)
            g = gx.detach().contiguous()
            lam = torch.zeros_like(g)
            res = lat.solve(g, lam, g.shape[0], dagger=True, **ctx.kw)
            if res.status != OK:
                raise LqcdError(res.status, f"adjoint solve did not converge: {res}")
            gU = None
            if ctx.needs_input_grad[1]:
                gU = torch.empty(U.shape, dtype=U.dtype, device=U.device)
                lat.force(g.shape[0], x, lam, gU)
            return (lam if ctx.needs_input_grad[0] else None), gU, None, None, None, None

    return DiracSolve


_DIRAC_SOLVE = None


def solve_differentiable(lattice, U, b, m0: float, c_sw: float, **solve_kw):
    """x = D^{-1} b (batched GMRES of lqcd_solve) as a torch autograd function of b and U.

    U: device complex128 [V][4][3][3] (canonical), b: device complex128 [nrhs][V][4][3]; solve_kw as for
    Lattice.solve (tol, precision, op, ...). Gradients: dL/db by one adjoint solve, dL/dU by lqcd_force.
    """
    global _DIRAC_SOLVE
    if _DIRAC_SOLVE is None:
        _DIRAC_SOLVE = _autograd_function()
    return _DIRAC_SOLVE.apply(b, U, lattice, float(m0), float(c_sw), dict(solve_kw))
