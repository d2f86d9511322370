"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module draws random numbers and builds SU(3) gauge fields and Gaussian
sources. It holds none of the Dirac-operator or solver arithmetic: it only
produces inputs, and both the CUDA path and the CPU oracle consume them.

Canonical layouts (the ones the C ABI takes at its boundary):

* dims = (T, Z, Y, X); direction mu = 0, 1, 2, 3 is t, z, y, x. Site number
  ((t*Z + z)*Y + y)*X + x, i.e. the last coordinate runs fastest (the paper's
  positional numbering of Sec. III-A-1 with the strides read as N1*N2*N3,
  N2*N3, N3, 1).
* gauge field U: complex128 array [T, Z, Y, X, 4, 3, 3]; U[..., mu, a, b] is
  row a, column b of U_mu(x) (row-major 3x3, Sec. III-A-1).
* spinor block: complex128 array [nrhs, T, Z, Y, X, 4, 3] (spin, colour); the
  rhs index is outermost, each rhs a column of the block vector of Eq. (1).

Generators (all numpy ``Generator(PCG64(seed))``):

* ``haar_su3``: QR of a 3x3 complex Gaussian, columns rephased by the phases of
  R's diagonal (Haar on U(3)), then divided by a cube root of the determinant
  (a centre-invariant choice, so the result is Haar on SU(3)).
* ``exp_su3``: U = exp(i eps H) with H = sum_a h_a lambda_a / 2 over the eight
  Gell-Mann matrices, h_a ~ N(0, 1) independently per link. The exponential is
  a scaling-and-squaring Taylor series accurate to ~1e-15, then the matrix is
  re-unitarised (rows orthonormalised, third row = conj(row0 x row1)), so every
  link is in SU(3) to rounding.
* ``gaussian_spinors``: real and imaginary parts ~ N(0, 1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "lattice_volume", "haar_su3", "exp_su3", "gauge_field", "gaussian_spinors",
    "random_gauge_transform", "unit_gauge", "rng",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def lattice_volume(dims) -> int:
    T, Z, Y, X = (int(d) for d in dims)
    return T * Z * Y * X


def _gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return lam


def _cm_matmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Product of two stacks of 3x3 matrices stored component-major [3, 3, N]."""
    out = np.empty_like(a)
    for i in range(3):
        for k in range(3):
            out[i, k] = a[i, 0] * b[0, k] + a[i, 1] * b[1, k] + a[i, 2] * b[2, k]
    return out


def _reunitarise_cm(m: np.ndarray) -> np.ndarray:
    """Project a stack of near-SU(3) matrices [3, 3, N] onto SU(3)."""
    r0 = m[0].copy()
    r0 /= np.sqrt(np.sum(np.abs(r0) ** 2, axis=0))
    r1 = m[1] - np.sum(np.conj(r0) * m[1], axis=0) * r0
    r1 /= np.sqrt(np.sum(np.abs(r1) ** 2, axis=0))
    r2 = np.conj(np.stack([r0[1] * r1[2] - r0[2] * r1[1],
                           r0[2] * r1[0] - r0[0] * r1[2],
                           r0[0] * r1[1] - r0[1] * r1[0]]))
    return np.stack([r0, r1, r2])


def _exp_chunk(h: np.ndarray, eps: float, lam: np.ndarray) -> np.ndarray:
    """exp(i eps H) for one chunk of Gell-Mann coefficient rows h [m, 8]; returns [m, 3, 3]."""
    # X = i eps H, component-major [3, 3, m]
    H = np.einsum("na,aij->ijn", h, lam) * 0.5
    X = 1j * eps * H
    norm = float(np.sqrt(np.max(np.sum(np.abs(X) ** 2, axis=(0, 1))))) if X.shape[2] else 0.0
    sq = max(0, int(np.ceil(np.log2(max(norm, 1e-300) / 0.25))))
    Xs = X / (2.0 ** sq)
    eye = np.zeros_like(Xs)
    for i in range(3):
        eye[i, i] = 1.0
    # Horner form of the degree-12 Taylor polynomial: |Xs| <= 1/4 gives < 1e-17.
    E = eye.copy()
    for k in range(12, 0, -1):
        E = eye + _cm_matmul(Xs, E) / k
    for _ in range(sq):
        E = _cm_matmul(E, E)
    E = _reunitarise_cm(E)
    return np.transpose(E, (2, 0, 1))


def exp_su3(g: np.random.Generator, n: int, eps: float, chunk: int = 1 << 20) -> np.ndarray:
    """n links U = exp(i eps H), H Gaussian traceless Hermitian; returns [n, 3, 3].

    The random numbers are drawn in one call; the chunks of 2^20 links are then
    exponentiated independently (on a few threads for large fields: numpy releases
    the interpreter lock inside its array operations), so the result does not
    depend on the thread count."""
    lam = _gell_mann()
    out = np.empty((n, 3, 3), dtype=np.complex128)
    h_all = g.standard_normal((n, 8))
    starts = list(range(0, n, chunk))

    def work(s):
        out[s:s + chunk] = _exp_chunk(h_all[s:s + chunk], eps, lam)

    if len(starts) > 2:
        import concurrent.futures as cf
        import os
        with cf.ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1, 16)) as ex:
            list(ex.map(work, starts))
    else:
        for s in starts:
            work(s)
    return out


def haar_su3(g: np.random.Generator, n: int) -> np.ndarray:
    """n Haar-random SU(3) matrices, [n, 3, 3]."""
    z = (g.standard_normal((n, 3, 3)) + 1j * g.standard_normal((n, 3, 3))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q * (det ** (-1.0 / 3.0))[:, None, None]
    return q


def gauge_field(dims, kind: str = "haar", eps: float = 0.0, seed: int = 0) -> np.ndarray:
    """Gauge field [T, Z, Y, X, 4, 3, 3] complex128, links drawn independently per (site, mu)."""
    T, Z, Y, X = (int(d) for d in dims)
    n = T * Z * Y * X * 4
    g = rng(seed)
    if kind == "haar":
        links = haar_su3(g, n)
    elif kind == "exp":
        links = exp_su3(g, n, float(eps))
    elif kind == "unit":
        links = np.broadcast_to(np.eye(3, dtype=np.complex128), (n, 3, 3)).copy()
    else:
        raise ValueError(f"unknown gauge kind {kind!r}")
    return links.reshape(T, Z, Y, X, 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    return gauge_field(dims, kind="unit")


def gaussian_spinors(dims, nrhs: int, seed: int) -> np.ndarray:
    """nrhs Gaussian sources [nrhs, T, Z, Y, X, 4, 3] complex128."""
    T, Z, Y, X = (int(d) for d in dims)
    g = rng(seed)
    shape = (int(nrhs), T, Z, Y, X, 4, 3)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """Haar-random g(x) in SU(3) per site, [T, Z, Y, X, 3, 3]."""
    T, Z, Y, X = (int(d) for d in dims)
    return haar_su3(rng(seed), T * Z * Y * X).reshape(T, Z, Y, X, 3, 3)
