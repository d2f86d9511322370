"""Brute-force dense Wilson(-clover) matrix on tiny lattices (oracle; test infrastructure only).

Built entry by entry from the definition of Sec. III-A-1 with explicit loops
over sites and directions, explicit coordinate wrap and the explicit time
boundary factor, independently of the array shifts in ``dirac``. Row/column
index 12 * site + 3 * spin + colour, site numbered with the last coordinate
fastest. On a 2^4 lattice x + mu-hat and x - mu-hat are the same site, so both
hopping terms land in the same block and must add.
"""
from __future__ import annotations

import itertools

import numpy as np

from .dirac import gamma_matrices


def dense_operator(U: np.ndarray, m0: float, C: np.ndarray | None = None,
                   bc: float = -1.0) -> np.ndarray:
    dims = U.shape[:4]
    V = int(np.prod(dims))
    D = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    g = gamma_matrices()
    one = np.eye(4, dtype=np.complex128)

    def site(c):
        t, z, y, x = c
        return ((t * dims[1] + z) * dims[2] + y) * dims[3] + x

    for c in itertools.product(*(range(d) for d in dims)):
        i = site(c)
        block = (4.0 + m0) * np.eye(12, dtype=np.complex128)
        if C is not None:
            block = block - C[c]
        D[12 * i:12 * i + 12, 12 * i:12 * i + 12] += block
        for mu in range(4):
            fwd = list(c)
            fwd[mu] = (c[mu] + 1) % dims[mu]
            sign_f = bc if (mu == 0 and c[0] == dims[0] - 1) else 1.0
            j = site(fwd)
            D[12 * i:12 * i + 12, 12 * j:12 * j + 12] += (
                -sign_f * np.kron((one - g[mu]) / 2, U[c][mu]))
            bwd = list(c)
            bwd[mu] = (c[mu] - 1) % dims[mu]
            sign_b = bc if (mu == 0 and c[0] == 0) else 1.0
            k = site(bwd)
            D[12 * i:12 * i + 12, 12 * k:12 * k + 12] += (
                -sign_b * np.kron((one + g[mu]) / 2, U[tuple(bwd)][mu].conj().T))
    return D
