"""Diagnostic run of the oracle (by hand; not part of the tests or the product path).

Two reports about the odd-even GMRES(32) system of the 32^3 x 64 Wilson-clover
workload (U = exp(i 0.25 H), c_sw = 1):

* ``ritz``: the harmonic Ritz values (oracle.spectrum) of the first FP64
  GMRES(32) cycle on the Schur operator S, started from the prepared source
  hat b_o of the workload's first rhs, for one or more bare masses m0. They are
  the roots of the cycle's residual polynomial; small ones mean S is close to
  singular as seen by a 32-step Krylov space.
* ``ladder``: FP64 odd-even GMRES(32) iteration counts to 1e-10 for the same
  gauge generator and mass on growing volumes (capped at a maximum count).

Usage: python -m oracle.report_spectrum ritz [m0 ...]
       python -m oracle.report_spectrum ladder [m0]
Prints one JSON object per result.
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from . import dirac, krylov, spectrum


def _synthetic():
    # the seeded input generators live outside the oracle package (repository root)
    import synthetic as syn
    return syn


def ritz_report(dims, eps, m0_list, gauge_seed, rhs_seed, m=32):
    syn = _synthetic()
    t0 = time.time()
    U = syn.gauge_field(dims, "exp", eps, seed=gauge_seed)
    b = syn.gaussian_spinors(dims, 1, rhs_seed)
    b_e, b_o = dirac.split_parity(b, 0), dirac.split_parity(b, 1)
    for m0 in m0_list:
        A, Ainv = dirac.diag_blocks(U, m0, 1.0)
        bhat = dirac.schur_prepare(U, Ainv, b_e, b_o)
        shape = bhat.shape

        def S(v):
            return dirac.apply_schur(U, A, Ainv, v.reshape(shape)).ravel()

        V, H = spectrum.arnoldi(S, bhat.ravel(), m)
        hr = spectrum.harmonic_ritz(H)
        rz = spectrum.ritz(H)
        # GMRES residual reduction of this first cycle: min ||beta e1 - H y|| / beta
        beta = float(np.linalg.norm(bhat))
        e1 = np.zeros(H.shape[0], dtype=np.complex128)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H, e1, rcond=None)
        red = float(np.linalg.norm(e1 - H @ y) / beta)
        print(json.dumps({
            "report": "harmonic_ritz", "dims": list(dims), "eps": eps, "m0": m0, "m": H.shape[1],
            "smallest_harmonic_ritz": [[float(z.real), float(z.imag)] for z in hr[:6]],
            "largest_harmonic_ritz_abs": float(np.abs(hr[-1])),
            "smallest_ritz": [[float(z.real), float(z.imag)] for z in rz[:4]],
            "cycle_residual_reduction": red, "seconds": time.time() - t0}), flush=True)
        del A, Ainv


def ladder_report(m0, eps=0.25, max_its=4096, m=32):
    syn = _synthetic()
    for dims in ((8, 8, 8, 8), (16, 8, 8, 8), (16, 16, 8, 8), (16, 16, 16, 8), (16, 16, 16, 16)):
        t0 = time.time()
        U = syn.gauge_field(dims, "exp", eps, seed=2000)
        b = syn.gaussian_spinors(dims, 1, 2001)
        A, Ainv = dirac.diag_blocks(U, m0, 1.0)
        x, infos = krylov.solve_eo(U, A, Ainv, b, tol=1e-10, m=m, max_restarts=max_its // m)
        info = infos[0]
        print(json.dumps({"report": "ladder", "dims": list(dims), "eps": eps, "m0": m0,
                          "converged": bool(info["converged"]), "iterations": int(info["iterations"]),
                          "relres": float(info["relres"]), "seconds": time.time() - t0}), flush=True)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "ritz"
    if what == "ritz":
        masses = [float(v) for v in sys.argv[2:]] or [-0.3, -0.1]
        ritz_report((64, 32, 32, 32), 0.25, masses, gauge_seed=2000, rhs_seed=2001)
    elif what == "ladder":
        ladder_report(float(sys.argv[2]) if len(sys.argv) > 2 else -0.3)
    else:
        raise SystemExit(__doc__)
