"""The oracle against the values the paper prints (fixtures under tests/golden/, each citing
the passage it comes from).

The paper prints no worked numerical example of the operator or the solver; what it does print
about the computation is the site numbering and the per-site storage counts of Sec. III-A-1.
These tests tie the oracle's readings (site order, chiral gamma basis, projectors, clover
construction) to those printed values.
"""
import os

import numpy as np

import oracle
import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                key, value = (s.strip() for s in line.split("=", 1))
                out[key] = value
    return out


def _strides(expr, N):
    """'N1*N2*N3, N1*N2, N1, 1' evaluated for the extents N = (N0, N1, N2, N3)."""
    out = []
    for term in expr.split(","):
        s = 1
        for factor in term.strip().split("*"):
            factor = factor.strip()
            s *= N[int(factor[1:])] if factor.startswith("N") else int(factor)
        out.append(s)
    return out


def _site_numbers(dims, strides):
    t, z, y, x = np.indices(dims)
    return t * strides[0] + z * strides[1] + y * strides[2] + x * strides[3]


def test_site_numbering_reading_is_the_oracle_order_and_the_printed_one_when_n1_eq_n3():
    g = _read("site_numbering.txt")
    for dims in [(4, 2, 6, 2), (2, 4, 4, 4), (4, 6, 2, 6)]:        # N1 = N3: both formulas agree
        printed = _site_numbers(dims, _strides(g["printed_strides"], dims))
        reading = _site_numbers(dims, _strides(g["reading_strides"], dims))
        assert np.array_equal(printed, reading)
        # the oracle stores sites in increasing site number (C order of [T, Z, Y, X]) and lists the
        # sites of one parity in that order
        assert np.array_equal(reading.ravel(), np.arange(np.prod(dims)))
        field = reading[None, ..., None, None] * np.ones((1,) + dims + (4, 3))
        for p in (0, 1):
            listed = oracle.split_parity(field, p)[0, :, 0, 0].real
            assert np.all(np.diff(listed) > 0)
    for dims in [(2, 4, 2, 2), (4, 2, 4, 6)]:                        # N1 != N3: the printed strides collide
        printed = _site_numbers(dims, _strides(g["printed_strides"], dims))
        assert len(np.unique(printed)) < np.prod(dims) or printed.max() >= np.prod(dims)
        reading = _site_numbers(dims, _strides(g["reading_strides"], dims))
        assert np.array_equal(np.sort(reading.ravel()), np.arange(np.prod(dims)))


def test_storage_counts_per_site():
    g = {k: int(v) for k, v in _read("storage_counts.txt").items()}
    dims = (2, 2, 2, 2)
    U = syn.gauge_field(dims, "exp", 0.5, seed=17)
    psi = syn.gaussian_spinors(dims, 1, 18)
    assert np.prod(psi.shape[-2:]) == g["spinor_per_site"]
    # clover: entries that are nonzero at some site form two Hermitian 6x6 diagonal blocks in the
    # chiral basis; the independent complex numbers are their upper triangles
    C = oracle.clover_term(U, 1.0).reshape(-1, 12, 12)
    assert np.allclose(C, np.conj(np.swapaxes(C, -1, -2)), atol=1e-14)
    support = np.any(np.abs(C) > 1e-12, axis=0)
    spin_block = np.kron(np.array([[1, 1, 0, 0], [1, 1, 0, 0], [0, 0, 1, 1], [0, 0, 1, 1]]), np.ones((3, 3))) > 0
    assert np.array_equal(support, spin_block)
    assert int(np.triu(support).sum()) == g["clover_per_site"]
    # the projectors pi^{+-}_mu = (1 +- gamma_mu)/2 keep 2 of 4 spins: 6 complex numbers per site
    gam = oracle.gamma_matrices()
    for mu in range(4):
        for sgn in (1, -1):
            P = np.kron((np.eye(4) + sgn * gam[mu]) / 2, np.eye(3))
            assert np.allclose(P @ P, P)
            assert np.linalg.matrix_rank(P) == g["half_spinor_per_site"]
