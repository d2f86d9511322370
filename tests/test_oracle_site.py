"""Pins of the per-site oracle (oracle/site.py) used for sampled parity on large lattices.

Each site-wise function is compared, at every site of small lattices, with the
whole-lattice oracle (itself pinned by closed forms, invariants and dense brute
force in test_oracle_operator.py); the two are written independently (explicit
coordinates and per-site 3x3 / 12x12 products here, lattice-wide rolls and
einsums there). Lattices: 2^4 (x + mu = x - mu, both time hops cross the
boundary), a non-cubic 8x2x6x4 and 4^4 with a time extent that exercises the
antiperiodic wrap in both directions.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import site
import synthetic as syn

CASES = [((2, 2, 2, 2), 0.6, 0.2, 1.0), ((8, 2, 6, 4), 0.5, 0.05, 1.3), ((4, 4, 4, 4), 0.3, -0.2, 1.0),
         ((4, 2, 2, 4), 0.4, 0.1, 0.0)]


@pytest.mark.parametrize("case", CASES)
def test_site_block_and_full_operator_every_site(case):
    dims, eps, m0, c_sw = case
    U = syn.gauge_field(dims, "exp", eps, seed=11)
    psi = syn.gaussian_spinors(dims, 1, 12)
    ref = oracle.apply_D(U, psi, m0, oracle.clover_term(U, c_sw))[0]
    A_ref, _ = oracle.diag_blocks(U, m0, c_sw)
    for x in itertools.product(*(range(d) for d in dims)):
        assert np.allclose(site.site_block(U, x, m0, c_sw), A_ref[x], atol=1e-13)
        assert np.allclose(site.apply_D_at(U, psi[0], x, m0, c_sw), ref[x], atol=1e-12)


@pytest.mark.parametrize("case", CASES)
def test_schur_operator_every_odd_site(case):
    dims, eps, m0, c_sw = case
    U = syn.gauge_field(dims, "exp", eps, seed=13)
    A, Ainv = oracle.diag_blocks(U, m0, c_sw)
    psi_o = oracle.split_parity(syn.gaussian_spinors(dims, 1, 14), 1)
    ref = oracle.apply_schur(U, A, Ainv, psi_o)[0]
    n = 0
    for x in itertools.product(*(range(d) for d in dims)):
        if sum(x) % 2 == 1:
            k = site.half_index(dims, x)
            assert np.allclose(site.apply_schur_at(U, psi_o[0], x, m0, c_sw), ref[k], atol=1e-12)
            n += 1
    assert n == np.prod(dims) // 2


def test_half_index_matches_split_parity_order():
    dims = (4, 2, 6, 4)
    lex = np.arange(np.prod(dims)).reshape(dims)
    for p in (0, 1):
        order = oracle.split_parity(lex[None, ..., None, None] * np.ones((1,) + dims + (4, 3)), p)[0, :, 0, 0]
        for k, l in enumerate(order.real.astype(int)):
            x = np.unravel_index(l, dims)
            assert site.half_index(dims, x) == k
