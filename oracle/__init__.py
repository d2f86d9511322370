"""FP64 CPU oracle for the multi-rhs Wilson(-clover) Dirac operator and batched GMRES.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or link
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares
no code with the CUDA library (``paper_2601_05816_gb300``) and imports nothing
from it; both sides only consume the seeded inputs of ``synthetic``.

The oracle is plain numpy in complex128, written from the paper's definitions:

* ``dirac``: gamma matrices (chiral basis), the Wilson-Dirac operator of
  Sec. III-A-1 (self term, projectors pi^-/pi^+ (x) U, lattice shifts), the
  clover term C(x) and D = D_W - C, the odd-even split and the Schur complement
  of Sec. III-A-2.
* ``krylov``: restarted GMRES with Arnoldi (modified Gram-Schmidt), Givens
  rotations and the least-squares update of Algorithm 2, run per rhs (the
  batched solver of Algorithm 2 runs the rhs independently), and the odd-even
  (Schur) solve.
* ``dense``: a brute-force dense matrix of D built entry by entry with explicit
  site loops, for tiny lattices.
* ``adjoint``: the adjoint operator D^dagger, the adjoint solve and the
  gradients dL/db and dL/dU (hopping and clover-leaf parts) of
  L = sum_i Re <eta_i, D^{-1} b_i> (the task's differentiable solve; not in the
  paper), pinned by finite differences of the dense operator's loss.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, invariants, brute force, library
solves); none is "parity unpinned". The paper prints no operator values, so the
operator itself is pinned by theory only.
"""
from .dirac import (  # noqa: F401
    gamma_matrices, gamma5, apply_D, hopping_sum, clover_term, site_matrix_apply,
    diag_blocks, parity_mask, split_parity, embed_parity, apply_D_eo, apply_D_oe,
    apply_Aee_inv, apply_Aoo, apply_schur, schur_prepare, schur_reconstruct,
    plaquette_leaves,
)
from .krylov import gmres, solve_full, solve_eo  # noqa: F401
from .dense import dense_operator  # noqa: F401
