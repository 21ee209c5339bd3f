"""CPU FP64 oracle for the block-tridiagonal solve -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
path (the C-ABI library and its Python binding) never imports, links or calls
it, and this package never imports the product path.

Contents (each function cites the passage of Terekhov, "A fast parallel
algorithm for solving block-tridiagonal systems ...", arXiv:1108.4181, that it
writes out):

* ``blocktri``  -- the system of Section 2 (eq. main-eq) by definition: the
  operator product, the assembled dense matrix, the exact solution by block
  Gaussian elimination (block Thomas) and by dense LU, residual and error norms.
* ``alg2``      -- the segment/interface decomposition of Section 2.2 written
  out by definition: the responses of eqs. sub1-sub3, the reduced system of
  eq. red1, Algorithm 1 applied to it, and the superposition of eq.
  superposition.  Used to pin the GPU path's intermediate products.
* ``band``      -- a band matrix in diagonal-ordered storage and its cut into
  the block-tridiagonal form (Section 3.3.1, item c: the PML operator solved
  by the dichotomy with triangular off-diagonal blocks), identity-padded.
* ``schur``     -- the Schur-complement CG of Section 3.3 on a strip
  decomposition of the five-point grid operator: the product with S (each
  strip inverted as a block-tridiagonal system), the reduced right-hand side,
  the recovery of eq. domains_equation, the probing band preconditioner of
  Section 3.3.2 and textbook preconditioned CG.
* ``adjoint``   -- gradients of a loss through X = P^{-1} F (not in the paper;
  the standard adjoint identity dL/dP = -lambda X^T with P^T lambda = dL/dX).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(``schur`` by ``tests/test_schur_oracle.py``)
against values fixed independently of this code (closed forms, library
routines, invariants, brute force).  No function is "parity unpinned".
"""

from .blocktri import (  # noqa: F401
    apply_P,
    dense_P,
    solve_dense,
    solve_block_thomas,
    col_err,
    residual,
    rel_err,
    rel_res,
)
from .alg2 import (  # noqa: F401
    segment_rows,
    segment_responses,
    segment_W,
    reduced_system,
    reduced_rhs,
    dichotomy_tree,
    dichotomy_solve,
    alg2_solve,
)
from .adjoint import transpose_blocks, adjoint_grads  # noqa: F401
from .band import band_dense, band_blocks, pad_rows  # noqa: F401
