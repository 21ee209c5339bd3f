"""Block-tridiagonal dichotomy solver for GB300 (sm_103a).

Terekhov, "A fast parallel algorithm for solving block-tridiagonal systems of
linear equations including the domain decomposition method" (arXiv:1108.4181):
Algorithm 2 with segments mapped to CTAs.  The compute path is the C-ABI
library ``libbt.so`` (declared in ``include/bt.h``); this package only
marshals arguments to it.
"""

from ._lib import BtError, load  # noqa: F401
from .solver import (BandFactorization, BatchPlan, Factorization, factor, factor_band,  # noqa: F401
                     solve_batched, solve_refined_sets)
from .autograd import BTSolve, bt_solve  # noqa: F401,E402
from . import tune  # noqa: F401,E402
from .schur import SchurPCG  # noqa: F401,E402
