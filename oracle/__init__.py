"""FP64 CPU oracle for polar-decomposition singular value soft-thresholding.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs may import, call, link or run anything
in this package. The GPU library never does: the two share no code, headers,
tables or generators; only the seeded input recipes in ``svt_workloads`` serve
both.

Contents (each function cites the passage of the paper it follows):

* ``native.jacobi_svd``: FP64 one-sided Jacobi SVD (plain C, OpenMP).
* ``svt.svt_definition``: Eq. 1, thresholding by definition.
* ``svt.prop1`` / ``prop1_footnote`` / ``prop1_factored`` / ``corollary_rank_r``:
  Proposition 1, its footnote, the factored form and Corollary 1 in FP64.
* ``svt.svt_polar_plain``: the method step by step as plain FP64 matrix products.
* ``schedule``: the oracle's own Remez derivation of the odd-polynomial schedules.
* ``spectral``: exact-arithmetic prediction of the method from the singular values.
* ``completion``: nuclear-norm matrix completion by proximal gradient with SVT by
  definition (Section 2's use of SVT), its objective and optimality residuals.

Pins (tests/test_oracle_*.py) tie these to closed forms, invariants, brute force
and LAPACK. Parity is pinned for every function listed above.
"""
from . import completion, native, schedule, spectral, svt  # noqa: F401
from .native import jacobi_svd  # noqa: F401
from .svt import (svt_definition, prop1, prop1_footnote, prop1_factored,  # noqa: F401
                  corollary_rank_r, best_rank_r, relerr, gap, svt_polar_plain,
                  polar_from_svd, sign_of_shifted_gram)
