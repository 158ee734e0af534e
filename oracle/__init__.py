"""CPU oracle for the l1-regularised CGGM solved by alternating Newton coordinate descent.

TEST INFRASTRUCTURE: a plain, slow, double-precision CPU restatement of what the CUDA
solver computes, written from the paper (Eq. 1, Eq. 3, Eq. 4, Algorithm 1, Sections 3.1
and 3.2, Appendix A.1, the stopping rule of Section 5.1; ``oracle.blocks``: the block
coordinate descent of Algorithm 2 and Section 4; ``oracle.symbolic``: the symbolic
Cholesky of a sparse Lambda by the elimination game, and its numeric factor).  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark may import it.  It shares no code
with the CUDA path; both take inputs from the ``synth`` generators only.

Pins (tests/test_oracle_*.py): the lambda = 0 closed form, the q = 1 reduction to a
Lasso, the p = q = 1 scalar closed form, the Theta = 0 regime against a brute-force
proximal solver of the diagonal-penalised graphical lasso, KKT conditions, finite
differences of the objective, one-dimensional brute force for every coordinate step,
monotone decrease, and a brute-force proximal-gradient solve on tiny inputs; for the
blocked passes, equality with the pinned sequential passes in the blocked order, the
cache counts of Section 4, the lambda = 0 closed form and Algorithm 1's optimum; for the
symbolic Cholesky, the nonzero pattern of LAPACK's numeric factor and closed forms; for the
numeric factor, reconstruction, the LU determinant and the closed-form determinant of the
second-difference matrix.
"""
from .cggm_oracle import (  # noqa: F401
    OracleError,
    NotPositiveDefinite,
    LineSearchFailed,
    covariances,
    objective,
    smooth_objective,
    gradients,
    min_norm_subgradient,
    active_sets,
    lambda_sweep,
    theta_sweep,
    line_search,
    solve,
    soft_threshold,
    spd_solve,
    predict,
)
from . import blocks  # noqa: F401,E402
from . import symbolic  # noqa: F401,E402
