"""FP64 CPU oracle for approximate-ordering VarLiNGAM (test infrastructure).

This package is test infrastructure.  Only the test-suite, the smoke check and
the timed CPU baseline of the benchmark may import it; the library's CUDA path
never does, and nothing here imports the library.  It is deliberately plain and
slow: float64 NumPy, one obvious loop per step of the paper, no blocking, no
fusion and no incremental tricks, so that a reader can check it against the
paper by eye.

Contents (all in :mod:`oracle.fp64`):

* ``var_ols``            VAR(p) least squares with intercept (Section 4.1).
* ``var_select``         lag order by AIC / BIC / HQ on a common sample (a reading:
                         the paper takes p as given).
* ``standardize``        zero mean, unit variance per variable (Section 3, step 1).
* ``entropy``            maximum-entropy approximation H(u) (Section 3, step 3;
                         the constants are pinned in ``entropy_constants``).
* ``pairwise_measure``   E_x, E_r and the likelihood-ratio matrix D
                         (Section 3 steps 2-3, Eqs. 1-2; Section 4.2 items 1-2).
* ``order_heuristic``    Algorithm 1: m greedy argmins of Eq. 3 over the static
                         precomputed tables.
* ``order_standard``     the iterative DirectLiNGAM search with the data
                         refinement of Eq. 4 (Section 3, steps 1-5).
* ``order_gap_ok`` / ``order_standard_gap_ok``  the order comparison rules
                         (near ties of Eq. 3 may go either way).
* ``b0_ols`` / ``b0_ldl`` two independent routes to B0 from a causal order.
* ``btau``               B_tau = (I - B0) M_tau.
* ``varlingam``          the whole pipeline, heuristic or standard.
* ``bootstrap``          the pipeline on moving-block resamples of the series
                         (a reading: the paper specifies no resampling), with
                         the counter-based generator ``splitmix64_draw``.

:mod:`oracle.parallel` runs the same functions with the rows of E_r on a
process pool, only to time the oracle on all host cores (its results are the
serial oracle's, bit for bit; a test checks that).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, quadrature, brute force or library routines, except the
literature constant k1 = 79.047 of ``entropy`` (reproduced to 4 digits by a
quadrature in the tests, see ``entropy_constants``) and the accuracy of the
heuristic relative to the standard method, which is reported, not asserted
("parity unpinned": the paper gives no worked example of it).
"""
from .fp64 import (  # noqa: F401
    ENTROPY_GAMMA,
    ENTROPY_K1,
    ENTROPY_K2,
    H_GAUSS,
    b0_ldl,
    b0_ols,
    bootstrap,
    bootstrap_indices,
    btau,
    entropy,
    logcosh,
    order_gap_ok,
    order_heuristic,
    order_standard,
    order_standard_gap_ok,
    pairwise_measure,
    relative_gap,
    residual,
    score,
    scores_over,
    splitmix64,
    splitmix64_draw,
    standardize,
    var_ols,
    var_select,
    varlingam,
)
