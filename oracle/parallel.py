"""Process-pool driver over the oracle's own functions (test infrastructure).

The same arithmetic as ``oracle.fp64.varlingam(X, p, "heuristic")``: VAR fit,
standardization, the residual entropies E_r, Eq. 2 and the likelihood-ratio
matrix D, Algorithm 1, B0 by predecessor OLS and B_tau; only the rows of E_r
(the O(m^2 n) part) are computed by worker processes, each running the
oracle's own ``residual`` and ``entropy`` on a block of rows.  It exists to
time the oracle on all host cores next to the one-core run; nothing in the
library imports it.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import fp64


def _er_rows(task: Tuple[np.ndarray, Sequence[int]]) -> Tuple[Sequence[int], np.ndarray]:
    """Rows `rows` of E_r (Section 3, step 3; the loop of fp64.pairwise_measure)."""
    Xs, rows = task
    m = Xs.shape[0]
    out = np.zeros((len(rows), m))
    for a, i in enumerate(rows):
        for j in range(m):
            if i == j:
                continue
            r = fp64.residual(Xs[i], Xs[j])
            out[a, j] = fp64.entropy(r / r.std())
    return rows, out


def pairwise_measure_pool(Xs: np.ndarray, pool, nproc: int) -> Dict[str, np.ndarray]:
    """fp64.pairwise_measure with the rows of E_r dealt round-robin to `pool`."""
    Xs = np.asarray(Xs, dtype=np.float64)
    m = Xs.shape[0]
    Ex = np.array([fp64.entropy(Xs[i]) for i in range(m)])
    blocks: List[List[int]] = [list(range(w, m, nproc)) for w in range(nproc) if w < m]
    Er = np.zeros((m, m))
    for rows, vals in pool.map(_er_rows, [(Xs, b) for b in blocks]):
        Er[rows, :] = vals
    T = Ex[:, None] - Er
    np.fill_diagonal(T, 0.0)
    D = T.T - T
    return {"Ex": Ex, "Er": Er, "T": T, "D": D}


def varlingam_pool(X: np.ndarray, p: int, pool, nproc: int) -> Dict[str, object]:
    """fp64.varlingam(X, p, "heuristic") with the pairwise measure on `pool`."""
    M, E = fp64.var_ols(X, p)
    Xs = fp64.standardize(E)
    meas = pairwise_measure_pool(Xs, pool, nproc)
    od = fp64.order_heuristic(meas["D"])
    B0 = fp64.b0_ols(E, od["order"])
    return {"M": M, "E": E, "order": od["order"], "B0": B0, "Btau": fp64.btau(B0, M), **meas}
