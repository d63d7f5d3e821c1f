"""Plain FP64 restatement of approximate-ordering VarLiNGAM (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU baseline use this
module.  Every function names the passage of the paper it follows.  Where the
paper is silent (the entropy formula, the aggregation function f, B0 and B_tau
estimation, the VAR details) the reading used is stated in the docstring; the
readings come from the two methods the paper builds on, DirectLiNGAM
(Shimizu et al. 2011) and VarLiNGAM (Hyvarinen et al. 2010).

Conventions: data matrices are variable-major, X[i, t] = variable i at time t.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import scipy.linalg

# ------------------------------------------------------------------ entropy
# Maximum-entropy approximation of differential entropy (Hyvarinen 1998) with
# the two contrast functions G1(u) = log cosh u and G2(u) = u exp(-u^2/2), the
# form DirectLiNGAM uses.  The paper uses an entropy approximation without
# defining it (Section 3, step 3).
H_GAUSS = 0.5 * (1.0 + math.log(2.0 * math.pi))  # entropy of N(0, 1)
ENTROPY_K1 = 79.047  # weight of (E log cosh u - gamma)^2 (literature value)
ENTROPY_K2 = 7.4129  # weight of (E u exp(-u^2/2))^2 (= 36 / (8 sqrt3 - 9))
ENTROPY_GAMMA = 0.37457  # E log cosh nu for nu ~ N(0, 1)


def logcosh(u: np.ndarray) -> np.ndarray:
    """log cosh u = log((e^u + e^-u) / 2), evaluated without overflow."""
    return np.logaddexp(u, -u) - math.log(2.0)


def entropy(u: np.ndarray) -> float:
    """H(u) = H_nu - k1 (E[log cosh u] - gamma)^2 - k2 (E[u exp(-u^2/2)])^2
    for a standardized sample u (Section 3, step 3; formula is the reading
    above)."""
    u = np.asarray(u, dtype=np.float64)
    a = np.mean(logcosh(u))
    b = np.mean(u * np.exp(-0.5 * u * u))
    return H_GAUSS - ENTROPY_K1 * (a - ENTROPY_GAMMA) ** 2 - ENTROPY_K2 * b ** 2


# ------------------------------------------------------------------ VAR fit
def var_ols(X: np.ndarray, p: int) -> Tuple[np.ndarray, np.ndarray]:
    """VAR(p) least-squares fit x_t = c + sum_tau M_tau x_{t-tau} + n_t
    (Section 2.1 and Section 4.1: VarLiNGAM first fits a VAR and hands its
    residuals, the instantaneous shocks, to LiNGAM).

    Reading: an intercept c is fitted (as a VAR fit of a series with unknown
    mean does); rows t = p .. n-1 are the n_eff = n - p equations.

    Returns M (p, m, m) with M[tau-1][i, k] the effect of x_k(t - tau) on
    x_i(t), and the residuals E (m, n_eff), E[:, s] = n_{p+s}.
    """
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    n_eff = n - p
    if n_eff <= m * p + 1:
        raise ValueError("VAR system has no unique least-squares solution")
    Y = X[:, p:].T  # (n_eff, m)
    cols = [X[:, p - tau:n - tau].T for tau in range(1, p + 1)]
    Z = np.hstack(cols + [np.ones((n_eff, 1))])  # (n_eff, m p + 1)
    coef, *_ = np.linalg.lstsq(Z, Y, rcond=None)  # (m p + 1, m)
    M = np.stack([coef[(tau - 1) * m:tau * m, :].T for tau in range(1, p + 1)])
    E = (Y - Z @ coef).T
    return M, np.ascontiguousarray(E)


def var_select(X: np.ndarray, p_max: int, criterion: str = "bic") -> Dict[str, object]:
    """Lag order of the VAR by an information criterion (the paper takes p as
    given, Sec. 4.1; the reading follows the standard VAR practice, Lutkepohl,
    New Introduction to Multiple Time Series Analysis, Sec. 4.3).

    Every candidate p = 1..p_max is fitted by :func:`var_ols` on the same
    T = n - p_max equations (t = p_max .. n-1), so the criteria compare fits of
    the same data.  With the ML residual covariance S(p) = E E^T / T:
        AIC(p) = ln det S(p) + 2 p m^2 / T
        BIC(p) = ln det S(p) + ln(T) p m^2 / T
        HQ(p)  = ln det S(p) + 2 ln(ln T) p m^2 / T
    (the m intercepts are common to every p and left out).  The smallest
    value wins; ties pick the smaller p."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    T = n - p_max
    pen = {"aic": 2.0, "bic": math.log(T), "hq": 2.0 * math.log(math.log(T))}[criterion]
    values = []
    for p in range(1, p_max + 1):
        _, E = var_ols(X[:, p_max - p:], p)
        S = E @ E.T / T
        sign, logdet = np.linalg.slogdet(S)
        if sign <= 0:
            raise ValueError("residual covariance is not positive definite")
        values.append(logdet + pen * p * m * m / T)
    best = 1 + min(range(p_max), key=lambda i: (values[i], i))
    return {"p": best, "values": values, "T": T}


# ------------------------------------------------------ pairwise measure
def standardize(X: np.ndarray) -> np.ndarray:
    """Zero mean and unit variance per variable (Section 3, step 1), with the
    population standard deviation (ddof = 0)."""
    X = np.asarray(X, dtype=np.float64)
    mu = X.mean(axis=1, keepdims=True)
    sd = X.std(axis=1, keepdims=True)
    return (X - mu) / sd


def residual(xi: np.ndarray, xj: np.ndarray) -> np.ndarray:
    """Eq. 1: r_{i<-j} = x_i - cov(x_i, x_j) / var(x_j) * x_j (ddof 0 for both,
    so the ratio is the least-squares slope)."""
    ci = xi - xi.mean()
    cj = xj - xj.mean()
    cov = np.mean(ci * cj)
    var = np.mean(cj * cj)
    return xi - (cov / var) * xj


def pairwise_measure(Xs: np.ndarray) -> Dict[str, np.ndarray]:
    """One-time precomputation of Section 4.2 (items 1-2; Algorithm 1, the two
    precompute calls) on the standardized data Xs (m, n).

    E_x[i]    = H(x_i)                              (variable entropies)
    E_r[i, j] = H(r_{i<-j} / std(r_{i<-j}))         (residual entropies)
    T[i, j]   = T_{i<-j} = E_x[i] - E_r[i, j]       (Eq. 2)
    D[i, j]   = T_{j<-i} - T_{i<-j}
              = E_x[j] + E_r[i, j] - E_x[i] - E_r[j, i]

    Reading: each residual is rescaled to unit variance before H, because the
    approximation of H holds for standardized variables (DirectLiNGAM does the
    same).  D[i, j] > 0 is evidence for i -> j.  Diagonals are zero.
    """
    Xs = np.asarray(Xs, dtype=np.float64)
    m, _ = Xs.shape
    Ex = np.array([entropy(Xs[i]) for i in range(m)])
    Er = np.zeros((m, m))
    for i in range(m):
        for j in range(m):
            if i == j:
                continue
            r = residual(Xs[i], Xs[j])
            Er[i, j] = entropy(r / r.std())
    T = Ex[:, None] - Er
    np.fill_diagonal(T, 0.0)
    D = T.T - T
    return {"Ex": Ex, "Er": Er, "T": T, "D": D}


# ------------------------------------------------------------- ordering
def score(D: np.ndarray, i: int, U: Sequence[int]) -> float:
    """Eq. 3: M_i = sum_{j in U, j != i} f(T_{i<-j}, T_{j<-i}) with the
    reading f(T_{i<-j}, T_{j<-i}) = min(0, T_{j<-i} - T_{i<-j})^2
    = min(0, D[i, j])^2 (DirectLiNGAM's pairwise likelihood-ratio penalty: i
    is penalised for every j that looks like its cause)."""
    return float(sum(min(0.0, D[i, j]) ** 2 for j in U if j != i))


def scores_over(D: np.ndarray, U: Sequence[int]) -> Dict[int, float]:
    """Eq. 3 for every candidate i in U at once (the same sum as :func:`score`,
    written as one array expression so that m = 400 runs in seconds)."""
    Ua = np.asarray(list(U), dtype=np.int64)
    sub = D[np.ix_(Ua, Ua)].copy()
    np.fill_diagonal(sub, 0.0)  # j != i
    vals = (np.minimum(0.0, sub) ** 2).sum(axis=1)
    return {int(i): float(v) for i, v in zip(Ua, vals)}


def order_heuristic(D: np.ndarray) -> Dict[str, object]:
    """Algorithm 1: for k = 1..m pick c_k in U minimising M (Eq. 3) by lookups
    in the static precomputed table, append it to K, remove it from U.  The
    scores are recomputed from scratch over U at every step, as written.

    Ties pick the lowest index.  Returns the order K and, per step, the sorted
    candidate scores (for the relative-gap rule of :func:`order_gap_ok`).
    """
    D = np.asarray(D, dtype=np.float64)
    m = D.shape[0]
    U = list(range(m))
    K: List[int] = []
    steps = []
    for _ in range(m):
        scores = scores_over(D, U)
        best = min(U, key=lambda i: (scores[i], i))
        steps.append({"U": list(U), "scores": scores, "pick": best})
        K.append(best)
        U.remove(best)
    return {"order": np.array(K, dtype=np.int64), "steps": steps}


def order_standard(Xs: np.ndarray) -> Dict[str, object]:
    """The iterative DirectLiNGAM search of Section 3 (steps 1-5): every
    iteration re-standardizes the remaining variables, recomputes all pairwise
    residuals and entropies, picks the minimiser of Eq. 3, then replaces every
    remaining x_j by its residual on the pick (Eq. 4)."""
    X = np.array(Xs, dtype=np.float64, copy=True)
    m = X.shape[0]
    U = list(range(m))
    K: List[int] = []
    steps = []
    for _ in range(m):
        if len(U) == 1:
            K.append(U[0])
            steps.append({"U": list(U), "scores": {U[0]: 0.0}, "pick": U[0]})
            break
        sub = standardize(X[U])
        meas = pairwise_measure(sub)
        Dsub = meas["D"]
        loc = list(range(len(U)))
        sub_scores = scores_over(Dsub, loc)
        scores = {U[a]: sub_scores[a] for a in loc}
        best = min(U, key=lambda i: (scores[i], i))
        steps.append({"U": list(U), "scores": scores, "pick": best})
        K.append(best)
        U.remove(best)
        for j in U:  # Eq. 4 on the data of this iteration
            X[j] = residual(X[j], X[best])
    return {"order": np.array(K, dtype=np.int64), "steps": steps}


def relative_gap(scores: Dict[int, float]) -> float:
    vals = sorted(scores.values())
    if len(vals) < 2:
        return math.inf
    s1, s2 = vals[0], vals[1]
    return (s2 - s1) / max(abs(s1), abs(s2), 1e-300)


def order_gap_ok(order_gpu: Sequence[int], D_ref: np.ndarray, rel_gap: float = 1e-6,
                 D_cand: Optional[np.ndarray] = None) -> Tuple[bool, int, List[int]]:
    """Order comparison rule: walk the candidate order step by step over ITS
    OWN remaining set U; at each step the pick must be a minimiser of the
    reference scores (Eq. 3 over D_ref), unless the reference scores of the
    pick and the true minimiser lie within `rel_gap` relative of each other
    (a near tie, where either choice is correct up to rounding).

    With D_cand (the matrix the candidate ordered, equal to D_ref up to the
    measure's tolerance), a step also passes when the two reference scores are
    closer than the change of those scores that the difference D_cand - D_ref
    itself produces: sum over U of |min(0, D_cand)^2 - min(0, D_ref)^2| for the
    pick plus the same for the minimiser.  The order is then Algorithm 1's on
    the candidate's own D, and the difference comes from D, which is checked
    against its own tolerance.

    Returns (ok, number of near-tie steps, list of failing steps)."""
    D_ref = np.asarray(D_ref, dtype=np.float64)
    m = D_ref.shape[0]
    U = list(range(m))
    ties = 0
    bad: List[int] = []
    if sorted(int(c) for c in order_gpu) != list(range(m)):
        return False, 0, [-1]
    dP = None
    if D_cand is not None:
        D_cand = np.asarray(D_cand, dtype=np.float64)
        dP = np.abs(np.minimum(0.0, D_cand) ** 2 - np.minimum(0.0, D_ref) ** 2)
        np.fill_diagonal(dP, 0.0)
    for k, c in enumerate(order_gpu):
        c = int(c)
        scores = scores_over(D_ref, U)
        imin = min(scores, key=lambda i: (scores[i], i))
        smin = scores[imin]
        sc = scores[c]
        if sc != smin:
            denom = max(abs(sc), abs(smin), 1e-300)
            band = 0.0
            if dP is not None:
                Ua = np.asarray(U)
                band = dP[c, Ua].sum() + dP[imin, Ua].sum()
            if (sc - smin) / denom <= rel_gap or sc - smin <= band:
                ties += 1
            else:
                bad.append(k)
        U.remove(c)
    return (not bad), ties, bad


def order_standard_gap_ok(Xs: np.ndarray, order_cand: Sequence[int], rel_gap: float = 1e-6,
                          d_tol: float = 0.0, gaps_cand: Optional[Sequence[float]] = None,
                          only_steps: Optional[Sequence[int]] = None
                          ) -> Tuple[bool, int, List[int]]:
    """Order comparison rule for the iterative search of Section 3: the
    search of :func:`order_standard` is replayed, but every iteration removes
    the CANDIDATE's pick and refines the remaining variables on it (Eq. 4), so
    that one early near tie does not make every later step incomparable.  At
    each iteration the pick must minimise the reference scores (Eq. 3 over the
    D of that iteration's data), unless the two scores lie within `rel_gap`
    relative of each other, or within the band that a difference of at most
    d_tol * max|D| in every entry of D can produce: for one score that is the
    sum over U of 2 |D_ij| delta + delta^2, taken for the pick and for the
    minimiser.

    With gaps_cand (the candidate's relative gap per iteration), an iteration
    also fails when that gap differs from the reference's (S_(2) - S_(1)) /
    S_(2) by more than a D difference of d_tol * max|D| explains: if no score
    moves by more than B (the largest band above), neither do the two
    smallest, and the gap moves by at most 2 B / (S_(2) - B), plus rel_gap.

    With only_steps, the measure is evaluated (and the step checked) only at
    those iterations; the others just apply Eq. 4 on the candidate's pick, so
    that a long search can be checked on a sample of its iterations.

    Returns (ok, number of near-tie steps, list of failing steps)."""
    X = np.array(Xs, dtype=np.float64, copy=True)
    m = X.shape[0]
    if sorted(int(c) for c in order_cand) != list(range(m)):
        return False, 0, [-1]
    check = None if only_steps is None else set(int(k) for k in only_steps)
    U = list(range(m))
    ties = 0
    bad: List[int] = []
    for k, c in enumerate(order_cand):
        c = int(c)
        if len(U) == 1:
            break
        if check is not None and k not in check:
            U.remove(c)
            for j in U:  # Eq. 4 on the candidate's pick
                X[j] = residual(X[j], X[c])
            continue
        D = pairwise_measure(standardize(X[U]))["D"]
        loc = {v: a for a, v in enumerate(U)}
        sub = scores_over(D, range(len(U)))
        scores = {v: sub[loc[v]] for v in U}
        imin = min(U, key=lambda i: (scores[i], i))
        sc, smin = scores[c], scores[imin]
        delta = d_tol * np.abs(D).max()
        A = np.abs(D)
        np.fill_diagonal(A, 0.0)
        nb = len(U) - 1
        bands = 2.0 * delta * A.sum(axis=1) + nb * delta * delta  # per local index
        failed = False
        if sc != smin:
            denom = max(abs(sc), abs(smin), 1e-300)
            band = bands[loc[c]] + bands[loc[imin]]
            if (sc - smin) / denom <= rel_gap or sc - smin <= band:
                ties += 1
            else:
                failed = True
        if gaps_cand is not None:
            vals = sorted(scores.values())
            s1, s2 = vals[0], vals[1]
            g_ref = (s2 - s1) / max(abs(s1), abs(s2), 1e-300)
            B = bands.max()
            tol = 2.0 * B / max(s2 - B, 1e-300) + rel_gap
            if not abs(float(gaps_cand[k]) - g_ref) <= tol:
                failed = True
        if failed:
            bad.append(k)
        U.remove(c)
        for j in U:  # Eq. 4 on the candidate's pick
            X[j] = residual(X[j], X[c])
    return (not bad), ties, bad


# --------------------------------------------------------- B0 and B_tau
def b0_ols(E: np.ndarray, order: Sequence[int]) -> np.ndarray:
    """B0 from a causal order (Section 4: the instantaneous matrix of
    VarLiNGAM).  Reading: row c_k of B0 holds the least-squares coefficients
    of e_{c_k} on its predecessors e_{c_1..c_{k-1}} (with an intercept); the
    first variable of the order has no parents.  B0[i, j] is the effect j -> i.
    """
    E = np.asarray(E, dtype=np.float64)
    m, n = E.shape
    B0 = np.zeros((m, m))
    order = [int(c) for c in order]
    for k in range(1, m):
        tgt = order[k]
        preds = order[:k]
        A = np.hstack([E[preds].T, np.ones((n, 1))])
        coef, *_ = np.linalg.lstsq(A, E[tgt], rcond=None)
        B0[tgt, preds] = coef[:-1]
    return B0


def b0_ldl(E: np.ndarray, order: Sequence[int]) -> np.ndarray:
    """Second, independent route to the same B0: with the centred covariance
    S of E permuted into the causal order, S_perm = L diag(d) L^T with L unit
    lower triangular, and I - L^{-1} holds every predecessor regression at
    once (sequential regression = Cholesky)."""
    E = np.asarray(E, dtype=np.float64)
    m, n = E.shape
    order = np.asarray(order, dtype=np.int64)
    C = E - E.mean(axis=1, keepdims=True)
    S = C @ C.T / n
    Sp = S[np.ix_(order, order)]
    Lc = scipy.linalg.cholesky(Sp, lower=True)
    L = Lc / np.diag(Lc)[None, :]
    Linv = scipy.linalg.solve_triangular(L, np.eye(m), lower=True, unit_diagonal=True)
    Bp = np.eye(m) - Linv
    B0 = np.zeros((m, m))
    B0[np.ix_(order, order)] = Bp
    return B0


def btau(B0: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Lagged effects of the structural VAR: x_t = B0 x_t + sum B_tau x_{t-tau}
    + e_t has reduced form M_tau = (I - B0)^{-1} B_tau, so
    B_tau = (I - B0) M_tau (VarLiNGAM, Hyvarinen et al. 2010)."""
    m = B0.shape[0]
    return np.stack([(np.eye(m) - B0) @ M[t] for t in range(M.shape[0])])


# ------------------------------------------------------------ pipeline
def varlingam(X: np.ndarray, p: int, method: str = "heuristic") -> Dict[str, object]:
    """Whole method on one series.  'heuristic' = the paper's Algorithm 1 on
    the VAR residuals (the data are never refined); 'standard' = iterative
    DirectLiNGAM (Section 3).  B0 by predecessor OLS, B_tau = (I - B0) M."""
    M, E = var_ols(X, p)
    Xs = standardize(E)
    out: Dict[str, object] = {"M": M, "E": E}
    if method == "heuristic":
        meas = pairwise_measure(Xs)
        out.update(meas)
        od = order_heuristic(meas["D"])
    elif method == "standard":
        od = order_standard(Xs)
    else:
        raise ValueError(method)
    out["order"] = od["order"]
    out["steps"] = od["steps"]
    B0 = b0_ols(E, od["order"])
    out["B0"] = B0
    out["Btau"] = btau(B0, M)
    return out


# ------------------------------------------------------------ bootstrap
# Bootstrap resampling of the batched path (the paper does not specify one;
# the reading is the moving-block bootstrap of Kuensch, Ann. Statist. 1989,
# the usual resampling for a dependent series).  Its random block starts are
# drawn from a counter-based generator written here from its published
# definition, the SplitMix64 output function (Steele, Lea and Flood, OOPSLA
# 2014), so that any draw can be produced independently of the others.
MASK64 = (1 << 64) - 1
SPLITMIX_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(state: int) -> int:
    """The SplitMix64 output for a state already advanced by the gamma:
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) *
    0x94D049BB133111EB; z ^ (z >> 31), all modulo 2^64."""
    z = state & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_draw(seed: int, counter: int) -> int:
    """Output number `counter` (1, 2, ...) of SplitMix64 seeded with `seed`:
    the state after `counter` steps is seed + counter * gamma."""
    return splitmix64((seed + counter * SPLITMIX_GAMMA) & MASK64)


def bootstrap_indices(n: int, block_len: int, seed: int, b: int) -> np.ndarray:
    """Time indices of moving-block resample b of a series of length n: blocks
    k = 0, 1, .. of block_len consecutive indices starting at
    s_k = floor(u_k (n - block_len + 1) / 2^64), u_k = draw b 2^32 + k + 1 of
    the generator, concatenated and cut to n."""
    if not 1 <= block_len <= n:
        raise ValueError("need 1 <= block_len <= n")
    span = n - block_len + 1
    idx = np.empty(n, dtype=np.int64)
    for t in range(n):
        k, off = divmod(t, block_len)
        u = splitmix64_draw(seed, (b << 32) + k + 1)
        idx[t] = ((u * span) >> 64) + off
    return idx


def bootstrap(X: np.ndarray, p: int, n_resamples: int, block_len: int, seed: int,
              threshold: float, method: str = "heuristic") -> Dict[str, object]:
    """The whole method on every resample b = 0..n_resamples-1 (resample b is
    X[:, bootstrap_indices(n, block_len, seed, b)]), then
        edge_prob[i, j]  = fraction of resamples with |B0[i, j]| > threshold,
        order_prob[i, j] = fraction of resamples in which i precedes j in the
                           causal order (0 on the diagonal);
    also the per-resample orders, B0 and smallest relative score gap of the
    search (for comparisons that must allow near ties)."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    edge = np.zeros((m, m))
    before = np.zeros((m, m))
    orders, B0s, gaps = [], [], []
    for b in range(n_resamples):
        r = varlingam(X[:, bootstrap_indices(n, block_len, seed, b)], p, method)
        order = [int(c) for c in r["order"]]
        pos = np.empty(m, dtype=np.int64)
        pos[order] = np.arange(m)
        edge += np.abs(r["B0"]) > threshold
        before += pos[:, None] < pos[None, :]
        orders.append(order)
        B0s.append(r["B0"])
        gaps.append(min([relative_gap(st["scores"]) for st in r["steps"][:-1]] or [math.inf]))
    return {"edge_prob": edge / n_resamples, "order_prob": before / n_resamples,
            "orders": orders, "B0s": B0s, "min_gaps": gaps}

