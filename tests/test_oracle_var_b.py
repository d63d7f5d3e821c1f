"""Pins for the oracle's VAR fit (Section 4.1) and its B0 / B_tau estimates."""
import numpy as np

import oracle
import synth


def test_var_normal_equations_and_zero_mean():
    inst = synth.make_instance(5, 400, 2, 11, "laplace", 0.3, 0.1, 0.5, "unif", 0.8)
    M, E = oracle.var_ols(inst.X, 2)
    m, n = inst.X.shape
    Z = np.vstack([inst.X[:, 2 - t:n - t] for t in (1, 2)])
    assert np.allclose(E.mean(axis=1), 0, atol=1e-12)
    assert np.max(np.abs(Z @ E.T)) < 1e-9 * np.abs(Z).max() * np.abs(E).max() * n


def test_var_matches_explicit_regression_per_equation():
    inst = synth.make_instance(4, 300, 1, 12, "uniform", 0.3, 0.1, 0.5, "unif", 0.6)
    M, E = oracle.var_ols(inst.X, 1)
    X = inst.X
    # equation i by the textbook formula beta = (Z^T Z)^{-1} Z^T y with intercept
    Z = np.hstack([X[:, :-1].T, np.ones((299, 1))])
    for i in range(4):
        beta = np.linalg.solve(Z.T @ Z, Z.T @ X[i, 1:])
        assert np.allclose(beta[:4], M[0][i], atol=1e-10)


def test_var_intercept_invariance():
    inst = synth.make_instance(4, 500, 2, 13, "t3", 0.3, 0.1, 0.5, "unif", 0.7)
    M1, E1 = oracle.var_ols(inst.X, 2)
    M2, E2 = oracle.var_ols(inst.X + np.array([[5.0], [-2.0], [0.0], [100.0]]), 2)
    assert np.allclose(M1, M2, atol=1e-9)
    assert np.allclose(E1, E2, atol=1e-8)


def test_var_recovers_truth_at_large_n():
    inst = synth.make_instance(4, 100_000, 2, 14, "uniform", 0.3, 0.1, 0.5, "unif", 0.8)
    M, _ = oracle.var_ols(inst.X, 2)
    assert np.max(np.abs(M - inst.M)) < 0.03


def test_b0_two_routes_agree():
    inst = synth.make_instance(7, 800, 1, 15, "laplace", 0.4, 0.1, 0.5, "unif", 0.6)
    _, E = oracle.var_ols(inst.X, 1)
    order = np.random.default_rng(3).permutation(7)
    B1 = oracle.b0_ols(E, order)
    B2 = oracle.b0_ldl(E, order)
    assert np.allclose(B1, B2, atol=1e-10)
    # strictly lower triangular in the causal order
    Bp = B1[np.ix_(order, order)]
    assert np.allclose(np.triu(Bp), 0)


def test_b0_and_btau_recover_truth_with_true_order():
    inst = synth.make_instance(5, 100_000, 2, 16, "uniform", 0.5, 0.2, 0.6, "unif", 0.7)
    M, E = oracle.var_ols(inst.X, 2)
    B0 = oracle.b0_ols(E, inst.perm)
    assert np.max(np.abs(B0 - inst.B0)) < 0.03
    Bt = oracle.btau(B0, M)
    assert np.max(np.abs(Bt - inst.Btau())) < 0.04
    # B_tau = (I - B0) M_tau, not M_tau (I - B0)
    wrong = np.stack([M[t] @ (np.eye(5) - B0) for t in range(2)])
    assert np.max(np.abs(wrong - inst.Btau())) > 0.05


def test_full_pipeline_heuristic_recovers_b0():
    inst = synth.make_instance(6, 50_000, 1, 17, "uniform", 0.4, 0.3, 0.7, "unif", 0.5)
    out = oracle.varlingam(inst.X, 1)
    assert np.max(np.abs(out["B0"] - inst.B0)) < 0.05


def test_lag_selection_recovers_the_true_order_at_large_n():
    """BIC is consistent: on long series of VAR(1), VAR(2) and VAR(3)
    processes with clear lag coefficients it selects the generating p."""
    for p_true, seed in ((1, 11), (2, 12), (3, 13)):
        inst = synth.make_instance(4, 20000, p_true, seed, "laplace", 0.3, 0.2, 0.5, "unif", 0.8,
                                   var_lo=0.2, var_hi=0.4)
        sel = oracle.var_select(inst.X, 5, "bic")
        assert sel["p"] == p_true, (p_true, sel["values"])


def test_lag_selection_invariances_and_penalty_order():
    """Scaling the data by c shifts every criterion by exactly 2 m ln c and
    permuting the variables changes none, so neither changes the choice; the
    penalties order AIC <= HQ <= BIC (T > 15), so the selected lags order the
    other way; the candidate with p = p_max is the plain fit on all rows."""
    rng = np.random.default_rng(4)
    inst = synth.make_instance(5, 400, 2, 21, "uniform", 0.3, 0.1, 0.5, "unif", 0.7)
    X = inst.X
    base = oracle.var_select(X, 4, "aic")
    c = 3.7
    scaled = oracle.var_select(c * X, 4, "aic")
    np.testing.assert_allclose(np.array(scaled["values"]) - np.array(base["values"]),
                               2 * 5 * np.log(c), rtol=0, atol=1e-9)
    assert scaled["p"] == base["p"]
    perm = rng.permutation(5)
    np.testing.assert_allclose(oracle.var_select(X[perm], 4, "aic")["values"], base["values"],
                               rtol=0, atol=1e-9)
    for k in range(20):
        Xr = synth.make_instance(3, 120, 1 + k % 3, 100 + k, "laplace", 0.3, 0.1, 0.5, "unif",
                                 0.6).X
        pa = oracle.var_select(Xr, 4, "aic")["p"]
        ph = oracle.var_select(Xr, 4, "hq")["p"]
        pb = oracle.var_select(Xr, 4, "bic")["p"]
        assert pb <= ph <= pa
    M, E = oracle.var_ols(X, 4)
    S = E @ E.T / E.shape[1]
    full = np.linalg.slogdet(S)[1] + np.log(X.shape[1] - 4) * 4 * 25 / (X.shape[1] - 4)
    assert abs(oracle.var_select(X, 4, "bic")["values"][3] - full) < 1e-9
