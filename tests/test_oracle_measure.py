"""Pins for the oracle's pairwise measure (Section 3 steps 2-3, Eqs. 1-2;
Section 4.2 items 1-2)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

SQ3 = math.sqrt(3.0)


def _h_from_moments(a, b):
    return (oracle.H_GAUSS - oracle.ENTROPY_K1 * (a - oracle.ENTROPY_GAMMA) ** 2
            - oracle.ENTROPY_K2 * b * b)


def _h_uniform_mix(c1, c2):
    """Approximate entropy of c1*A + c2*B, A, B iid uniform(-sqrt3, sqrt3),
    c1^2 + c2^2 = 1, by 2-D quadrature of the two moments (odd moment = 0 by
    symmetry)."""
    dens = 1.0 / (2 * SQ3) ** 2
    a, _ = integrate.dblquad(lambda y, x: math.log(math.cosh(c1 * x + c2 * y)) * dens,
                             -SQ3, SQ3, -SQ3, SQ3, epsabs=1e-11)
    return _h_from_moments(a, 0.0)


@pytest.fixture(scope="module")
def bivariate():
    rng = np.random.default_rng(7)
    n = 1_000_000
    a = rng.uniform(-SQ3, SQ3, n)
    b = rng.uniform(-SQ3, SQ3, n)
    xj = a
    xi = 0.8 * a + 0.6 * b  # j -> i with independent uniform noise
    X = oracle.standardize(np.vstack([xi, xj]))
    return oracle.pairwise_measure(X)


def test_residual_entropies_match_closed_form(bivariate):
    """Index convention and residual standardization: with x_i = 0.8 x_j + 0.6 e,
    r_{i<-j} is e itself (entropy of a uniform) while r_{j<-i} is the mixture
    0.6 x_j - 0.8 e; E_x are the entropies of a uniform and of 0.8a + 0.6b."""
    m = bivariate
    h_u = _h_uniform_mix(1.0, 0.0)
    h_86 = _h_uniform_mix(0.8, 0.6)
    tol = 1.5e-3  # Monte Carlo error at n = 1e6
    assert abs(m["Ex"][1] - h_u) < tol
    assert abs(m["Ex"][0] - h_86) < tol
    assert abs(m["Er"][0, 1] - h_u) < tol  # r_{i<-j} = noise of i
    assert abs(m["Er"][1, 0] - h_86) < tol  # 0.6a - 0.8b has the law of 0.8a + 0.6b
    # D[j, i] = T_{i<-j} - T_{j<-i} > 0: evidence for j -> i
    expect = h_86 + h_86 - 2 * h_u
    assert expect > 0.01
    assert abs(m["D"][1, 0] - expect) < 3 * tol
    assert abs(m["D"][0, 1] + expect) < 3 * tol


def test_d_antisymmetric_zero_diagonal():
    rng = np.random.default_rng(0)
    X = oracle.standardize(rng.normal(size=(6, 6)) @ rng.laplace(size=(6, 3000)))
    D = oracle.pairwise_measure(X)["D"]
    assert np.allclose(D, -D.T, atol=1e-14)
    assert np.all(np.diag(D) == 0)


def test_t_matches_eq2():
    rng = np.random.default_rng(1)
    X = oracle.standardize(rng.uniform(size=(4, 2000)) + 0.3 * rng.normal(size=(4, 2000)))
    meas = oracle.pairwise_measure(X)
    for i in range(4):
        for j in range(4):
            if i != j:
                r = oracle.residual(X[i], X[j])
                t = oracle.entropy(X[i]) - oracle.entropy(r / r.std())
                assert abs(meas["T"][i, j] - t) < 1e-12
                assert abs(meas["D"][i, j] - (meas["T"][j, i] - meas["T"][i, j])) < 1e-12


def test_permutation_equivariance():
    rng = np.random.default_rng(2)
    X = rng.laplace(size=(5, 4000))
    X[1] += 0.7 * X[0]
    X[3] -= 0.5 * X[1]
    perm = np.array([3, 0, 4, 1, 2])
    D = oracle.pairwise_measure(oracle.standardize(X))["D"]
    Dp = oracle.pairwise_measure(oracle.standardize(X[perm]))["D"]
    assert np.allclose(Dp, D[np.ix_(perm, perm)], atol=1e-12)


def test_affine_and_sign_invariance():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, size=(4, 3000))
    X[2] += 0.6 * X[0] - 0.4 * X[1]
    D = oracle.pairwise_measure(oracle.standardize(X))["D"]
    Y = X.copy()
    Y[0] = -3.0 * Y[0] + 11.0
    Y[2] = 0.25 * Y[2] - 4.0
    D2 = oracle.pairwise_measure(oracle.standardize(Y))["D"]
    assert np.allclose(D, D2, atol=1e-10)


def test_gaussian_data_gives_small_d():
    rng = np.random.default_rng(4)
    n = 200_000
    X = rng.normal(size=(4, n))
    X[1] += 0.8 * X[0]
    D = oracle.pairwise_measure(oracle.standardize(X))["D"]
    # both moments deviate from their Gaussian values by O(n^-1/2) and H
    # depends on them quadratically, so |D| = O(1/n)
    assert np.max(np.abs(D)) < 20.0 / n


def test_standardize_ddof0():
    rng = np.random.default_rng(5)
    X = rng.normal(3.0, 2.0, size=(3, 101))
    Z = oracle.standardize(X)
    assert np.allclose(Z.mean(axis=1), 0, atol=1e-14)
    assert np.allclose(np.mean(Z * Z, axis=1), 1, atol=1e-14)
