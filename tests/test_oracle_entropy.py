"""Pins for the entropy approximation of the oracle (Section 3, step 3).

The constants are checked against quantities computed here from their
definition (Gauss-Hermite quadrature of Gaussian integrals, closed forms), not
against the constants retyped."""
import math

import numpy as np
from numpy.polynomial.hermite_e import hermegauss
from scipy import integrate

import oracle


def _gauss_expect(f, deg=200):
    x, w = hermegauss(deg)
    w = w / math.sqrt(2.0 * math.pi)
    return float(np.sum(w * f(x)))


def _logcosh_ref(x):
    return np.log(np.cosh(x))


def test_h_gauss_is_gaussian_entropy():
    # differential entropy of N(0,1): integral of -phi log phi, by quadrature
    def integrand(x):
        log_phi = -0.5 * x * x - 0.5 * math.log(2.0 * math.pi)
        return -math.exp(log_phi) * log_phi

    val, _ = integrate.quad(integrand, -40, 40, limit=200)
    assert abs(val - oracle.H_GAUSS) < 1e-10


def test_gamma_is_gaussian_mean_of_logcosh():
    g = _gauss_expect(_logcosh_ref)
    assert abs(g - 0.3745672075) < 1e-9  # quadrature itself converged
    assert abs(g - oracle.ENTROPY_GAMMA) < 5e-6


def _orthonormal_weight(G, even):
    """1 / (2 Var) of G after removing its Gaussian projection on {1, u, u^2}:
    the weight the maximum-entropy approximation gives (E G(u) - E G(nu))^2."""
    EG = _gauss_expect(G)
    EG2 = _gauss_expect(lambda x: G(x) ** 2)
    if even:
        cov = _gauss_expect(lambda x: x * x * G(x)) - EG
        var = EG2 - EG * EG - cov * cov / 2.0  # Var(u^2) = 2
    else:
        cov = _gauss_expect(lambda x: x * G(x))
        var = EG2 - cov * cov  # Var(u) = 1
    return 1.0 / (2.0 * var)


def test_k2_closed_form_and_quadrature():
    closed = 36.0 / (8.0 * math.sqrt(3.0) - 9.0)
    quad = _orthonormal_weight(lambda x: x * np.exp(-0.5 * x * x), even=False)
    assert abs(quad - closed) < 1e-9
    assert abs(oracle.ENTROPY_K2 - closed) / closed < 2e-5


def test_k1_reproduced_by_quadrature():
    # The literature value 79.047 is reproduced to 4e-4 relative; a typo in
    # any of its leading digits would fail this.
    quad = _orthonormal_weight(_logcosh_ref, even=True)
    assert abs(quad - oracle.ENTROPY_K1) / oracle.ENTROPY_K1 < 1e-3


def test_entropy_of_large_gaussian_sample():
    rng = np.random.default_rng(1)
    u = rng.standard_normal(2_000_000)
    u = (u - u.mean()) / u.std()
    assert abs(oracle.entropy(u) - oracle.H_GAUSS) < 2e-4


def _h_from_moments(a, b):
    return (oracle.H_GAUSS - oracle.ENTROPY_K1 * (a - oracle.ENTROPY_GAMMA) ** 2
            - oracle.ENTROPY_K2 * b * b)


def test_entropy_of_uniform_matches_quadrature():
    h = math.sqrt(3.0)
    a, _ = integrate.quad(lambda x: math.log(math.cosh(x)) / (2 * h), -h, h)
    # the odd moment of a symmetric law is zero
    expect = _h_from_moments(a, 0.0)
    rng = np.random.default_rng(2)
    u = rng.uniform(-h, h, 2_000_000)
    u = (u - u.mean()) / u.std()
    assert abs(oracle.entropy(u) - expect) < 5e-4
    assert expect < oracle.H_GAUSS - 1e-3  # non-Gaussian => lower entropy


def test_entropy_of_skewed_law_uses_odd_moment():
    # Exponential(1) - 1 is skewed: its E[u exp(-u^2/2)] is non-zero, so the
    # k2 term must be present.  Moments by quadrature of the density e^{-(u+1)}.
    f = lambda u: math.exp(-(u + 1.0))
    a, _ = integrate.quad(lambda u: math.log(math.cosh(u)) * f(u), -1, 60, limit=200)
    b, _ = integrate.quad(lambda u: u * math.exp(-0.5 * u * u) * f(u), -1, 60, limit=200)
    assert abs(b) > 0.05
    expect = _h_from_moments(a, b)
    rng = np.random.default_rng(3)
    u = rng.exponential(1.0, 4_000_000) - 1.0
    u = (u - u.mean()) / u.std()
    assert abs(oracle.entropy(u) - expect) < 2e-3


def test_logcosh_matches_numpy_and_the_stable_form():
    u = np.linspace(-20, 20, 4001)
    ref = np.log(np.cosh(u))
    assert np.max(np.abs(oracle.logcosh(u) - ref)) < 1e-12
    # |u| + log1p(exp(-2|u|)) - log 2: the overflow-free form a kernel may use
    alt = np.abs(u) + np.log1p(np.exp(-2 * np.abs(u))) - math.log(2.0)
    assert np.max(np.abs(alt - ref)) < 1e-12
