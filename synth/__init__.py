"""Seeded synthetic LiNGAM-VAR series.

This module only *draws data*: a random instantaneous DAG B0, reduced-form VAR
matrices M_tau, non-Gaussian shocks, and the simulated series
    x_t = sum_tau M_tau x_{t-tau} + (I - B0)^{-1} e_t .
It contains none of the estimation method (no VAR fit, no entropy, no ordering),
so the CUDA path and the FP64 oracle can both be fed from it without sharing
any of the method's arithmetic.

The model is the VarLiNGAM model (Section 2.1 of the paper; x_t has
instantaneous effects B0 and lagged effects B_tau = (I - B0) M_tau).  The
workload shapes stand in for the paper's data sets, which are not available:
  * "pr1"    m=10,  n=1000,  p=1  uniform noise       (small reference case)
  * "fmri"   m=50,  n=200,   p=1  sign(g)|g|^1.5 noise (fMRI, Table 1)
  * "server" m=120, n=10000, p=3  Laplace noise        (IT monitoring, Table 1)
  * "finance" m=400, n=2500, p=1  Student-t3 noise     (S&P500, Table 2)
  * "batched" 256 independent series of mixed sizes

Arrays are returned as float64, variable-major: X[i, t] is variable i at time t.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

BASE_SEED = 2409055
BURN_IN = 200

NOISE_KINDS = ("uniform", "powgauss", "laplace", "t3", "gauss")


@dataclasses.dataclass
class Instance:
    """One simulated series plus the ground truth it was drawn from."""

    X: np.ndarray  # (m, n) float64, variable-major
    B0: np.ndarray  # (m, m) true instantaneous effects, B0[i, j]: j -> i
    M: np.ndarray  # (p, m, m) true reduced-form VAR matrices, M[tau-1][i, k]
    perm: np.ndarray  # (m,) a true causal order (causes first)
    noise: str
    seed: int

    @property
    def m(self) -> int:
        return self.X.shape[0]

    @property
    def n(self) -> int:
        return self.X.shape[1]

    @property
    def p(self) -> int:
        return self.M.shape[0]

    def Btau(self) -> np.ndarray:
        """True lagged effects B_tau = (I - B0) M_tau."""
        eye = np.eye(self.m)
        return np.stack([(eye - self.B0) @ Mt for Mt in self.M])


def draw_noise(rng: np.random.Generator, kind: str, size) -> np.ndarray:
    """Unit-variance, zero-mean shocks of the named family."""
    if kind == "uniform":
        return rng.uniform(-math.sqrt(3.0), math.sqrt(3.0), size=size)
    if kind == "laplace":
        return rng.laplace(0.0, 1.0 / math.sqrt(2.0), size=size)
    if kind == "t3":
        return rng.standard_t(3.0, size=size) / math.sqrt(3.0)
    if kind == "powgauss":
        g = rng.standard_normal(size=size)
        # E|g|^3 = 2 sqrt(2/pi) for a standard normal g
        return np.sign(g) * np.abs(g) ** 1.5 / math.sqrt(2.0 * math.sqrt(2.0 / math.pi))
    if kind == "gauss":
        return rng.standard_normal(size=size)
    raise ValueError(f"unknown noise kind {kind!r}")


def draw_dag(rng: np.random.Generator, m: int, edge_prob: float, lo: float, hi: float):
    """Random DAG under a random causal order perm: edge perm[a] -> perm[b]
    (a < b) with probability edge_prob, weight +-U[lo, hi]."""
    perm = rng.permutation(m)
    edge = rng.random((m, m)) < edge_prob
    mag = rng.uniform(lo, hi, size=(m, m))
    sgn = np.where(rng.random((m, m)) < 0.5, -1.0, 1.0)
    a_idx, b_idx = np.triu_indices(m, 1)  # a < b in the causal order
    keep = edge[a_idx, b_idx]
    B0 = np.zeros((m, m))
    B0[perm[b_idx[keep]], perm[a_idx[keep]]] = (mag * sgn)[a_idx, b_idx][keep]
    return B0, perm


def companion_radius(M: np.ndarray) -> float:
    """Spectral radius of the VAR(p) companion matrix of M (p, m, m)."""
    p, m, _ = M.shape
    C = np.zeros((m * p, m * p))
    C[:m, :] = np.concatenate(list(M), axis=1)
    if p > 1:
        C[m:, :-m] = np.eye(m * (p - 1))
    return float(np.max(np.abs(np.linalg.eigvals(C))))


def scale_to_radius(M: np.ndarray, target: float) -> np.ndarray:
    """Scale M_tau <- c^tau M_tau.  This multiplies every companion eigenvalue
    by c, so c = target / current radius hits the target exactly."""
    r = companion_radius(M)
    if r == 0.0:
        return M.copy()
    c = target / r
    return np.stack([c ** (tau + 1) * M[tau] for tau in range(M.shape[0])])


def draw_var(rng: np.random.Generator, m: int, p: int, kind: str, radius: float,
             density: float = 1.0, lo: float = 0.05, hi: float = 0.3, sd: float = 0.02):
    """Reduced-form VAR matrices.  kind 'unif': +-U[lo, hi] entries (kept with
    probability `density`); kind 'normal': N(0, sd^2) entries."""
    M = np.zeros((p, m, m))
    for tau in range(p):
        if kind == "unif":
            mag = rng.uniform(lo, hi, size=(m, m))
            sgn = np.where(rng.random(size=(m, m)) < 0.5, -1.0, 1.0)
            keep = rng.random(size=(m, m)) < density
            M[tau] = mag * sgn * keep
        elif kind == "normal":
            M[tau] = rng.normal(0.0, sd, size=(m, m))
        else:
            raise ValueError(kind)
    return scale_to_radius(M, radius)


def simulate(rng: np.random.Generator, B0: np.ndarray, M: np.ndarray, n: int,
             noise: str, burn_in: int = BURN_IN) -> np.ndarray:
    """x_t = sum_tau M_tau x_{t-tau} + (I - B0)^{-1} e_t from a zero initial
    state; the first burn_in steps are discarded."""
    p, m, _ = M.shape
    A = np.linalg.inv(np.eye(m) - B0)
    total = n + burn_in
    e = draw_noise(rng, noise, (total, m))
    shocks = e @ A.T  # row t: (I - B0)^{-1} e_t
    x = np.zeros((total + p, m))
    for t in range(total):
        acc = shocks[t].copy()
        for tau in range(p):
            acc += M[tau] @ x[t + p - 1 - tau]
        x[t + p] = acc
    return np.ascontiguousarray(x[p + burn_in:].T)


def make_instance(m: int, n: int, p: int, seed: int, noise: str = "uniform",
                  edge_prob: float = 0.3, w_lo: float = 0.1, w_hi: float = 0.5,
                  var_kind: str = "unif", radius: float = 0.8, density: float = 1.0,
                  var_lo: float = 0.05, var_hi: float = 0.3, var_sd: float = 0.02) -> Instance:
    rng = np.random.Generator(np.random.PCG64(seed))
    B0, perm = draw_dag(rng, m, edge_prob, w_lo, w_hi)
    M = draw_var(rng, m, p, var_kind, radius, density, var_lo, var_hi, var_sd)
    X = simulate(rng, B0, M, n, noise)
    return Instance(X=X, B0=B0, M=M, perm=perm, noise=noise, seed=seed)


def batched_edge_prob(m: int) -> float:
    """Edge probability for the mixed-size batch: the small reference case's
    0.3 at m=10 keeps the expected degree 0.3*(m-1)=2.7 for larger m."""
    return min(0.3, 2.7 / max(m - 1, 1))


# ---------------------------------------------------------------- workloads
CONFIGS = ("pr1", "fmri", "server", "finance", "batched")


def config_seed(idx: int) -> int:
    return BASE_SEED + 1000 * idx


def make_config(name: str, m: Optional[int] = None, n: Optional[int] = None):
    """The named workload.  Returns an Instance, or for 'batched' a list of
    Instances.  `m`/`n` override the size for 'finance' (the m=800/1600,
    n=5000 sweep)."""
    if name == "pr1":
        return make_instance(10, 1000, 1, config_seed(0), "uniform", 0.3, 0.1, 0.5,
                             "unif", 0.8)
    if name == "fmri":
        return make_instance(50, 200, 1, config_seed(1), "powgauss", 0.1, 0.1, 0.6,
                             "unif", 0.7)
    if name == "server":
        return make_instance(120, 10000, 3, config_seed(2), "laplace", 0.05, 0.1, 0.5,
                             "unif", 0.9, density=0.05)
    if name == "finance":
        mm = 400 if m is None else m
        nn = 2500 if n is None else n
        seed = config_seed(3) + (0 if m is None else mm)
        return make_instance(mm, nn, 1, seed, "t3", 0.02, 0.05, 0.4, "normal", 0.5)
    if name == "batched":
        return make_batched(256, config_seed(4))
    raise ValueError(f"unknown workload {name!r}")


def draw_batched_shapes(count: int, seed: int):
    """(m, n, p, noise, redraws) per instance; (m, n, p) is redrawn until
    n - p >= 2 (m p + 1) so every VAR fit is well posed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        redraws = 0
        while True:
            m = int(rng.integers(20, 401))
            n = int(rng.integers(250, 5001))
            p = int(rng.integers(1, 4))
            if n - p >= 2 * (m * p + 1):
                break
            redraws += 1
        noise = ("uniform", "laplace", "t3")[int(rng.integers(0, 3))]
        out.append((m, n, p, noise, redraws))
    return out


def make_batched(count: int, seed: int, max_m: Optional[int] = None,
                 max_n: Optional[int] = None) -> List[Instance]:
    """Mixed-size batch: m~U{20..400}, n~U{250..5000}, p~U{1..3}, noise from
    {uniform, Laplace, t3}; otherwise as the small reference case."""
    shapes = draw_batched_shapes(count, seed)
    insts = []
    for k, (m, n, p, noise, _) in enumerate(shapes):
        if max_m is not None:
            m = min(m, max_m)
        if max_n is not None:
            n = min(n, max_n)
            if n - p < 2 * (m * p + 1):
                n = 2 * (m * p + 1) + p
        insts.append(make_instance(m, n, p, seed + 1 + k, noise, batched_edge_prob(m),
                                   0.1, 0.5, "unif", 0.8))
    return insts
