"""Writes the stored expected values of tests/golden/ from the FP64 oracle.

Only the oracle (and the seeded input generator) is called here: no value in
these fixtures comes from the CUDA path.  The fixtures pin the oracle against
silent change: a later change of its arithmetic shows up as a fixture
difference, and its commit names the passage of the paper (or the reading of
it) that justifies the new values.

    python tests/golden/make_golden.py              # pr1_oracle.json
    python tests/golden/make_golden.py --batched    # batched_oracle.json.gz
    python tests/golden/make_golden.py --stretch    # stretch_m800/m1600_oracle.json.gz

The large fixtures (the 256-series mixed batch and the m = 800 / 1600,
n = 5000 finance-shaped series) hold, per series, the whole causal order of
Algorithm 1 with the relative score gap of every step, all variable
entropies E_x, and seeded samples of D, E_r, M, B0 and B_tau (with their
indices), because the full m x m tables would be tens of megabytes.  They are
computed on a process pool (each worker runs the oracle's own functions).
"""
from __future__ import annotations

import argparse
import gzip
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

N_SAMPLE = 64


def pr1_values():
    """The small workload (m=10, n=1000, p=1, uniform shocks, seed 2409055):
    Sec. 4.1 VAR fit, Sec. 3 steps 1-3 (Eqs. 1-2) measure, Algorithm 1 order,
    the iterative search of Sec. 3 (Eq. 4), B0 by predecessor regression and
    B_tau = (I - B0) M_tau."""
    inst = synth.make_config("pr1")
    res = oracle.varlingam(inst.X, inst.p)
    Xs = oracle.standardize(res["E"])
    std = oracle.order_standard(Xs)
    heur = oracle.order_heuristic(res["D"])
    return {
        "workload": "pr1: m=10, n=1000, p=1, uniform shocks, seed 2409055",
        "written_by": "tests/golden/make_golden.py (oracle only)",
        "M": res["M"].tolist(),
        "Ex": res["Ex"].tolist(),
        "D": res["D"].tolist(),
        "order_heuristic": [int(c) for c in res["order"]],
        "gaps_heuristic": [oracle.relative_gap(st["scores"]) for st in heur["steps"][:-1]],
        "order_standard": [int(c) for c in std["order"]],
        "gaps_standard": [oracle.relative_gap(st["scores"]) for st in std["steps"][:-1]],
        "B0": res["B0"].tolist(),
        "Btau": res["Btau"].tolist(),
    }


def _f(x: float) -> float:
    """12 significant digits: far below every tolerance the tests apply."""
    return float(f"{x:.12e}")


def sampled_record(X, p, meas, b0_route, seed, n_sample=N_SAMPLE):
    """The per-series record of a large fixture from the oracle's results:
    M, E by the VAR fit (Sec. 4.1), the measure `meas` (Sec. 3 steps 1-3,
    Eqs. 1-2), Algorithm 1's order and step gaps (Eq. 3), B0 on that order by
    `b0_route` and B_tau = (I - B0) M_tau."""
    M, E = oracle.var_ols(X, p)
    D = meas["D"]
    m = D.shape[0]
    od = oracle.order_heuristic(D)
    order = od["order"]
    gaps = [oracle.relative_gap(st["scores"]) for st in od["steps"][:-1]]
    B0 = b0_route(E, order)
    Bt = oracle.btau(B0, M)
    rng = np.random.default_rng(seed)
    ii = rng.integers(0, m, size=n_sample)
    jj = (ii + rng.integers(1, m, size=n_sample)) % m  # off the diagonal
    imax, jmax = np.unravel_index(np.argmax(np.abs(D)), D.shape)
    pos = np.empty(m, dtype=np.int64)
    pos[order] = np.arange(m)
    # B0 entries where the order allows an edge (predecessor j of i), and a
    # few where it forbids one (those must be exactly zero)
    a = rng.integers(1, m, size=n_sample)
    b = (rng.random(n_sample) * a).astype(np.int64)
    bi, bj = order[a], order[b]
    zi, zj = order[b[: n_sample // 4]], order[a[: n_sample // 4]]
    tt = rng.integers(0, p, size=n_sample)
    ti = rng.integers(0, m, size=n_sample)
    tk = rng.integers(0, m, size=n_sample)
    return {
        "m": int(m), "n": int(X.shape[1]), "p": int(p),
        "order": [int(c) for c in order],
        "gaps": [_f(g) for g in gaps],
        "Ex": [_f(v) for v in meas["Ex"]],
        "D_maxabs": _f(float(np.abs(D).max())),
        "D": [[int(i), int(j), _f(D[i, j])] for i, j in zip(ii, jj)]
             + [[int(imax), int(jmax), _f(D[imax, jmax])]],
        "Er": [[int(i), int(j), _f(meas["Er"][i, j])] for i, j in zip(ii, jj)],
        "M_maxabs": _f(float(np.abs(M).max())),
        "M": [[int(t), int(i), int(k), _f(M[t, i, k])] for t, i, k in zip(tt, ti, tk)],
        "B0": [[int(i), int(j), _f(B0[i, j])] for i, j in zip(bi, bj)]
              + [[int(i), int(j), _f(B0[i, j])] for i, j in zip(zi, zj)],
        "Btau": [[int(t), int(i), int(k), _f(Bt[t, i, k])] for t, i, k in zip(tt, ti, tk)],
    }


def _batched_instance(k):
    """Series k of synth.make_batched(256, seed 2409055 + 4000), drawn alone."""
    seed = synth.config_seed(4)
    m, n, p, noise, _ = synth.draw_batched_shapes(256, seed)[k]
    return synth.make_instance(m, n, p, seed + 1 + k, noise, synth.batched_edge_prob(m),
                               0.1, 0.5, "unif", 0.8)


def _batched_one(k):
    """Worker: the whole oracle on series k of the 256-series batch."""
    inst = _batched_instance(k)
    M, E = oracle.var_ols(inst.X, inst.p)
    meas = oracle.pairwise_measure(oracle.standardize(E))
    rec = sampled_record(inst.X, inst.p, meas, oracle.b0_ols, inst.seed)
    rec["series"] = k
    rec["noise"] = inst.noise
    return rec


def batched_values(nproc):
    """All 256 series of the mixed-size batch (seed 2409055 + 4000): m in
    20..400, n in 250..5000, p in 1..3, uniform / Laplace / t3 shocks."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(nproc, initializer=_single_thread) as pool:
        recs = pool.map(_batched_one, range(256), chunksize=1)
    return {"workload": "batched: 256 series, m~U{20..400}, n~U{250..5000}, p~U{1..3}, "
                        "seed 2409055 + 4000",
            "written_by": "tests/golden/make_golden.py --batched (oracle only)",
            "b0_route": "oracle.b0_ols (predecessor least squares)",
            "series": recs}


def stretch_values(m, nproc):
    """The finance-shaped stretch series (Student-t3 shocks, p = 1, n = 5000,
    m = 800 or 1600): the measure's residual-entropy rows on a process pool
    (oracle.parallel, bit-identical to the serial oracle), B0 by the oracle's
    Cholesky route (b0_ldl; predecessor least squares at m = 1600 would take
    hours, and the two routes are pinned equal by the oracle tests)."""
    import multiprocessing as mp

    import oracle.parallel as op

    inst = synth.make_config("finance", m=m, n=5000)
    M, E = oracle.var_ols(inst.X, inst.p)
    with mp.get_context("spawn").Pool(nproc, initializer=_single_thread) as pool:
        meas = op.pairwise_measure_pool(oracle.standardize(E), pool, nproc)
    rec = sampled_record(inst.X, inst.p, meas, oracle.b0_ldl, inst.seed, n_sample=4 * N_SAMPLE)
    return {"workload": f"finance-like stretch: m={m}, n=5000, p=1, Student-t3 shocks, "
                        f"seed {inst.seed}",
            "written_by": "tests/golden/make_golden.py --stretch (oracle only)",
            "b0_route": "oracle.b0_ldl (Cholesky of the ordered covariance)",
            "series": [rec]}


def _single_thread():
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        import threadpoolctl

        threadpoolctl.threadpool_limits(1)
    except ImportError:
        pass


def _write_gz(name, obj):
    with gzip.open(os.path.join(HERE, name), "wt") as f:
        json.dump(obj, f, separators=(",", ":"))
        f.write("\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batched", action="store_true")
    ap.add_argument("--stretch", action="store_true")
    ap.add_argument("--procs", type=int, default=len(os.sched_getaffinity(0)))
    args = ap.parse_args()
    if not (args.batched or args.stretch):
        with open(os.path.join(HERE, "pr1_oracle.json"), "w") as f:
            json.dump(pr1_values(), f, indent=1)
            f.write("\n")
    if args.batched:
        _write_gz("batched_oracle.json.gz", batched_values(args.procs))
    if args.stretch:
        for m in (800, 1600):
            _write_gz(f"stretch_m{m}_oracle.json.gz", stretch_values(m, args.procs))


if __name__ == "__main__":
    main()
