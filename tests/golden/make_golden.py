"""Writes the stored expected values of tests/golden/ from the FP64 oracle.

Only the oracle (and the seeded input generator) is called here: no value in
these fixtures comes from the CUDA path.  The fixtures pin the oracle against
silent change: a later change of its arithmetic shows up as a fixture
difference, and its commit names the passage of the paper (or the reading of
it) that justifies the new values.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


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


def main():
    with open(os.path.join(HERE, "pr1_oracle.json"), "w") as f:
        json.dump(pr1_values(), f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
