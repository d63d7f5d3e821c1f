"""Stored expected values (tests/golden/): closed forms behind the entropy
approximation, and the FP64 oracle's own results on the small workload, written
by tests/golden/make_golden.py from the oracle alone (a change of the oracle's
arithmetic shows up here and must name the passage that justifies it)."""
import json
import math
import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _closed_forms():
    vals = {}
    for line in open(os.path.join(GOLDEN, "closed_forms.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            vals[name] = float(value)
    return vals


def test_closed_forms_and_the_oracle_constants():
    c = _closed_forms()
    assert c["H_nu"] == (1.0 + math.log(2.0 * math.pi)) / 2.0
    assert oracle.H_GAUSS == c["H_nu"]
    assert abs(c["k2"] - 36.0 / (8.0 * math.sqrt(3.0) - 9.0)) < 1e-15
    assert abs(oracle.ENTROPY_K2 - c["k2"]) < 5e-5          # the literature's 4 decimals
    x, w = np.polynomial.hermite_e.hermegauss(300)
    w = w / math.sqrt(2.0 * math.pi)
    assert abs((w * oracle.logcosh(x)).sum() - c["gamma"]) < 1e-13
    assert abs(oracle.ENTROPY_GAMMA - c["gamma"]) < 5e-6     # the literature's 5 digits
    assert abs((w * (x * np.exp(-x * x / 2)) ** 2).sum() - c["E_G2_sq"]) < 1e-13
    assert abs(c["E_G2_sq"] - 1.0 / (3.0 * math.sqrt(3.0))) < 1e-16


def test_oracle_reproduces_its_stored_small_workload_values():
    g = json.load(open(os.path.join(GOLDEN, "pr1_oracle.json")))
    inst = synth.make_config("pr1")
    res = oracle.varlingam(inst.X, inst.p)
    for key in ("M", "Ex", "D", "B0", "Btau"):
        np.testing.assert_allclose(res[key], np.array(g[key]), rtol=1e-9, atol=1e-12,
                                   err_msg=key)
    assert [int(c) for c in res["order"]] == g["order_heuristic"]
    std = oracle.order_standard(oracle.standardize(res["E"]))
    assert [int(c) for c in std["order"]] == g["order_standard"]
    gaps = [oracle.relative_gap(st["scores"]) for st in std["steps"][:-1]]
    np.testing.assert_allclose(gaps, g["gaps_standard"], rtol=1e-7)
