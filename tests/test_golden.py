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


def _sampled(name):
    import gzip

    with gzip.open(os.path.join(GOLDEN, name), "rt") as f:
        return json.load(f)


def test_stored_batch_values_are_the_oracles():
    """The stored values of the 256-series batch (written by make_golden.py
    from the oracle) for the three cheapest series, recomputed here: the
    fixture holds the oracle's order, gaps and samples."""
    import sys

    sys.path.insert(0, GOLDEN)
    import make_golden

    gold = _sampled("batched_oracle.json.gz")["series"]
    assert len(gold) == 256
    cheapest = sorted(range(256), key=lambda k: gold[k]["m"] ** 2 * gold[k]["n"])[:3]
    for k in cheapest:
        rec = make_golden._batched_one(k)
        g = gold[k]
        assert rec["order"] == g["order"]
        np.testing.assert_allclose(rec["gaps"], g["gaps"], rtol=1e-9, atol=1e-15)
        for key in ("Ex", "D", "Er", "M", "B0", "Btau"):
            np.testing.assert_allclose(np.array(rec[key], dtype=float), np.array(g[key], dtype=float),
                                       rtol=1e-10, atol=1e-13, err_msg=key)


def test_stored_stretch_values_are_consistent():
    for m in (800, 1600):
        g = _sampled(f"stretch_m{m}_oracle.json.gz")["series"][0]
        assert g["m"] == m and g["n"] == 5000 and sorted(g["order"]) == list(range(m))
        assert len(g["gaps"]) == m - 1 and len(g["Ex"]) == m
        # D is antisymmetric: every sampled entry and the stored maximum agree in size
        assert max(abs(v) for _, _, v in g["D"]) <= g["D_maxabs"] * (1 + 1e-12)
