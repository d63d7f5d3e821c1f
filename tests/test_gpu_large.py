"""GPU parity at full size against stored oracle values: all 256 series of the
mixed-size batch through vl_fit_batched, and the finance-shaped stretch
series (m = 800 and 1600, n = 5000) through the step-by-step calls; and the
ordering above 2048 variables (four per thread) and at the maximum size
against the oracle's Algorithm 1 on random antisymmetric D, and the
pairwise measure at the maximum size on sampled pairs.

The stored values (tests/golden/*_oracle.json.gz) were written by
tests/golden/make_golden.py from the FP64 oracle alone: per series the whole
Algorithm 1 order with every step's relative score gap, all variable
entropies, and seeded samples of D, E_r, M, B0 and B_tau.

Tolerances as in test_gpu_parity.py: D within 1e-5 of max|D|, H within 1e-5
of max(|H|, H_nu), M within 1e-5, B0 and B_tau within 1e-4 absolute; the
order identical to the oracle's at every step before the first step whose
oracle gap is <= 1e-6 (from there on, the samples of B0 only hold for the
oracle's order and are not compared).  The certified mixed path meets the
order rule; the plain mixed path is also run and its agreement reported.
"""
import gzip
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
D_REL, H_REL, B_ABS, M_ABS, GAP = 1e-5, 1e-5, 1e-4, 1e-5, 1e-6


def _load(name):
    with gzip.open(os.path.join(GOLDEN, name), "rt") as f:
        return json.load(f)


def _report(key, **vals):
    out = os.environ.get("VL_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "parity_errors.jsonl"), "a") as f:
            f.write(json.dumps({"case": key, **{k: float(v) for k, v in vals.items()}}) + "\n")


def _order_prefix(g):
    """Steps before the first oracle near tie (gap <= 1e-6), and whether there
    is none at all (then the whole order must be identical)."""
    gaps = g["gaps"]
    for k, v in enumerate(gaps):
        if v <= GAP:
            return k, False
    return len(g["order"]), True


def _check_series(g, order, D, M, B0, Bt, Hx=None, Hr=None):
    """Returns the per-series errors; asserts the tolerances."""
    m = g["m"]
    assert sorted(order.tolist()) == list(range(m))
    k, whole = _order_prefix(g)
    same = order[:k].tolist() == g["order"][:k]
    assert same, ("order differs before the first oracle near tie", k)
    dmax = g["D_maxabs"]
    d_err = max(abs(D[i, j] - v) for i, j, v in g["D"]) / dmax
    assert d_err <= D_REL, d_err
    m_err = max(abs(M[t, i, kk] - v) for t, i, kk, v in g["M"])
    assert m_err <= M_ABS, m_err
    errs = {"d_rel": d_err, "m_err": m_err, "prefix": k}
    if whole:
        b_err = max(abs(B0[i, j] - v) for i, j, v in g["B0"])
        t_err = max(abs(Bt[t, i, kk] - v) for t, i, kk, v in g["Btau"])
        assert b_err <= B_ABS and t_err <= B_ABS, (b_err, t_err)
        errs.update(b0_err=b_err, btau_err=t_err)
    if Hx is not None:
        ex = np.array(g["Ex"])
        hx_err = np.max(np.abs(Hx - ex) / np.maximum(np.abs(ex), oracle.H_GAUSS))
        hr_err = max(abs(Hr[i, j] - v) / max(abs(v), oracle.H_GAUSS) for i, j, v in g["Er"])
        assert hx_err <= H_REL and hr_err <= H_REL, (hx_err, hr_err)
        errs.update(hx=hx_err, hr=hr_err)
    return errs


@pytest.fixture(scope="module")
def h(vl):
    handle = vl.Handle(0)
    yield handle
    handle.close()


def test_batched_all_256_series_against_the_oracle(vl, h):
    """vl_fit_batched on the 256 seeded series (m 20..400, n 250..5000, p
    1..3) in certified mixed precision: every series at the oracle's
    tolerances and order rule.  The plain mixed batch runs too; its orders
    are reported (they may swap near ties the certified path re-decides)."""
    gold = _load("batched_oracle.json.gz")["series"]
    insts = synth.make_batched(256, synth.config_seed(4))
    assert len(gold) == len(insts) == 256
    dicts = []
    for inst, g in zip(insts, gold):
        assert (inst.m, inst.n, inst.p) == (g["m"], g["n"], g["p"])
        o = vl.alloc_outputs(inst.m, inst.p)
        o["X"] = torch.from_numpy(inst.X).cuda()
        o["p"] = inst.p
        dicts.append(o)
    status = vl.vl_fit_batched(h, dicts, "mixed_certified")
    assert all(s == 0 for s in status), status
    worst = {}
    for k, (o, g) in enumerate(zip(dicts, gold)):
        errs = _check_series(g, o["order"].cpu().numpy(), o["D"].cpu().numpy(),
                             o["M"].cpu().numpy(), o["B0"].cpu().numpy(),
                             o["Btau"].cpu().numpy())
        for key, v in errs.items():
            worst[key] = max(worst.get(key, 0.0), v) if key != "prefix" else 0.0
    # the plain mixed batch: how many series keep the oracle's order
    plain = []
    for o in dicts:
        o2 = {key: (torch.empty_like(v) if torch.is_tensor(v) and key != "X" else v)
              for key, v in o.items()}
        plain.append(o2)
    vl.vl_fit_batched(h, plain, "mixed")
    agree = sum(int(o2["order"].cpu().numpy()[:_order_prefix(g)[0]].tolist()
                    == g["order"][:_order_prefix(g)[0]]) for o2, g in zip(plain, gold))
    _report("batched 256 certified", mixed_plain_agree=agree, **worst)


@pytest.mark.parametrize("m", [800, 1600])
@pytest.mark.parametrize("prec", ["mixed_certified", "fp64"])
def test_stretch_series_against_the_oracle(vl, h, m, prec):
    """The stretch sizes (finance-shaped, n = 5000): m = 800 runs the
    one-cluster Cholesky, m = 1600 the blocked multi-kernel one, the
    two-variables-per-thread ordering and the column-sweep triangular
    solves."""
    g = _load(f"stretch_m{m}_oracle.json.gz")["series"][0]
    inst = synth.make_config("finance", m=m, n=5000)
    X = torch.from_numpy(inst.X).cuda()
    out = vl.fit(h, X, inst.p, prec=prec, steps=True)
    errs = _check_series(g, out["order"].cpu().numpy(), out["D"].cpu().numpy(),
                         out["M"].cpu().numpy(), out["B0"].cpu().numpy(),
                         out["Btau"].cpu().numpy(), out["Hx"].cpu().numpy(),
                         out["Hr"].cpu().numpy())
    if "cert_stats" in out:
        st = out["cert_stats"].cpu().numpy()
        errs.update(flagged=st[0], pairs=st[1], changed=st[2], unverified=st[3])
    _report(f"stretch m={m} {prec}", **errs)


def test_causal_order_four_variables_per_thread(vl):
    """m = 2100 (above 2048, where the search holds four variables per
    thread): the whole order equals Algorithm 1's on the same D."""
    h = vl.Handle(0)
    try:
        m = 2100
        rng = np.random.default_rng(2100)
        A = rng.normal(size=(m, m))
        D = A - A.T
        order = torch.empty(m, dtype=torch.int32, device="cuda")
        vl.vl_causal_order(h, torch.from_numpy(D).cuda(), order)
        h.sync()
        ref = oracle.order_heuristic(D)
        assert [int(c) for c in order.cpu().numpy()] == [int(c) for c in ref["order"]]
    finally:
        h.close()


def test_causal_order_at_the_maximum_size(vl):
    """m = VL_MAX_M = 4096 (the oracle's whole search would take minutes):
    the order is a permutation, and at the first 10 and the last 300 steps,
    walked over the GPU's own remaining sets, the pick minimises the oracle's
    scores of Eq. 3 (or lies within 1e-6 relative of the minimum)."""
    h = vl.Handle(0)
    try:
        m = 4096
        rng = np.random.default_rng(4096)
        A = rng.normal(size=(m, m))
        D = A - A.T
        order_t = torch.empty(m, dtype=torch.int32, device="cuda")
        vl.vl_causal_order(h, torch.from_numpy(D).cuda(), order_t)
        h.sync()
        order = [int(c) for c in order_t.cpu().numpy()]
        assert sorted(order) == list(range(m))
        left = np.ones(m, dtype=bool)
        checked = 0
        for k, c in enumerate(order):
            if k < 10 or k >= m - 300:
                scores = oracle.scores_over(D, np.nonzero(left)[0])
                smin = min(scores.values())
                assert scores[c] - smin <= GAP * max(abs(smin), abs(scores[c]), 1e-300), k
                checked += 1
            left[c] = False
        assert checked == 310
    finally:
        h.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_pairwise_measure_at_the_maximum_size(vl, prec):
    """m = VL_MAX_M = 4096 variables, n = 300 samples (a ragged sample tail):
    every variable entropy against the oracle's, and D at 300 seeded pairs,
    each computed by the oracle from its own residual (within D_REL of the
    largest |D| of the whole matrix, taken from the GPU's D since the
    oracle's is too large to form here; H within H_REL of max(|H|, H_nu))."""
    h = vl.Handle(0)
    try:
        m, n = 4096, 300
        rng = np.random.default_rng(43)
        E = rng.laplace(size=(m, n))
        E[1:] += 0.4 * E[:-1]
        Et = torch.from_numpy(E).cuda()
        f64 = dict(dtype=torch.float64, device="cuda")
        Hx, Hr, D = torch.empty(m, **f64), torch.empty((m, m), **f64), torch.empty((m, m), **f64)
        vl.vl_pairwise_measure(h, Et, prec, Hx, Hr, D)
        h.sync()
        Hx, D = Hx.cpu().numpy(), D.cpu().numpy()
        Xs = oracle.standardize(E)
        ex = np.array([oracle.entropy(Xs[i]) for i in range(m)])
        assert np.max(np.abs(Hx - ex) / np.maximum(np.abs(ex), oracle.H_GAUSS)) <= H_REL
        pairs = rng.choice(m, size=(300, 2))
        pairs = pairs[pairs[:, 0] != pairs[:, 1]]
        ref, got = [], []
        for i, j in pairs:
            rij = oracle.residual(Xs[i], Xs[j])
            rji = oracle.residual(Xs[j], Xs[i])
            ref.append(ex[j] + oracle.entropy(rij / rij.std()) - ex[i]
                       - oracle.entropy(rji / rji.std()))
            got.append(D[i, j])
        ref, got = np.array(ref), np.array(got)
        assert np.max(np.abs(got - ref)) <= D_REL * np.max(np.abs(D))
        assert np.allclose(D, -D.T, atol=1e-15 + 1e-12 * np.max(np.abs(D)))
    finally:
        h.close()
