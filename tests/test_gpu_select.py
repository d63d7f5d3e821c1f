"""GPU lag selection (vl_var_select) against the oracle's var_select: every
candidate p = 1..p_max fitted on the same T = n - p_max equations, the
criterion values AIC / BIC / HQ and the chosen p.

Tolerances: FP64 path within 1e-9 of the oracle's values (relative to
max(1, |value|)); mixed path within 1e-5 m absolute (ln det of an m x m
covariance whose entries carry FP32-level relative error is off by about m
times that error, far below the penalty step 2 m^2 / T between candidates).
The chosen p must be the oracle's unless the oracle's best two values lie
within that tolerance of each other."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

CASES = [("pr1", 4), ("fmri", 2), ("server", 4), ("finance", 2)]


@pytest.fixture(scope="module")
def h(vl):
    handle = vl.Handle(0)
    yield handle
    handle.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("criterion", ["aic", "bic", "hq"])
@pytest.mark.parametrize("name,p_max", CASES)
def test_lag_selection_matches_the_oracle(vl, h, name, p_max, criterion, prec):
    inst = synth.make_config(name)
    ref = oracle.var_select(inst.X, p_max, criterion)
    X = torch.from_numpy(inst.X).cuda()
    values = torch.empty(p_max, dtype=torch.float64, device="cuda")
    p_best = torch.empty(1, dtype=torch.int32, device="cuda")
    vl.vl_var_select(h, X, p_max, criterion, prec, values, p_best)
    h.sync()
    got = values.cpu().numpy()
    want = np.array(ref["values"])
    m = inst.X.shape[0]
    if prec == "fp64":
        err = np.max(np.abs(got - want) / np.maximum(1.0, np.abs(want)))
        tol = 1e-9
    else:
        err = np.max(np.abs(got - want))
        tol = 1e-5 * m
    assert err <= tol, (err, tol, got, want)
    srt = np.sort(want)
    if len(srt) < 2 or srt[1] - srt[0] > tol:
        assert int(p_best.item()) == ref["p"], (int(p_best.item()), ref["p"])
    else:
        assert int(p_best.item()) in {1 + int(i) for i in np.argsort(want)[:2]}


def test_lag_selection_rejects_too_short_series(vl, h):
    """n - p_max must exceed m (p_max + 1): the host answers VL_ERR_RANK."""
    X = torch.zeros(10, 40, dtype=torch.float64, device="cuda")
    values = torch.empty(3, dtype=torch.float64, device="cuda")
    p_best = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(vl.VLError) as e:
        vl.vl_var_select(h, X, 3, "bic", "fp64", values, p_best)
    assert e.value.code == 3  # VL_ERR_RANK
