"""GPU bootstrap (vl_bootstrap_resample, vl_bootstrap) against the oracle's
moving-block bootstrap on the same seeds.

Resamples: bit-exact (a gather of FP64 values at indices the oracle computes
from the same counter-based generator), for ragged lengths, block lengths 1
and n, several seeds including ones near 2^64 (the generator's wrap-around),
and independent of how the resamples are grouped into calls.

Probabilities: the edge and order counts of every (i, j) equal the oracle's
except where a resample is ambiguous: its search had a relative score gap at
or below GAP (its order may legitimately differ, and with it its B0), or its
|B0[i, j]| lies within B_MARGIN of the threshold.  Each such resample may move
a count by one.  GAP = 1e-6 for the FP64 and certified paths (the parity rule
of the single fits), 1e-3 for the plain mixed path (whose ordering follows its
own FP32-level measure); B_MARGIN = 1e-8 (FP64) and 1e-4 (mixed: the B0
tolerance of the single fits)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

GAP = {"fp64": 1e-6, "mixed_certified": 1e-6, "mixed": 1e-3}
B_MARGIN = {"fp64": 1e-8, "mixed_certified": 1e-4, "mixed": 1e-4}
THRESHOLD = 0.05


@pytest.fixture(scope="module")
def h(vl):
    handle = vl.Handle(0)
    yield handle
    handle.close()


def _resample(vl, h, X, L, seed, b0, nb):
    m, n = X.shape
    Xb = torch.empty((nb, m, n), dtype=torch.float64, device="cuda")
    vl.vl_bootstrap_resample(h, X, L, seed, b0, Xb)
    h.sync()
    return Xb.cpu().numpy()


@pytest.mark.parametrize("m,n,L,seed", [
    (10, 1000, 50, 7),           # a short series in blocks of 50
    (7, 517, 33, 2**64 - 3),     # ragged n and L; a seed at the wrap-around
    (5, 300, 1, 123456789),      # i.i.d. resampling of time points
    (6, 257, 257, 5),            # one block: every resample is the series
    (37, 1283, 64, 2**63 + 11),  # rows not a multiple of the gather's 16
])
def test_resample_is_the_oracles(vl, h, m, n, L, seed):
    X = torch.from_numpy(np.random.default_rng(m * n).standard_normal((m, n))).cuda()
    b0, nb = 3, 5
    got = _resample(vl, h, X, L, seed, b0, nb)
    Xh = X.cpu().numpy()
    for z in range(nb):
        idx = oracle.bootstrap_indices(n, L, seed, b0 + z)
        assert np.array_equal(got[z], Xh[:, idx]), z
    # grouping: resample b0 + 2 alone equals the third of the group
    one = _resample(vl, h, X, L, seed, b0 + 2, 1)
    assert np.array_equal(one[0], got[2])


def test_resample_of_a_strided_view_at_finance_size(vl, h):
    """The 400 x 2500 series as a view with row stride 2600, high resample
    numbers: indices and values exact."""
    inst = synth.make_config("finance")
    m, n = inst.X.shape
    buf = torch.zeros((m, n + 100), dtype=torch.float64, device="cuda")
    buf[:, :n] = torch.from_numpy(inst.X).cuda()
    X = buf[:, :n]
    b0 = 2**32 - 4
    got = _resample(vl, h, X, 125, 99, b0, 4)
    for z in range(4):
        assert np.array_equal(got[z], inst.X[:, oracle.bootstrap_indices(n, 125, 99, b0 + z)])


def test_resample_rejects_bad_arguments(vl, h):
    X = torch.zeros((4, 50), dtype=torch.float64, device="cuda")
    Xb = torch.empty((1, 4, 50), dtype=torch.float64, device="cuda")
    for L, b0 in [(0, 0), (51, 0), (10, -1), (10, 2**32)]:
        with pytest.raises(vl.VLError) as e:
            vl.vl_bootstrap_resample(h, X, L, 1, b0, Xb)
        assert e.value.code == 2  # VL_ERR_SHAPE


def _allowed(ref, prec, B):
    """Per-entry slack of the edge and order counts (see the module text)."""
    m = ref["order_prob"].shape[0]
    amb = np.array([g <= GAP[prec] for g in ref["min_gaps"]])
    near = np.zeros((m, m))
    for b, B0 in enumerate(ref["B0s"]):
        if not amb[b]:
            near += np.abs(np.abs(B0) - THRESHOLD) <= B_MARGIN[prec]
    return near + amb.sum(), np.full((m, m), float(amb.sum())), int(amb.sum())


_refs = {}


def _oracle_bootstrap(name, inst, B, L, seed):
    key = (name, B, L, seed)
    if key not in _refs:
        _refs[key] = oracle.bootstrap(inst.X, inst.p, B, L, seed, THRESHOLD)
    return _refs[key]


def _check(vl, h, name, B, L, seed, prec):
    inst = synth.make_config(name)
    X = torch.from_numpy(inst.X).cuda()
    m = inst.X.shape[0]
    ep = torch.empty((m, m), dtype=torch.float64, device="cuda")
    op = torch.empty((m, m), dtype=torch.float64, device="cuda")
    vl.vl_bootstrap(h, X, inst.p, B, L, seed, THRESHOLD, prec, ep, op)
    h.sync()
    ep, op = ep.cpu().numpy(), op.cpu().numpy()
    ref = _oracle_bootstrap(name, inst, B, L, seed)
    # structure that holds at any size
    off = ~np.eye(m, dtype=bool)
    assert np.all(np.diag(op) == 0) and np.allclose((op + op.T)[off], 1.0)
    for t in (ep, op):
        assert np.all((t >= 0) & (t <= 1)) and np.allclose(t * B, np.round(t * B), rtol=0, atol=1e-9)
    slack_e, slack_o, n_amb = _allowed(ref, prec, B)
    de = np.abs(ep - ref["edge_prob"]) * B
    do = np.abs(op - ref["order_prob"]) * B
    assert np.all(de <= slack_e + 1e-9), (np.argwhere(de > slack_e + 1e-9)[:5], n_amb)
    assert np.all(do <= slack_o + 1e-9), (np.argwhere(do > slack_o + 1e-9)[:5], n_amb)
    if not slack_e.any():
        assert np.array_equal(ep, ref["edge_prob"])
    if n_amb == 0:
        assert np.array_equal(op, ref["order_prob"])
    return n_amb


@pytest.mark.parametrize("prec", ["fp64", "mixed_certified", "mixed"])
def test_bootstrap_pr1_over_two_chunks(vl, h, prec):
    """300 resamples of the 10-variable series: more than one chunk of the
    batched path (256), so the counts carry across chunks."""
    n_amb = _check(vl, h, "pr1", 300, 50, 2024, prec)
    assert n_amb <= 30


@pytest.mark.parametrize("prec", ["fp64", "mixed_certified"])
def test_bootstrap_fmri(vl, h, prec):
    """16 resamples of the 50-variable, 200-point series in blocks of 20."""
    _check(vl, h, "fmri", 16, 20, 31, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed_certified"])
def test_bootstrap_server_var3(vl, h, prec):
    """Two resamples of the 120-variable, 10,000-point VAR(3) series in blocks
    of 500 (the oracle takes several seconds per resample)."""
    _check(vl, h, "server", 2, 500, 5, prec)


def test_bootstrap_single_resample_is_the_fit_of_that_resample(vl, h):
    """At the finance size (m = 400, n = 2500), one resample: the tables are
    the thresholded B0 and order relation of vl_fit on vl_bootstrap_resample's
    output (the GPU against itself, through two independent entry points;
    the fit itself is checked against the oracle elsewhere): the order
    relation exactly, the edges up to entries within 1e-6 of the threshold."""
    inst = synth.make_config("finance")
    m, n = inst.X.shape
    X = torch.from_numpy(inst.X).cuda()
    Xb = torch.empty((1, m, n), dtype=torch.float64, device="cuda")
    vl.vl_bootstrap_resample(h, X, 100, 77, 0, Xb)
    out = vl.alloc_outputs(m, inst.p)
    vl.vl_fit(h, Xb[0], inst.p, "mixed_certified", out["M"], out["order"], out["B0"],
              out["Btau"], None)
    ep = torch.empty((m, m), dtype=torch.float64, device="cuda")
    op = torch.empty((m, m), dtype=torch.float64, device="cuda")
    vl.vl_bootstrap(h, X, inst.p, 1, 100, 77, THRESHOLD, "mixed_certified", ep, op)
    h.sync()
    order = out["order"].cpu().numpy()
    pos = np.empty(m, dtype=int)
    pos[order] = np.arange(m)
    assert np.array_equal(op.cpu().numpy(), (pos[:, None] < pos[None, :]).astype(float))
    # the phase-major batch and the single call agree on B0 to 1e-6
    B0 = out["B0"].cpu().numpy()
    differ = ep.cpu().numpy() != (np.abs(B0) > THRESHOLD)
    assert not np.any(differ & (np.abs(np.abs(B0) - THRESHOLD) > 1e-6))


def test_bootstrap_rejects_bad_arguments(vl, h):
    X = torch.zeros((4, 50), dtype=torch.float64, device="cuda")
    t = torch.empty((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(vl.VLError) as e:
        vl.vl_bootstrap(h, X, 1, 0, 10, 1, THRESHOLD, "mixed", t, t)
    assert e.value.code == 2  # VL_ERR_SHAPE: no resamples
    with pytest.raises(vl.VLError) as e:
        vl.vl_bootstrap(h, X, 1, 4, 10, 1, -1.0, "mixed", t, t)
    assert e.value.code == 1  # VL_ERR_ARG: negative threshold
    with pytest.raises(vl.VLError) as e:
        vl.vl_bootstrap(h, X, 12, 4, 10, 1, THRESHOLD, "mixed", t, t)
    assert e.value.code == 3  # VL_ERR_RANK: n - p <= m p + 1
