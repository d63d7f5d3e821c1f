"""Pins of the oracle's bootstrap (a reading: moving-block resampling, Kuensch
1989, with block starts from the counter-based SplitMix64 generator):
properties of the generator and of the resamples that a mistake in the
mixing steps, the block arithmetic or the aggregation would break, and the
reduction of the bootstrap to the plain fit when one block covers the
series."""
import math

import numpy as np

import oracle
import synth


def test_generator_strict_avalanche():
    """Flipping input bit i flips output bit j with probability close to 1/2
    for every (i, j) (strict avalanche): dropping either multiply-xorshift
    round or the final xor-shift of the mixer leaves pairs at 0 or 1."""
    rng = np.random.default_rng(1)
    N = 120
    rate = np.zeros((64, 64))
    for i in range(64):
        for _ in range(N):
            x = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
            d = oracle.splitmix64(x) ^ oracle.splitmix64(x ^ (1 << i))
            rate[i] += [(d >> j) & 1 for j in range(64)]
    rate /= N
    assert 0.2 <= rate.min() and rate.max() <= 0.8, (rate.min(), rate.max())


def test_generator_is_uniform_and_counter_based():
    """Draws are uniform over [0, 2^64) (chi-square over 32 bins) and depend
    only on (seed, counter): the same counter gives the same draw, nearby
    counters and seeds give unrelated ones."""
    draws = [oracle.splitmix64_draw(11, k) for k in range(1, 32001)]
    counts = np.bincount([d >> 59 for d in draws], minlength=32)
    chi2 = float(((counts - 1000.0) ** 2 / 1000.0).sum())
    assert chi2 < 70.0  # 31 degrees of freedom: P(chi2 > 70) ~ 1e-4
    assert oracle.splitmix64_draw(11, 5) == draws[4]
    assert oracle.splitmix64_draw(12, 5) != draws[4]
    assert len(set(draws)) == len(draws)


def test_resample_blocks():
    """Each resample has n indices made of block_len-long runs of consecutive
    time points (the last one cut), each run starting in [0, n - block_len];
    different resamples differ; the starts cover their range evenly."""
    n, L = 103, 10
    idx = [oracle.bootstrap_indices(n, L, 3, b) for b in range(6)]
    for a in idx:
        assert a.shape == (n,)
        for k in range(0, n, L):
            run = a[k:k + L]
            assert 0 <= run[0] <= n - L
            assert np.array_equal(run, run[0] + np.arange(len(run)))
    assert len({tuple(a) for a in idx}) == 6
    # starts of a short series: span 3, each start about a third of the time
    starts = np.concatenate([oracle.bootstrap_indices(12, 10, 9, b)[[0]] for b in range(1500)])
    counts = np.bincount(starts, minlength=3)
    assert counts.shape == (3,) and np.all(np.abs(counts - 500) < 100)


def test_one_block_reduces_to_the_plain_fit():
    """With block_len = n every resample is the series itself, so the edge
    probabilities are the plain fit's thresholded |B0| and the order
    probabilities its order relation."""
    inst = synth.make_config("pr1")
    n = inst.X.shape[1]
    r = oracle.bootstrap(inst.X, inst.p, 3, n, 21, 0.05)
    fit = oracle.varlingam(inst.X, inst.p)
    assert np.array_equal(r["edge_prob"], (np.abs(fit["B0"]) > 0.05).astype(float))
    pos = np.empty(len(fit["order"]), dtype=int)
    pos[fit["order"]] = np.arange(len(fit["order"]))
    assert np.array_equal(r["order_prob"], (pos[:, None] < pos[None, :]).astype(float))


def test_probabilities_are_consistent():
    """order_prob[i, j] + order_prob[j, i] = 1 off the diagonal, 0 on it; both
    tables are multiples of 1 / n_resamples in [0, 1]; B0 of every resample
    is strictly lower triangular in its own order."""
    inst = synth.make_config("pr1")
    B = 5
    r = oracle.bootstrap(inst.X, inst.p, B, 40, 4, 0.05)
    op, ep = r["order_prob"], r["edge_prob"]
    m = op.shape[0]
    off = ~np.eye(m, dtype=bool)
    assert np.allclose((op + op.T)[off], 1.0) and np.all(np.diag(op) == 0)
    for t in (op, ep):
        assert np.all((t >= 0) & (t <= 1))
        assert np.allclose(t * B, np.round(t * B))
    for order, B0 in zip(r["orders"], r["B0s"]):
        P = B0[np.ix_(order, order)]
        assert np.allclose(np.triu(P), 0.0)
    assert all(g > 0 for g in r["min_gaps"]) and not math.isnan(sum(r["min_gaps"]))
