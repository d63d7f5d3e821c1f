"""The seeded input recipe (the generator both sides are fed from): unit-
variance shock laws, exact companion-radius scaling, acyclic B0 under its
stated order, the workload shapes and seeds, the batch's redraw rule, and
determinism.  CPU only; no estimation arithmetic is involved."""
import math

import numpy as np
import pytest

import synth


@pytest.mark.parametrize("kind,tol", [("uniform", 0.01), ("laplace", 0.02), ("powgauss", 0.03),
                                      ("t3", 0.15), ("gauss", 0.01)])
def test_shock_laws_have_zero_mean_and_unit_variance(kind, tol):
    rng = np.random.Generator(np.random.PCG64(5))
    e = synth.draw_noise(rng, kind, 400000)
    assert abs(e.mean()) < 0.01
    assert abs(e.var() - 1.0) < tol


def test_shock_laws_are_the_named_families():
    rng = np.random.Generator(np.random.PCG64(6))
    u = synth.draw_noise(rng, "uniform", 200000)
    assert abs(u.max() - math.sqrt(3)) < 1e-3 and abs(u.min() + math.sqrt(3)) < 1e-3
    lap = synth.draw_noise(rng, "laplace", 400000)
    assert abs(np.mean(np.abs(lap)) - 1 / math.sqrt(2)) < 0.01   # E|x| = b for Laplace(0, b)
    pg = synth.draw_noise(rng, "powgauss", 400000)
    assert abs(np.mean(pg ** 3)) < 0.05                          # symmetric
    assert np.mean(pg ** 4) > 4.0                                # heavier tails than a Gaussian


@pytest.mark.parametrize("p,target", [(1, 0.5), (2, 0.7), (3, 0.9)])
def test_scaling_hits_the_companion_radius_exactly(p, target):
    rng = np.random.Generator(np.random.PCG64(10 + p))
    M = synth.draw_var(rng, 6, p, "unif", target)
    assert abs(synth.companion_radius(M) - target) < 1e-10


def test_dag_is_acyclic_under_its_order_with_bounded_weights():
    rng = np.random.Generator(np.random.PCG64(7))
    B0, perm = synth.draw_dag(rng, 30, 0.3, 0.1, 0.5)
    pos = np.empty(30, dtype=int)
    pos[perm] = np.arange(30)
    i, j = np.nonzero(B0)
    assert len(i) > 0
    assert np.all(pos[j] < pos[i])                    # every edge j -> i follows the order
    assert np.all((np.abs(B0[i, j]) >= 0.1) & (np.abs(B0[i, j]) <= 0.5))
    assert np.all(np.diag(B0) == 0)


def test_workload_shapes_and_seeds():
    shapes = {"pr1": (10, 1000, 1), "fmri": (50, 200, 1), "server": (120, 10000, 3)}
    for k, (name, (m, n, p)) in enumerate(shapes.items()):
        inst = synth.make_config(name)
        assert (inst.m, inst.n, inst.p) == (m, n, p)
        assert inst.seed == 2409055 + 1000 * k
        assert np.all(np.isfinite(inst.X))
    fin = synth.make_config("finance", m=40, n=300)
    assert (fin.m, fin.n, fin.p, fin.noise) == (40, 300, 1, "t3")


def test_batch_redraws_until_the_var_fit_is_well_posed():
    shapes = synth.draw_batched_shapes(256, synth.config_seed(4))
    assert len(shapes) == 256
    for m, n, p, noise, redraws in shapes:
        assert 20 <= m <= 400 and 250 <= n <= 5000 and 1 <= p <= 3
        assert n - p >= 2 * (m * p + 1)
        assert noise in ("uniform", "laplace", "t3")
    assert sum(r for *_, r in shapes) > 0             # the rule did act


def test_generator_is_deterministic_per_seed():
    a = synth.make_instance(8, 300, 2, 99, "laplace")
    b = synth.make_instance(8, 300, 2, 99, "laplace")
    c = synth.make_instance(8, 300, 2, 100, "laplace")
    assert np.array_equal(a.X, b.X) and np.array_equal(a.B0, b.B0)
    assert not np.array_equal(a.X, c.X)
