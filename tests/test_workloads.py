"""CPU checks of the seeded input recipes: the five workloads have the shapes, sizes and value
distributions they are defined with, and a seed gives the same inputs every time."""

import math

import numpy as np

import workloads as w
from workloads import configs as cfg
from workloads import families as fam


def is_perm(p, n):
    return sorted(p) == list(range(n))


def test_fixed_configs():
    j = cfg.config_s8_coxeter()
    assert (j.n, j.k, j.inverse_closed, j.max_radius, j.stop_above) == (8, 7, True, -1, 0)
    j = cfg.config_s11_lrx()
    assert (j.n, j.k, j.inverse_closed) == (11, 3, True)
    j = cfg.config_s14_pancake()
    assert (j.n, j.k, j.inverse_closed, j.stop_above) == (14, 13, True, 2 ** 31)
    assert all(is_perm(g, 14) for g in j.gens)


def test_batch_groups_recipe():
    jobs = cfg.batch_groups(count=400)
    assert jobs == cfg.batch_groups(count=400)                 # the seed fixes the inputs
    assert cfg.batch_groups(seed=1, count=8) != cfg.batch_groups(count=8)
    ns = [j.n for j in jobs]
    assert min(ns) == 6 and max(ns) == 10
    for i, j in enumerate(jobs):
        assert all(is_perm(g, j.n) and g != list(range(j.n)) for g in j.gens)
        if i % 2 == 0:                                         # inverses appended: undirected
            assert j.inverse_closed and fam.is_inverse_closed(j.gens)
            assert 2 <= j.k <= 10
        else:                                                  # directed: the k drawn
            assert 2 <= j.k <= 5
    ks = [j.k for j in jobs[1::2]]
    assert set(ks) == {2, 3, 4, 5}
    # the draw order: n, then k, then the k permutations of each group in index order
    rng = np.random.Generator(np.random.PCG64(cfg.BATCH_SEED))
    n0 = int(rng.integers(6, 11))
    k0 = int(rng.integers(2, 6))
    first = fam.inverse_closure(fam.random_perms(rng, n0, k0))
    assert (jobs[0].n, jobs[0].gens) == (n0, first)


def test_serve_stream_recipe():
    jobs = cfg.serve_stream(count=4000)
    assert [j.arrival for j in jobs] == [j.arrival for j in cfg.serve_stream(count=4000)]
    gaps = np.diff([0.0] + [j.arrival for j in jobs])
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 1.0) < 0.05                        # unit-rate Poisson arrivals
    assert abs(gaps.std() - 1.0) < 0.07                         # exponential gaps: sd = mean
    fams = {j.family for j in jobs}
    assert fams == set(cfg.SERVE_FAMILIES)
    for j in jobs:
        assert 8 <= j.n <= 16 and j.inverse_closed
        assert fam.is_inverse_closed(j.gens)
        D = max(6, cfg.serve_diameter_guess(j.family, j.n))
        assert 6 <= j.max_radius <= D


def test_serve_diameter_guesses():
    assert cfg.serve_diameter_guess("coxeter", 10) == 45
    assert cfg.serve_diameter_guess("lrx", 11) == 55
    assert cfg.serve_diameter_guess("all_transpositions", 9) == 8
    assert cfg.serve_diameter_guess("pancake", 10) == math.ceil(12.0) + 2
    assert cfg.serve_diameter_guess("random_inv", 8) == 32 + 32


def test_random_perms_reject_the_identity():
    rng = np.random.Generator(np.random.PCG64(3))
    for n in (2, 3):
        gens = fam.random_perms(rng, n, 50)
        assert len(gens) == 50 and all(g != list(range(n)) and is_perm(g, n) for g in gens)


def test_family_sizes():
    n = 9
    assert len(w.coxeter(n)) == n - 1
    assert len(w.all_transpositions(n)) == n * (n - 1) // 2
    assert len(w.pancake(n)) == n - 1
    assert len(w.lrx(n)) == 3 and len(w.lx(n)) == 2
    for name, f in w.FAMILIES.items():
        gens = f(n)
        assert all(is_perm(g, n) for g in gens), name
