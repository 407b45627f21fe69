"""Pins of the oracle's Schreier coset mode (growth of the orbit of a central state).

A Schreier coset graph of S_n / H is given by a vector whose stabiliser is H; its vertices are
the vector's images under the group and its growth is taken from that vector (Section 3.1.2,
Section 3.2, the Schreier-graph table).  The checks here do not come from the oracle:

* all-pairs shortest paths of the explicit coset graph from scipy.sparse.csgraph (n <= 7,
  random generator sets and random vectors with repeated entries);
* orbit sizes: n! / prod(c_v!) for the multiset of values c_v when the generators give all of
  S_n, the group order when the vector has distinct entries;
* the Gaussian multinomial (MacMahon's inversion enumerator of multiset permutations) for
  adjacent transpositions acting on a sorted multiset vector;
* numbers the paper prints for the "Bin" coset S_n / (S_m x S_{n-m}), m = floor(n/2), from the
  sorted vector 0^m 1^(n-m): God's number floor(n/2) for transposons and reversals and equal
  growth of the two; God's number (n(3n-4) + 32 - 2(n mod 4)) / 16 for LRX (even n); n - 1
  for pancake (even n); n^2/12 + 1 (n = 0 mod 6) and (n^2 + 4n - 5)/12 (n = 1 mod 6) for
  consecutive 4-cycles, n >= 12 (Section 3.2).
"""

import itertools
import math

import numpy as np
import pytest

import oracle
import workloads as w


def _apsp_coset_growth(n, gens, start):
    """Sphere sizes around `start` in the explicit graph on all distinct rearrangements of it."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    from sympy.utilities.iterables import multiset_permutations
    verts = sorted(tuple(v) for v in multiset_permutations(list(start)))
    index = {v: i for i, v in enumerate(verts)}
    rows, cols = [], []
    for v in verts:
        for g in gens:
            t = tuple(v[g[i]] for i in range(n))
            rows.append(index[v])
            cols.append(index[t])
    m = csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(len(verts), len(verts)))
    dist = shortest_path(m, directed=True, unweighted=True, indices=[index[tuple(start)]])[0]
    dist = dist[np.isfinite(dist)].astype(int)
    return [int(x) for x in np.bincount(dist)]


def _multinomial(vec):
    out = math.factorial(len(vec))
    for v in set(vec):
        out //= math.factorial(list(vec).count(v))
    return out


@pytest.mark.parametrize("seed", range(16))
def test_coset_growth_equals_all_pairs_shortest_paths(seed):
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(2, 8))
    gens = w.random_perms(rng, n, int(rng.integers(1, 4)))
    if seed % 2 == 0:
        gens = w.inverse_closure(gens)
    start = [int(x) for x in rng.integers(0, int(rng.integers(1, n + 1)), size=n)]
    g, rc = oracle.growth(n, gens, start=start)
    assert rc == 0
    assert g == _apsp_coset_growth(n, gens, start)
    if seed % 2 == 0:
        assert g == oracle.growth(n, gens, two_layer=True, start=start)[0]


@pytest.mark.parametrize("n", range(2, 11))
def test_orbit_sizes(n):
    rng = np.random.default_rng(n)
    for _ in range(3):
        start = [int(x) for x in rng.integers(0, 4, size=n)]
        # Coxeter generators give all of S_n: the orbit is every rearrangement
        assert sum(oracle.growth(n, w.coxeter(n), start=start)[0]) == _multinomial(start)
    # a vector with distinct entries: the orbit is a copy of the group (free action)
    perm = [int(x) for x in rng.permutation(n)]
    assert oracle.growth(n, w.lrx(n), start=perm)[0] == oracle.growth(n, w.lrx(n))[0]
    assert oracle.growth(n, w.lx(n), start=list(range(n)))[0] == oracle.growth(n, w.lx(n))[0]
    # values above n - 1 are labels like any other
    assert oracle.growth(n, w.coxeter(n), start=[15] * n)[0] == [1]


@pytest.mark.parametrize("n", range(2, 17))
def test_bin_transposons_and_reversals(n):
    start = w.binary_start(n)
    t, _ = oracle.growth(n, w.transposons(n), start=start)
    r, _ = oracle.growth(n, w.reversals(n), start=start)
    assert len(t) - 1 == n // 2                  # God's number floor(n/2)
    assert r == t                                # "growth coincides with transposons"
    assert sum(t) == math.comb(n, n // 2)


@pytest.mark.parametrize("n", list(range(6, 17, 2)) + [18, 20])
def test_bin_lrx_gods_number_even_n(n):
    g, _ = oracle.growth(n, w.lrx(n), start=w.binary_start(n))
    assert len(g) - 1 == (n * (3 * n - 4) + 32 - 2 * (n % 4)) // 16
    assert sum(g) == math.comb(n, n // 2)


@pytest.mark.parametrize("n", range(4, 17, 2))
def test_bin_pancake_gods_number_even_n(n):
    g, _ = oracle.growth(n, w.pancake(n), start=w.binary_start(n))
    assert len(g) - 1 == n - 1


@pytest.mark.parametrize("n,want", [(12, 12 * 12 // 12 + 1), (13, (13 * 13 + 4 * 13 - 5) // 12),
                                    (18, 18 * 18 // 12 + 1), (19, (19 * 19 + 4 * 19 - 5) // 12)])
def test_bin_consecutive_4cycles_gods_number(n, want):
    g, _ = oracle.growth(n, w.consecutive_4cycles(n), start=w.binary_start(n))
    assert len(g) - 1 == want


def test_coset_limits():
    start = w.binary_start(12)
    full, _ = oracle.growth(12, w.lrx(12), start=start)
    g, rc = oracle.growth(12, w.lrx(12), start=start, max_radius=5)
    assert rc == 1 and g == full[:6]
    g, rc = oracle.growth(12, w.lrx(12), start=start, stop_above=50)
    assert rc == 1 and g[-1] > 50 and g == full[:len(g)]
    with pytest.raises(ValueError):
        oracle.growth(4, w.coxeter(4), start=[0, 1, 2, 16])


def _poly_mul(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _poly_div_exact(a, b):
    a = list(a)
    q = [0] * (len(a) - len(b) + 1)
    for i in range(len(q) - 1, -1, -1):
        q[i] = a[i + len(b) - 1] // b[-1]
        for j, y in enumerate(b):
            a[i + j] -= q[i] * y
    assert not any(a), "not an exact division"
    return q


def q_multinomial(counts):
    """Gaussian multinomial [n; c_1, ..., c_k]_q = [n]_q! / prod [c_i]_q!, as coefficients."""
    def qfact(m):
        p = [1]
        for j in range(1, m + 1):
            p = _poly_mul(p, [1] * j)
        return p
    num = qfact(sum(counts))
    for c in counts:
        num = _poly_div_exact(num, qfact(c))
    return num


@pytest.mark.parametrize("counts", [(1, 1, 1, 1), (2, 2), (3, 2, 1), (2, 3, 2), (4, 4), (5, 1, 1),
                                    (3, 3, 3), (6, 5), (2, 2, 2, 2, 2)])
def test_coxeter_on_multiset_is_q_multinomial(counts):
    # Adjacent transpositions acting on a sorted multiset vector: the distance to a rearrangement
    # is its number of inversions (swapping equal neighbours is a loop), so the growth is the
    # inversion enumerator of multiset permutations, the Gaussian multinomial (MacMahon).
    start = [v for v, c in enumerate(counts) for _ in range(c)]
    n = len(start)
    assert oracle.growth(n, w.coxeter(n), start=start)[0] == q_multinomial(counts)


@pytest.mark.parametrize("seed", range(8))
def test_long_vectors_equal_all_pairs_shortest_paths(seed):
    # n > 16: the oracle's 256-bit keys; vectors of two or three values, explicit graph by scipy
    rng = np.random.default_rng(6000 + seed)
    n = int(rng.integers(17, 21))
    nvals = 2 if seed % 2 == 0 else 3
    counts = [n - 2 * (nvals - 1)] + [2] * (nvals - 1)      # few rearrangements: small graph
    start = [v for v, c in enumerate(counts) for _ in range(c)]
    rng.shuffle(start)
    start = [int(x) for x in start]
    gens = w.random_perms(rng, n, 2)
    if seed % 4 < 2:
        gens = w.inverse_closure(gens)
    g, rc = oracle.growth(n, gens, start=start)
    assert rc == 0 and g == _apsp_coset_growth(n, gens, start)
