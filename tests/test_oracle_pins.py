"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Every check here would fail under a plausible mistake in the oracle (a dropped generator,
a wrong sign or index in the action, a visited set that forgets a layer, an off-by-one in
the layer count):

* closed forms the paper states: Mahonian numbers for Coxeter generators (the word metric is
  the number of inversions, Section 3.3 table "Metric"), unsigned Stirling numbers of the
  first kind for all transpositions (Section 3.3 table "Growth/F-la"), Fibonacci leading
  terms for LX (Section 4.2);
* published diameters: Section 3.2 examples and the Section 3.3 table (Coxeter, cyclic
  Coxeter, star, LRX, LX, 3-cycles, (01i)I, (i,i+1,i+2)I, prefix cycles, reversals,
  transposons), the Section 3.4 maximal-diameter tables, Section 3.7 Koltsov3involutions;
* the reversal spheres |S_1| = C(n,2), |S_2| = (n^4 - 2n^3 - n^2 - 16n + 42)/6 (Section 5.2);
* group orders from sympy's Schreier-Sims (a library routine), n! and n!/2;
* all-pairs shortest paths of the explicit graph from scipy.sparse.csgraph (n <= 5).
"""

import itertools
import math

import numpy as np
import pytest

import oracle
import workloads as w


def mahonian(n):
    """Coefficients of prod_{j=1}^{n} (1 + q + ... + q^{j-1})."""
    poly = np.array([1], dtype=object)
    for j in range(1, n + 1):
        poly = np.convolve(poly, np.ones(j, dtype=object))
    return [int(x) for x in poly]


def stirling1_unsigned(n):
    """c(n, k) for k = 0..n by c(m+1, k) = m c(m, k) + c(m, k-1)."""
    row = [1]
    for m in range(n):
        new = [0] * (m + 2)
        for k in range(m + 2):
            a = m * row[k] if k < len(row) else 0
            b = row[k - 1] if k >= 1 else 0
            new[k] = a + b
        row = new
    return row


def diam(n, gens):
    g, rc = oracle.growth(n, gens)
    assert rc == 0
    return len(g) - 1


@pytest.mark.parametrize("n", range(1, 9))
@pytest.mark.parametrize("two_layer", [False, True])
def test_coxeter_is_mahonian(n, two_layer):
    gens = w.coxeter(n) if n > 1 else [[0]]
    g, _ = oracle.growth(n, gens, two_layer=two_layer)
    assert g == mahonian(n)
    assert g == g[::-1]                       # palindromic
    assert sum(g) == math.factorial(n)
    assert len(g) - 1 == n * (n - 1) // 2     # diameter n(n-1)/2


@pytest.mark.parametrize("n", range(2, 7))
def test_coxeter_word_metric_is_inversions_bruteforce(n):
    hist = [0] * (n * (n - 1) // 2 + 1)
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        hist[inv] += 1
    g, _ = oracle.growth(n, w.coxeter(n))
    assert g == hist


def test_coxeter_distance_equals_inversions():
    rng = np.random.default_rng(7)
    n = 7
    for _ in range(20):
        p = [int(x) for x in rng.permutation(n)]
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        assert oracle.distance(n, w.coxeter(n), p) == inv


@pytest.mark.parametrize("n", range(2, 9))
def test_all_transpositions_is_stirling(n):
    c = stirling1_unsigned(n)
    g, _ = oracle.growth(n, w.all_transpositions(n))
    assert g == [c[n - r] for r in range(n)]
    assert len(g) - 1 == n - 1


@pytest.mark.parametrize("n", range(3, 9))
def test_closed_form_diameters(n):
    assert diam(n, w.cyclic_coxeter(n)) == n * n // 4
    assert diam(n, w.star(n)) == (3 * (n - 1)) // 2
    if n >= 4:  # for n = 3 the LRX graph is S_3 with 3 generators, diameter 2
        assert diam(n, w.lrx(n)) == n * (n - 1) // 2
    assert diam(n, w.three_cycles(n)) == n // 2
    assert diam(n, w.cycles_01i_inv(n)) == (3 * n - 6) // 2
    assert diam(n, w.consecutive_3cycles_inv(n)) == n * (n - 1) // 4
    assert diam(n, w.prefix_cycles(n)) == n - 1
    assert diam(n, w.reversals(n)) == n - 1
    assert diam(n, w.transposons(n)) == -(-(n + 1) // 2)


@pytest.mark.parametrize("n", range(3, 10))
def test_reversal_spheres(n):
    g, _ = oracle.growth(n, w.reversals(n))
    assert g[1] == n * (n - 1) // 2
    assert g[2] == (n ** 4 - 2 * n ** 3 - n ** 2 - 16 * n + 42) // 6
    assert sum(g) == math.factorial(n)


@pytest.mark.parametrize("n", range(5, 11))
def test_lx_diameter_and_fibonacci(n):
    g, _ = oracle.growth(n, w.lx(n))
    want = (3 * n * n - 8 * n + 9) // 4 if n % 2 else (3 * n * n - 8 * n + 12) // 4
    assert len(g) - 1 == want
    fib = [1, 2]
    while len(fib) < n - 1:
        fib.append(fib[-1] + fib[-2])
    # The leading layers follow Fibonacci numbers for r = 0..n-2.
    assert g[: n - 1] == fib[: n - 1]
    assert sum(g) == math.factorial(n)


@pytest.mark.parametrize("n,type_,k,want", [(5, 1, 1, 10), (6, 1, 0, 16), (7, 2, 1, 30)])
def test_koltsov3_diameters(n, type_, k, want):
    assert diam(n, w.koltsov3(n, type_, k)) == want


def _golden_max_diameter():
    import os
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "max_diameter_sets.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kind, n, d, gs = [x.strip() for x in line.split("|")]
        n, d = int(n), int(d)
        rows.append((kind, n, d, [w.from_cycles(n, g) for g in gs.split(";")]))
    return rows


MAXD = _golden_max_diameter()


@pytest.mark.parametrize("kind,n,d,gens", [r for r in MAXD if r[1] <= 9],
                         ids=[f"{r[0]}{r[1]}" for r in MAXD if r[1] <= 9])
def test_published_max_diameters(kind, n, d, gens):
    assert w.is_inverse_closed(gens) == (kind == "undirected") or n == 3
    g, _ = oracle.growth(n, gens)
    assert len(g) - 1 == d
    assert sum(g) == math.factorial(n)


@pytest.mark.slow
@pytest.mark.parametrize("kind,n,d,gens", [r for r in MAXD if r[1] == 10],
                         ids=[f"{r[0]}{r[1]}" for r in MAXD if r[1] == 10])
def test_published_max_diameters_n10(kind, n, d, gens):
    g, _ = oracle.growth(n, gens)
    assert len(g) - 1 == d
    assert sum(g) == math.factorial(n)


def test_group_order_matches_sympy():
    sympy_comb = pytest.importorskip("sympy.combinatorics")
    rng = np.random.default_rng(1234)
    for trial in range(40):
        n = int(rng.integers(3, 9))
        k = int(rng.integers(1, 4))
        gens = w.random_perms(rng, n, k)
        if trial % 2 == 0:
            gens = w.inverse_closure(gens)
        order = sympy_comb.PermutationGroup([sympy_comb.Permutation(g) for g in gens]).order()
        g, _ = oracle.growth(n, gens)
        assert sum(g) == order
        if w.is_inverse_closed(gens):
            g2, _ = oracle.growth(n, gens, two_layer=True)
            assert g2 == g


def test_alternating_families_have_half_order():
    for n in range(3, 8):
        for gens in (w.three_cycles(n), w.cycles_01i_inv(n), w.consecutive_3cycles_inv(n)):
            g, _ = oracle.growth(n, gens)
            assert sum(g) == math.factorial(n) // 2


def _apsp_growth_from(n, gens, start):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path
    perms = list(itertools.permutations(range(n)))
    index = {p: i for i, p in enumerate(perms)}
    rows, cols = [], []
    for p in perms:
        for g in gens:
            t = tuple(p[g[i]] for i in range(n))
            rows.append(index[p])
            cols.append(index[t])
    m = csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(len(perms), len(perms)))
    dist = shortest_path(m, directed=True, unweighted=True, indices=[index[tuple(start)]])[0]
    dist = dist[np.isfinite(dist)].astype(int)
    return [int(x) for x in np.bincount(dist)]


@pytest.mark.parametrize("seed", range(12))
def test_growth_equals_all_pairs_shortest_paths(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 6))
    gens = w.random_perms(rng, n, int(rng.integers(1, 4)))
    if seed % 3 == 0:
        gens = w.inverse_closure(gens)
    g, _ = oracle.growth(n, gens)
    assert g == _apsp_growth_from(n, gens, list(range(n)))
    # vertex-transitive: growth from another element of the group is the same
    if len(g) > 1:
        other = oracle.layer_keys(n, gens, len(g) - 1)[0]
        start = [int((int(other) >> (4 * i)) & 15) for i in range(n)]
        assert g == _apsp_growth_from(n, gens, start)


@pytest.mark.parametrize("seed", range(10))
def test_growth_invariant_under_inverting_generators(seed):
    # gamma_S = gamma_{S^-1}: the action convention (gather / scatter / left) is immaterial.
    rng = np.random.default_rng(seed)
    n = int(rng.integers(4, 8))
    gens = w.random_perms(rng, n, 2)
    a, _ = oracle.growth(n, gens)
    b, _ = oracle.growth(n, [w.inverse(x) for x in gens])
    assert a == b


def test_antipodes():
    # Coxeter: the single longest element is the full reversal (table "Antipodes" = 1).
    for n in range(2, 8):
        last = oracle.layer_keys(n, w.coxeter(n), n * (n - 1) // 2)
        rev = sum((n - 1 - i) << (4 * i) for i in range(n))
        assert list(last) == [rev]
    # All transpositions: the last layer (distance n-1) is the (n-1)! n-cycles.
    for n in range(2, 8):
        last = oracle.layer_keys(n, w.all_transpositions(n), n - 1)
        assert len(last) == math.factorial(n - 1)
    # Reversals: the Gollan permutation and its inverse are the only elements at distance
    # n-1 (Section 5.2), n >= 4.
    for n in range(4, 9):
        assert len(oracle.layer_keys(n, w.reversals(n), n - 1)) == 2


def test_limits_and_codes():
    g, rc = oracle.growth(8, w.coxeter(8), max_radius=5)
    assert rc == 1 and g == mahonian(8)[:6]
    g, rc = oracle.growth(8, w.coxeter(8), stop_above=1000)
    assert rc == 1 and g[-1] > 1000 and all(x <= 1000 for x in g[:-1])
    assert oracle.growth(3, [[0, 1, 2]]) == ([1], 0)     # identity generator only
    with pytest.raises(ValueError):
        oracle.growth(3, [[0, 0, 1]])


# ---- oracle B (rank-bitmap BFS for large groups) is pinned to oracle A ----------------------

@pytest.mark.parametrize("family", ["coxeter", "lrx", "lx", "pancake", "reversals", "star",
                                    "three_cycles", "prefix_cycles", "cyclic_coxeter"])
@pytest.mark.parametrize("n", [2, 5, 8])
def test_oracle_b_equals_oracle_a_on_families(family, n):
    gens = w.FAMILIES[family](n)
    if not gens:
        pytest.skip("empty set")
    assert oracle.growth_bitmap(n, gens, threads=3) == oracle.growth(n, gens)


@pytest.mark.parametrize("seed", range(10))
def test_oracle_b_equals_oracle_a_random(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(3, 10))
    gens = w.random_perms(rng, n, int(rng.integers(1, 4)))
    if seed % 2:
        gens = w.inverse_closure(gens)
    assert oracle.growth_bitmap(n, gens, threads=1 + seed % 4) == oracle.growth(n, gens)


def test_oracle_b_limits_and_closed_forms():
    assert oracle.growth_bitmap(9, w.coxeter(9))[0] == mahonian(9)
    c = stirling1_unsigned(9)
    assert oracle.growth_bitmap(9, w.all_transpositions(9))[0] == [c[9 - r] for r in range(9)]
    assert oracle.growth_bitmap(10, w.lrx(10), max_radius=12) == oracle.growth(10, w.lrx(10), max_radius=12)
    g, rc = oracle.growth_bitmap(9, w.coxeter(9), stop_above=5000)
    assert rc == 1 and g == mahonian(9)[:len(g)] and g[-1] > 5000


def test_stored_values_of_both_oracles_agree():
    import os
    d = os.path.join(os.path.dirname(__file__), "golden")
    read = lambda f: [int(l.split()[1]) for l in open(os.path.join(d, f)) if not l.startswith("#")]
    a = read("s14_pancake_layers.txt")       # oracle A, layers 0..8
    b = read("s14_pancake_layers_b.txt")     # oracle B, layers 0..10
    assert len(a) == 9 and len(b) == 11 and b[:9] == a
    assert b[10] > 2 ** 31 >= max(b[:10])     # config 3 stops after layer 10


# ---- oracle C (visited set and layers as bitmaps over all n! ranks) is pinned to A and B ----

@pytest.mark.parametrize("family", ["coxeter", "lrx", "lx", "pancake", "reversals", "star",
                                    "three_cycles", "prefix_cycles", "all_transpositions"])
@pytest.mark.parametrize("n", [2, 5, 8])
def test_oracle_c_equals_oracle_a_on_families(family, n):
    gens = w.FAMILIES[family](n)
    if not gens:
        pytest.skip("empty set")
    assert oracle.growth_bitmask(n, gens, threads=3) == oracle.growth(n, gens)


@pytest.mark.parametrize("seed", range(10))
def test_oracle_c_equals_oracle_a_random(seed):
    rng = np.random.default_rng(1900 + seed)
    n = int(rng.integers(3, 10))
    gens = w.random_perms(rng, n, int(rng.integers(1, 4)))
    if seed % 2:
        gens = w.inverse_closure(gens)
    assert oracle.growth_bitmask(n, gens, threads=1 + seed % 4) == oracle.growth(n, gens)


def test_oracle_c_limits_closed_forms_and_progress():
    assert oracle.growth_bitmask(9, w.coxeter(9))[0] == mahonian(9)
    c = stirling1_unsigned(8)
    assert oracle.growth_bitmask(8, w.all_transpositions(8))[0] == [c[8 - r] for r in range(8)]
    g, rc = oracle.growth_bitmask(9, w.coxeter(9), max_radius=6)
    assert rc == 1 and g == mahonian(9)[:7]
    g, rc = oracle.growth_bitmask(9, w.coxeter(9), stop_above=5000)
    assert rc == 1 and g == mahonian(9)[:len(g)] and g[-1] > 5000
    seen = []
    oracle.growth_bitmask(7, w.pancake(7), progress=lambda r, s: seen.append((r, s)))
    assert [s for _, s in seen] == oracle.growth(7, w.pancake(7))[0][1:]
    assert oracle.growth_bitmask(10, w.lrx(10), max_radius=12) == oracle.growth_bitmap(10, w.lrx(10), max_radius=12)


# ---- oracle C against oracle B on whole growths of S_12 ----
# Oracle B indexes S_n by the classic Lehmer rank and expands a list frontier; oracle C indexes
# it by the position-major rank and keeps every layer as a bitmap.  A mistake shared by the two
# designs would have to appear in two different rank functions and two different traversals.

def _stored(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name + ".txt")
    return [int(l.split()[1]) for l in open(path) if not l.startswith("#")]


@pytest.mark.parametrize("family,diameter", [("pancake", None), ("lrx", 66)])
def test_stored_whole_s12_growths_of_oracles_b_and_c_agree(family, diameter):
    b = _stored(f"s12_{family}_growth_b")
    c = _stored(f"s12_{family}_growth_c")
    assert b == c
    assert sum(b) == math.factorial(12)
    k = len(w.FAMILIES[family](12))
    assert b[1] == k
    if diameter is not None:                  # LRX: n(n-1)/2 (Section 3.3 table)
        assert len(b) - 1 == diameter
    else:                                     # pancake: girth 6, so sphere 2 is k(k-1)
        assert b[2] == k * (k - 1)


@pytest.mark.slow
@pytest.mark.skipif(not __import__("os").environ.get("CG_SLOW_TESTS"),
                    reason="about 6 minutes on 8 host threads; set CG_SLOW_TESTS=1")
@pytest.mark.parametrize("family", ["pancake", "lrx"])
def test_whole_s12_growth_oracle_b_equals_oracle_c(family):
    gens = w.FAMILIES[family](12)
    b = oracle.growth_bitmap(12, gens)
    c = oracle.growth_bitmask(12, gens)
    assert b == c and b[1] == 0
    assert b[0] == _stored(f"s12_{family}_growth_b")


# ---- growth from the identity beyond 16 elements (keys of the permutation's bytes) ----------

@pytest.mark.parametrize("n", [17, 20, 24, 32])
@pytest.mark.parametrize("two_layer", [False, True])
def test_identity_beyond_16_is_mahonian_prefix(n, two_layer):
    g, rc = oracle.growth(n, w.coxeter(n), two_layer=two_layer, max_radius=4)
    assert rc == 1 and g == mahonian(n)[:5]


@pytest.mark.parametrize("n", [17, 19])
def test_identity_beyond_16_is_stirling_prefix(n):
    c = stirling1_unsigned(n)
    g, rc = oracle.growth(n, w.all_transpositions(n), max_radius=2)
    assert g == [c[n - r] for r in range(3)]


def test_identity_beyond_16_embeds_a_smaller_group():
    # generators that move only the first 8 of 20 elements generate a copy of S_8: the growth
    # of the whole orbit is that of S_8 Coxeter (40,320 states, diameter 28)
    gens = [list(g) + list(range(8, 20)) for g in w.coxeter(8)]
    g, rc = oracle.growth(20, gens)
    assert rc == 0 and g == mahonian(8)
