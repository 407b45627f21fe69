"""GPU parity of two-word (128-bit) keys: vectors whose packed form needs more than 64 bits --
coset vectors of 4-bit values up to n = 32, 2-bit up to 64, binary up to 128 -- and the
identity of S_n for 17 <= n <= 25 (5-bit elements).  Checked against the oracle (n <= 64 with
a start vector, n <= 32 from the identity) and against closed forms beyond its reach: the
Mahonian numbers, the Stirling numbers of the first kind, and MacMahon's Gaussian multinomial
for adjacent transpositions on a sorted multiset vector."""

import math

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available()
    import paper_2509_19162_gb300 as p
    p.build()
    return p


def mahonian(n):
    poly = np.array([1], dtype=object)
    for j in range(1, n + 1):
        poly = np.convolve(poly, np.ones(j, dtype=object))
    return [int(x) for x in poly]


def stirling_growth(n):
    c = [[0] * (n + 1) for _ in range(n + 1)]
    c[0][0] = 1
    for m in range(1, n + 1):
        for j in range(1, m + 1):
            c[m][j] = c[m - 1][j - 1] + (m - 1) * c[m - 1][j]
    return [c[n][n - r] for r in range(n)]


def q_multinomial(counts):
    """[n; c_1, ..., c_k]_q = [n]_q! / prod [c_i]_q!, as integer coefficients."""
    def mul(a, b):
        out = [0] * (len(a) + len(b) - 1)
        for i, x in enumerate(a):
            if x:
                for j, y in enumerate(b):
                    out[i + j] += x * y
        return out

    def div(a, b):
        a = list(a)
        q = [0] * (len(a) - len(b) + 1)
        for i in range(len(q) - 1, -1, -1):
            q[i] = a[i + len(b) - 1] // b[-1]
            for j, y in enumerate(b):
                a[i + j] -= q[i] * y
        assert not any(a)
        return q

    def qfact(m):
        p = [1]
        for j in range(1, m + 1):
            p = mul(p, [1] * j)
        return p
    num = qfact(sum(counts))
    for c in counts:
        num = div(num, qfact(c))
    return num


@pytest.mark.parametrize("n", [17, 20, 24, 25])
def test_identity_beyond_16_is_mahonian_prefix(cg, n):
    with cg.Growth(n, w.coxeter(n), max_radius=6) as g:
        r = g.run()
        assert g.key_words == 2 and g.key_width == 5
    assert r.status == 1 and r.layers == mahonian(n)[:7]


def test_identity_beyond_16_all_transpositions_and_lrx(cg):
    r = cg.growth(18, w.all_transpositions(18), max_radius=3)
    assert r.layers == stirling_growth(18)[:4]
    for n, gens, rad in [(20, w.lrx(20), 14), (17, w.pancake(17), 4), (22, w.lx(22), 12)]:
        want, rc = oracle.growth(n, gens, max_radius=rad)
        got = cg.growth(n, gens, max_radius=rad)
        assert got.layers == want and got.status == 1


def test_identity_beyond_16_complete_orbit(cg):
    # generators moving the first 8 of 20 elements: a copy of S_8, grown to the end
    gens = [list(g) + list(range(8, 20)) for g in w.coxeter(8)]
    r = cg.growth(20, gens)
    assert r.status == 0 and r.layers == mahonian(8)


@pytest.mark.parametrize("n,vals", [(17, 5), (24, 5), (31, 6), (32, 5), (40, 4), (52, 3), (62, 4),
                                    (64, 3)])
@pytest.mark.parametrize("family", ["lrx", "coxeter", "pancake"])
def test_long_coset_vectors_vs_oracle(cg, n, vals, family):
    # values 0..vals-1 in a seeded order: 4-bit elements when a value exceeds 3, else 2-bit;
    # every case needs more than 64 bits (n = 32 and 64: all 128, no parent-edge tag)
    rng = np.random.default_rng(n * 7 + vals)
    start = [int(x) for x in rng.integers(0, vals, size=n)]
    start[:vals] = list(range(vals))
    gens = w.FAMILIES[family](n)
    rad = {"lrx": 9, "coxeter": 3, "pancake": 3 if n < 40 else 2}[family]
    want, rc = oracle.growth(n, gens, start=start, max_radius=rad)
    with cg.Growth(n, gens, max_radius=rad, start=start) as g:
        r = g.run()
        assert n * g.key_width > 64 and g.key_words == 2
    assert r.layers == want


@pytest.mark.parametrize("n,ones", [(70, 2), (100, 2), (124, 3), (128, 2)])
def test_binary_vectors_beyond_64_are_q_binomial(cg, n, ones):
    # adjacent transpositions on 1^m 0^(n-m): the growth of the whole orbit (C(n, m) states) is
    # the Gaussian binomial [n choose m]_q
    start = [1] * ones + [0] * (n - ones)
    r = cg.growth(n, w.coxeter(n), start=start)
    assert r.status == 0 and r.layers == q_multinomial((ones, n - ones))


def test_two_word_buffers_regrow(cg):
    # 26 elements of three values (18, 4, 4): 109,230,750 states in the orbit, more than the
    # first allocation of 2^22 states, so the states and the table grow (x4) and the table is
    # rebuilt from the stored states; the growth is the Gaussian multinomial [26; 18, 4, 4]_q
    counts = (18, 4, 4)
    start = [v for v, c in enumerate(counts) for _ in range(c)]
    with cg.Growth(26, w.coxeter(26), start=start) as g:
        r = g.run()
        st = g.stats()
    assert r.status == 0 and r.layers == q_multinomial(counts)
    assert r.total == math.factorial(26) // (math.factorial(18) * 24 * 24)
    assert st["state_capacity"] >= r.total and st["launches"] > 2


def test_two_word_memcap_truncation_and_last_layer(cg):
    n = 40
    start = [0] * 20 + [1] * 10 + [2] * 10
    np.random.default_rng(1).shuffle(start)
    start = [int(x) for x in start]
    full, _ = oracle.growth(n, w.coxeter(n), start=start, max_radius=5)   # 107,751 states
    r = cg.growth(n, w.coxeter(n), start=start, mem_cap=2 << 20)    # room for 16,383 states
    assert r.status == 2 and 1 < len(r.layers) <= len(full) and r.layers == full[:len(r.layers)]
    with cg.Growth(n, w.lrx(n), start=start, max_radius=6) as g:
        r = g.run()
        vecs = g.last_layer_vectors()
        keys = g.last_layer()
    assert keys.shape == (r.layers[-1], 2) and vecs.shape == (r.layers[-1], n)
    assert len({tuple(v) for v in vecs.tolist()}) == r.layers[-1]
    for v in vecs.tolist():
        assert sorted(v) == sorted(start)                 # rearrangements of the start vector


def test_constant_start_vector_is_fixed(cg):
    assert cg.growth(32, w.lrx(32), start=[15] * 32).layers == [1]
    assert cg.growth(64, w.coxeter(64)[:3], start=[3] * 64).layers == [1]
