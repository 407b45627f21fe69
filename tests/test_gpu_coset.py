"""GPU parity of Schreier coset growth (growth of the orbit of a central state, Section 3.1.2
and Section 3.2) through the C ABI, against the oracle and against closed forms at sizes the
oracle does not reach in seconds."""

import math

import numpy as np
import pytest

import oracle
import workloads as w
from test_oracle_coset_pins import q_multinomial

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available()
    import paper_2509_19162_gb300 as p
    p.build()
    return p


@pytest.mark.parametrize("strategy", ["hash", "auto", "sort"])
@pytest.mark.parametrize("seed", range(16))
def test_random_cosets_vs_oracle(cg, seed, strategy):
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(2, 13))
    gens = w.random_perms(rng, n, int(rng.integers(1, 4)))
    if strategy == "sort" or seed % 2 == 0:
        gens = w.inverse_closure(gens)
    start = [int(x) for x in rng.integers(0, int(rng.integers(1, n + 1)), size=n)]
    want, _ = oracle.growth(n, gens, start=start)
    got = cg.growth(n, gens, strategy=strategy, start=start)
    assert got.status == 0
    assert got.layers == want


@pytest.mark.parametrize("family", ["lrx", "pancake", "transposons", "reversals", "coxeter",
                                    "consecutive_4cycles", "star", "lx"])
@pytest.mark.parametrize("n", [5, 12, 16])
def test_binary_cosets_vs_oracle(cg, family, n):
    gens = w.FAMILIES[family](n)
    start = w.binary_start(n)
    want, _ = oracle.growth(n, gens, start=start)
    for strategy in ("hash", "auto"):
        assert cg.growth(n, gens, strategy=strategy, start=start).layers == want


@pytest.mark.parametrize("strategy", ["hash", "bitmap", "sort"])
def test_permutation_start_is_a_copy_of_the_group(cg, strategy):
    # distinct entries: the orbit is the regular action, growth equal to that from e
    rng = np.random.default_rng(7)
    for n, gens in [(9, w.lrx(9)), (8, w.pancake(8)), (10, w.coxeter(10))]:
        perm = [int(x) for x in rng.permutation(n)]
        assert cg.growth(n, gens, strategy=strategy, start=perm).layers == oracle.growth(n, gens)[0]


def test_bitmap_rejects_repeated_entries_and_start_resets(cg):
    g = cg.Growth(8, w.coxeter(8), strategy="bitmap", start=w.binary_start(8))
    with pytest.raises(RuntimeError):
        g.run()
    g.close()
    g = cg.Growth(8, w.coxeter(8), start=w.binary_start(8), keep_last=True)
    r = g.run()
    assert r.layers == q_multinomial((4, 4))
    assert g.key_width == 1                              # binary vector: one bit per element
    assert list(np.sort(g.last_layer())) == [sum(v << i for i, v in enumerate([1] * 4 + [0] * 4))]
    assert g.last_layer_vectors().tolist() == [[1] * 4 + [0] * 4]
    g.set_start(None)
    assert g.run().layers == oracle.growth(8, w.coxeter(8))[0]
    g.set_start([3, 3, 2, 2, 1, 1, 0, 0])
    assert g.run().layers == q_multinomial((2, 2, 2, 2))
    g.close()


@pytest.mark.parametrize("strategy", ["hash", "sort"])
def test_full_size_multiset_orbit_is_q_multinomial(cg, strategy):
    # 16 entries, four values four times each: 16! / (4!)^4 = 63,063,000 states, growth the
    # Gaussian multinomial [16; 4,4,4,4]_q (adjacent transpositions count inversions).
    counts = (4, 4, 4, 4)
    start = [v for v, c in enumerate(counts) for _ in range(c)]
    r = cg.growth(16, w.coxeter(16), strategy=strategy, start=start)
    assert r.status == 0
    assert r.total == math.factorial(16) // math.factorial(4) ** 4
    assert r.layers == q_multinomial(counts)


def test_binary_coset_n16_lrx_closed_form(cg):
    g = cg.growth(16, w.lrx(16), start=w.binary_start(16))
    assert len(g.layers) - 1 == (16 * 44 + 32) // 16
    assert g.total == math.comb(16, 8)


# ---- long vectors: 1 or 2 bits per element (n up to 60 / 30) ----------------------------

@pytest.mark.parametrize("n", [17, 20, 22])
@pytest.mark.parametrize("family", ["lrx", "pancake", "reversals", "coxeter", "consecutive_4cycles", "star"])
def test_binary_vectors_beyond_16_vs_oracle(cg, n, family):
    gens = w.FAMILIES[family](n)
    start = w.binary_start(n)
    want, _ = oracle.growth(n, gens, start=start)
    for strategy in ("hash", "auto"):
        assert cg.growth(n, gens, strategy=strategy, start=start).layers == want
    if w.is_inverse_closed(gens):
        assert cg.growth(n, gens, strategy="sort", start=start).layers == want


@pytest.mark.parametrize("seed", range(8))
def test_two_bit_vectors_vs_oracle(cg, seed):
    rng = np.random.default_rng(7000 + seed)
    n = int(rng.integers(10, 19))
    start = [int(x) for x in rng.integers(0, 4, size=n)]
    start[0], start[1] = 3, 2            # values up to 3: two bits per element
    gens = w.random_perms(rng, n, 2)
    if seed % 2 == 0:
        gens = w.inverse_closure(gens)
    want, _ = oracle.growth(n, gens, start=start, max_radius=12)
    got = cg.growth(n, gens, start=start, max_radius=12)
    assert got.layers == want


@pytest.mark.parametrize("n", [26, 28, 30, 32])
def test_binary_lrx_gods_number_large_n(cg, n):
    # Schreier-graph table, LRX on the binary coset: (n(3n-4) + 32 - 2(n mod 4)) / 16 for even n
    r = cg.growth(n, w.lrx(n), start=w.binary_start(n))
    assert r.status == 0
    assert len(r.layers) - 1 == (n * (3 * n - 4) + 32 - 2 * (n % 4)) // 16
    assert r.total == math.comb(n, n // 2)


@pytest.mark.parametrize("n", [24, 25, 30, 31])
def test_binary_consecutive_4cycles_large_n(cg, n):
    # Section 3.2: n^2/12 + 1 (n = 0 mod 6) and (n^2 + 4n - 5)/12 (n = 1 mod 6)
    r = cg.growth(n, w.consecutive_4cycles(n), start=w.binary_start(n))
    want = n * n // 12 + 1 if n % 6 == 0 else (n * n + 4 * n - 5) // 12
    assert len(r.layers) - 1 == want and r.total == math.comb(n, n // 2)


@pytest.mark.parametrize("n", [28, 32])
def test_binary_reversals_large_n(cg, n):
    # Schreier-graph table: God's number floor(n/2) for reversals on the binary coset
    r = cg.growth(n, w.reversals(n), start=w.binary_start(n))
    assert len(r.layers) - 1 == n // 2 and r.total == math.comb(n, n // 2)


def test_long_vector_limits(cg):
    with pytest.raises(RuntimeError):          # the identity of S_26 needs more than 128 bits
        cg.growth(26, w.coxeter(26), max_radius=2)
    with pytest.raises(Exception):             # 33 elements of 4 bits do not fit 128 bits
        cg.growth(33, w.coxeter(33), start=[5] + [0] * 32)
    # 62 elements of 2 bits take two-word keys: the orbit of 3 0^61 is the 62 positions of the 3
    r = cg.growth(62, w.coxeter(62), start=[3] + [0] * 61)
    assert r.layers == [1] * 62
