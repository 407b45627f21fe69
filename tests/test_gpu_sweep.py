"""GPU parity of the sweep strategy (bitmask BFS over S_n, Section 3.1.3): layers held as bitmaps
over the n! Lehmer ranks.  Checked against the oracle at small n and against closed forms and the
stored oracle values at sizes the oracle does not reach in seconds."""

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
    # all transpositions: layer r = c(n, n - r), unsigned Stirling numbers of the first kind
    c = [[0] * (n + 1) for _ in range(n + 1)]
    c[0][0] = 1
    for m in range(1, n + 1):
        for j in range(1, m + 1):
            c[m][j] = c[m - 1][j - 1] + (m - 1) * c[m - 1][j]
    return [c[n][n - r] for r in range(n)]


def golden(name):
    import os
    vals = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name + ".txt")):
        if line.startswith("#") or not line.strip():
            continue
        vals.append(int(line.split()[1]))
    return vals


@pytest.mark.parametrize("seed", range(24))
def test_random_sets_vs_oracle(cg, seed):
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.integers(2, 10))
    gens = w.random_perms(rng, n, int(rng.integers(1, 6)))
    if seed % 2 == 0:
        gens = w.inverse_closure(gens)
    r = cg.growth(n, gens, strategy="sweep")
    assert r.status == 0
    assert r.layers == oracle.growth(n, gens)[0]


@pytest.mark.parametrize("family", ["coxeter", "cyclic_coxeter", "all_transpositions", "star", "lrx",
                                    "lx", "pancake", "reversals", "transposons", "three_cycles",
                                    "prefix_cycles", "consecutive_4cycles"])
@pytest.mark.parametrize("n", [2, 3, 6, 9])
def test_families_vs_oracle(cg, family, n):
    gens = w.FAMILIES[family](n)
    if not gens:
        pytest.skip("empty generating set")
    assert cg.growth(n, gens, strategy="sweep").layers == oracle.growth(n, gens)[0]


@pytest.mark.parametrize("order", ["discovery", "rank"])
@pytest.mark.parametrize("family,n", [("pancake", 10), ("coxeter", 10), ("lrx", 9), ("star", 10),
                                      ("three_cycles", 8), ("reversals", 9)])
def test_block_orders_vs_oracle(cg, family, n, order):
    # every layer taken in one block order (auto mixes the two by layer density)
    gens = w.FAMILIES[family](n)
    with cg.Growth(n, gens, strategy="sweep") as g:
        g.set_sweep_order(order)
        assert g.run().layers == oracle.growth(n, gens)[0]


@pytest.mark.parametrize("order", ["discovery", "rank"])
def test_block_orders_s12_coxeter_and_start(cg, order):
    with cg.Growth(12, w.coxeter(12), strategy="sweep") as g:
        g.set_sweep_order(order)
        assert g.run().layers == mahonian(12)
    start = [3, 0, 7, 1, 6, 2, 5, 4, 8]
    gens = w.pancake(9)
    with cg.Growth(9, gens, strategy="sweep", start=start) as g:
        g.set_sweep_order(order)
        assert g.run().layers == oracle.growth(9, gens)[0]   # a coset of the whole group


def test_s11_lrx_and_s10_lx(cg):
    assert cg.growth(11, w.lrx(11), strategy="sweep").layers == golden("s11_lrx_growth")
    assert cg.growth(10, w.lx(10), inverse_closed=False, strategy="sweep").layers == golden("s10_lx_growth")


@pytest.mark.parametrize("n", [8, 12, 13])
def test_coxeter_mahonian_full_size(cg, n):
    r = cg.growth(n, w.coxeter(n), strategy="sweep")
    assert r.status == 0
    assert r.layers == mahonian(n)


@pytest.mark.parametrize("n", [9, 12])
def test_all_transpositions_stirling(cg, n):
    assert cg.growth(n, w.all_transpositions(n), strategy="sweep").layers == stirling_growth(n)


def test_s14_pancake_to_layer_10_vs_oracle_b(cg):
    # layers 0..10 of the S_14 pancake graph, stored from the rank-bitmap CPU oracle
    want = golden("s14_pancake_layers_b")
    r = cg.growth(14, w.pancake(14), strategy="sweep", max_radius=10)
    assert r.status == 1
    assert r.layers == want
    r = cg.growth(14, w.pancake(14), strategy="sweep", stop_above=2 ** 31)
    assert r.status == 3 and r.layers == want


@pytest.mark.parametrize("n,gens_fn,radius", [(8, w.coxeter, 28), (7, w.reversals, 6), (8, w.lx, None),
                                              (7, w.all_transpositions, 6)])
def test_last_layer_matches_oracle(cg, n, gens_fn, radius):
    gens = gens_fn(n)
    g = cg.Growth(n, gens, strategy="sweep", keep_last=True)
    r = g.run()
    keys = np.sort(g.last_layer())
    assert np.array_equal(keys, oracle.layer_keys(n, gens, len(r.layers) - 1))
    # a truncated run exports its last reported layer
    g2 = cg.Growth(n, gens, strategy="sweep", keep_last=True, max_radius=3)
    g2.run()
    assert np.array_equal(np.sort(g2.last_layer()), oracle.layer_keys(n, gens, 3))
    g.close()
    g2.close()


def test_start_and_rerun(cg):
    rng = np.random.default_rng(11)
    g = cg.Growth(9, w.lrx(9), strategy="sweep")
    want = oracle.growth(9, w.lrx(9))[0]
    assert g.run().layers == want
    assert g.run().layers == want                     # buffers reused, cleared per run
    g.set_start([int(x) for x in rng.permutation(9)])
    assert g.run().layers == want                     # vertex-transitive
    g.set_start(w.binary_start(9))
    with pytest.raises(RuntimeError):                 # repeated values: not a permutation
        g.run()
    g.close()


def test_limits(cg):
    m = mahonian(9)
    r = cg.growth(9, w.coxeter(9), strategy="sweep", max_radius=7)
    assert r.status == 1 and r.layers == m[:8]
    r = cg.growth(9, w.coxeter(9), strategy="sweep", stop_above=1000)
    assert r.status == 3 and r.layers == m[:len(r.layers)] and r.layers[-1] > 1000
    assert cg.growth(1, [[0]], strategy="sweep").layers == [1]


def test_whole_s14_coxeter_is_mahonian(cg):
    # all 14! = 87,178,291,200 states, 92 layers: the Mahonian numbers of n = 14
    r = cg.growth(14, w.coxeter(14), strategy="sweep")
    assert r.status == 0
    assert r.layers == mahonian(14)


def test_whole_s14_pancake(cg):
    # AUTO takes the sweep for the whole growth (the states would not fit as keys); the layers
    # sum to 14! and begin with the rank-bitmap CPU oracle's layers 0..10
    with cg.Growth(14, w.pancake(14)) as g:
        r = g.run()
        assert g.stats()["strategy_used"] == 4
    assert r.status == 0
    assert sum(r.layers) == math.factorial(14)
    assert r.layers[:11] == golden("s14_pancake_layers_b")


def _pack(p):
    return sum(int(v) << (4 * i) for i, v in enumerate(p))


def _rank_by_definition(p):
    # sum over positions i of (#{j < i : p_j < p_i}) * i!
    return sum(sum(1 for j in range(i) if p[j] < p[i]) * math.factorial(i) for i in range(len(p)))


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_perm_rank_is_a_bijection(cg, n):
    import itertools
    import torch
    from paper_2509_19162_gb300 import _cg
    perms = list(itertools.permutations(range(n)))
    keys = np.array([_pack(p) for p in perms], dtype=np.uint64)
    d_keys = torch.tensor(keys.view(np.int64), device="cuda")
    d_ranks = torch.empty_like(d_keys)
    d_back = torch.empty_like(d_keys)
    assert _cg.cg_perm_rank(n, d_keys.data_ptr(), len(keys), d_ranks.data_ptr(), None) == 0
    assert _cg.cg_perm_unrank(n, d_ranks.data_ptr(), len(keys), d_back.data_ptr(), None) == 0
    torch.cuda.synchronize()
    ranks = d_ranks.cpu().numpy().view(np.uint64)
    assert sorted(int(r) for r in ranks) == list(range(math.factorial(n)))
    assert np.array_equal(d_back.cpu().numpy().view(np.uint64), keys)
    for p, r in list(zip(perms, ranks))[:: max(1, len(perms) // 500)]:
        assert int(r) == _rank_by_definition(p)


@pytest.mark.parametrize("n", [13, 14, 16])
def test_perm_rank_large_n(cg, n):
    import torch
    from paper_2509_19162_gb300 import _cg
    rng = np.random.default_rng(n)
    perms = [list(range(n)), list(range(n))[::-1]] + [list(rng.permutation(n)) for _ in range(2000)]
    keys = np.array([_pack(p) for p in perms], dtype=np.uint64)
    d_keys = torch.tensor(keys.view(np.int64), device="cuda")
    d_ranks = torch.empty_like(d_keys)
    d_back = torch.empty_like(d_keys)
    assert _cg.cg_perm_rank(n, d_keys.data_ptr(), len(keys), d_ranks.data_ptr(), None) == 0
    assert _cg.cg_perm_unrank(n, d_ranks.data_ptr(), len(keys), d_back.data_ptr(), None) == 0
    torch.cuda.synchronize()
    ranks = [int(r) for r in d_ranks.cpu().numpy().view(np.uint64)]
    assert ranks[0] == math.factorial(n) - 1 and ranks[1] == 0     # identity, full reversal
    assert all(r == _rank_by_definition(p) for p, r in zip(perms, ranks))
    assert np.array_equal(d_back.cpu().numpy().view(np.uint64), keys)


@pytest.mark.parametrize("strategy", ["sweep", "bitmap"])
def test_whole_s13_pancake_vs_oracle_c(cg, strategy):
    # all 13! states; the 16 layers stored from the layer-bitmap CPU oracle (oracle C)
    r = cg.growth(13, w.pancake(13), strategy=strategy)
    assert r.status == 0
    assert r.layers == golden("s13_pancake_growth")


@pytest.mark.parametrize("family", ["pancake", "lrx"])
@pytest.mark.parametrize("strategy", ["sweep", "bitmap", "hash"])
def test_whole_s12_vs_oracle_b(cg, family, strategy):
    # all 12! states against the classic-Lehmer-rank CPU oracle (oracle B), whose whole S_12
    # growths also equal oracle C's (tests/golden/s12_*_growth_b.txt, _c.txt)
    r = cg.growth(12, w.FAMILIES[family](12), strategy=strategy)
    assert r.status == 0
    assert r.layers == golden(f"s12_{family}_growth_b")
