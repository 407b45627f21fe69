"""GPU parity of the sort strategy (radix sort + unique, merge-path set difference, look-back
compaction) and of its step-level entry points, against numpy and the CPU oracle."""

import ctypes
import math
import os

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    return [int(l.split()[1]) for l in open(os.path.join(GOLDEN, name + ".txt")) if not l.startswith("#")]


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available()
    import paper_2509_19162_gb300 as p
    p.build()
    return p


def _dev(arr):
    import torch
    return torch.tensor(np.asarray(arr, dtype=np.uint64).view(np.int64), device="cuda")


def _scratch(lib, n):
    import torch
    nb = lib.cg_sort_unique_scratch_bytes(max(n, 1))
    return torch.empty(nb, dtype=torch.uint8, device="cuda"), nb


@pytest.mark.parametrize("n,bits,hi", [(0, 8, 10), (1, 8, 10), (4095, 44, 1 << 44), (4096, 12, 1 << 12),
                                       (4097, 64, None), (100003, 20, 5000), ((1 << 20) + 7, 56, 1 << 56)])
def test_sort_unique_matches_numpy(cg, n, bits, hi):
    import torch
    from paper_2509_19162_gb300 import _cg
    rng = np.random.default_rng(n + bits)
    if hi is None:
        keys = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
    else:
        keys = rng.integers(0, hi, size=n, dtype=np.uint64)
    d = _dev(keys) if n else torch.empty(1, dtype=torch.int64, device="cuda")
    out = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    scr, nb = _scratch(_cg, n)
    rc = _cg.cg_sort_unique(d.data_ptr(), n, bits, out.data_ptr(), cnt.data_ptr(), scr.data_ptr(), nb, None)
    assert rc == 0
    torch.cuda.synchronize()
    c = int(cnt.item())
    want_sorted = np.sort(keys)
    want_unique = np.unique(keys)
    if n:
        assert np.array_equal(d.cpu().numpy().view(np.uint64), want_sorted)
    assert c == len(want_unique)
    assert np.array_equal(out[:c].cpu().numpy().view(np.uint64), want_unique)


@pytest.mark.parametrize("seed", range(6))
def test_set_difference_matches_numpy(cg, seed):
    import torch
    from paper_2509_19162_gb300 import _cg
    rng = np.random.default_rng(seed)
    na, nb, nc = [int(x) for x in rng.integers(0, 200000, size=3)]
    if seed == 0:
        nb = nc = 0
    universe = int(rng.integers(10, 400000))
    a = np.sort(rng.integers(0, universe, size=na, dtype=np.uint64))
    b = np.unique(rng.integers(0, universe, size=nb, dtype=np.uint64))
    c = np.unique(rng.integers(0, universe, size=nc, dtype=np.uint64))
    da = _dev(a) if na else torch.empty(1, dtype=torch.int64, device="cuda")
    db = _dev(b) if len(b) else None
    dc = _dev(c) if len(c) else None
    out = torch.empty(max(na, 1), dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    scr, nbytes = _scratch(_cg, na)
    rc = _cg.cg_set_difference(da.data_ptr(), na, db.data_ptr() if db is not None else None, len(b),
                               dc.data_ptr() if dc is not None else None, len(c), out.data_ptr(),
                               cnt.data_ptr(), scr.data_ptr(), nbytes, None)
    assert rc == 0
    torch.cuda.synchronize()
    want = np.setdiff1d(np.setdiff1d(np.unique(a), b), c)
    k = int(cnt.item())
    assert k == len(want)
    assert np.array_equal(out[:k].cpu().numpy().view(np.uint64), want)


def test_sort_strategy_s11_lrx(cg):
    r = cg.growth(11, w.lrx(11), strategy="sort")
    assert r.status == 0 and r.layers == golden("s11_lrx_growth")


@pytest.mark.parametrize("family", ["coxeter", "all_transpositions", "lrx", "pancake", "reversals",
                                    "cycles_01i_inv", "consecutive_3cycles_inv", "star"])
@pytest.mark.parametrize("n", [2, 4, 7, 9])
def test_sort_strategy_families(cg, family, n):
    gens = w.FAMILIES[family](n)
    if not gens or not w.is_inverse_closed(gens):
        pytest.skip("not an inverse-closed set")
    want, _ = oracle.growth(n, gens)
    assert cg.growth(n, gens, strategy="sort").layers == want


@pytest.mark.parametrize("seed", range(12))
def test_sort_equals_hash_on_random_undirected_sets(cg, seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(3, 11))
    gens = w.inverse_closure(w.random_perms(rng, n, int(rng.integers(1, 4))))
    a = cg.growth(n, gens, strategy="sort")
    b = cg.growth(n, gens, strategy="hash")
    assert a.layers == b.layers and a.status == b.status == 0
    if n <= 8:
        assert a.layers == oracle.growth(n, gens)[0]


def test_sort_strategy_limits_and_last_layer(cg):
    g = cg.Growth(8, w.coxeter(8), strategy="sort", keep_last=True)
    r = g.run()
    assert list(g.last_layer()) == [sum((7 - i) << (4 * i) for i in range(8))]
    g.close()
    r = cg.growth(9, w.coxeter(9), strategy="sort", max_radius=10)
    assert r.status == 1 and r.layers == oracle.growth(9, w.coxeter(9), max_radius=10)[0]
    r = cg.growth(9, w.coxeter(9), strategy="sort", stop_above=5000)
    assert r.status == 3 and r.layers[-1] > 5000
    want = golden("s11_lrx_growth")
    r = cg.growth(11, w.lrx(11), strategy="sort", mem_cap=48 << 20)
    assert r.status == 2 and r.layers == want[:len(r.layers)]


def test_sort_small_steps_stop_inside_one_block(cg):
    # Steps of at most 4096 candidates run back to back in one block on the device, with the host
    # loop's stop tests: a radius cap and a layer-size stop that fire inside them, and a growth all
    # of whose steps are small, whose last layer comes out of those steps.
    want = oracle.growth(8, w.coxeter(8))[0]
    r = cg.growth(8, w.coxeter(8), strategy="sort", max_radius=3)
    assert r.status == 1 and r.layers == want[:4]
    r = cg.growth(8, w.coxeter(8), strategy="sort", stop_above=100)
    first = next(i for i, x in enumerate(want) if x > 100)
    assert r.status == 3 and r.layers == want[:first + 1]
    g = cg.Growth(6, w.lrx(6), strategy="sort", keep_last=True)
    r = g.run()
    assert r.status == 0 and r.layers == oracle.growth(6, w.lrx(6))[0]
    last = np.sort(np.asarray(g.last_layer(), dtype=np.uint64))
    g.close()
    assert np.array_equal(last, oracle.layer_keys(6, w.lrx(6), len(r.layers) - 1))


def test_sort_strategy_key_range_chunks(cg):
    # 200 MB holds the three largest layers of S_11 LRX but not their 9.15M candidates at once:
    # the large steps run in key-range chunks (top-digit histogram, then one sort per range)
    r = cg.growth(11, w.lrx(11), strategy="sort", mem_cap=200 << 20)
    assert r.status == 0 and r.layers == golden("s11_lrx_growth")
    r = cg.growth(11, w.lrx(11), strategy="sort", mem_cap=120 << 20)
    want = golden("s11_lrx_growth")
    assert r.layers == want[:len(r.layers)] and (r.status == 0 or r.status == 2)


def test_sort_strategy_s12_pancake_whole(cg):
    # all 12! states through the sorted two-layer step (11 generators), against oracle B
    r = cg.growth(12, w.pancake(12), strategy="sort")
    assert r.status == 0 and r.layers == golden("s12_pancake_growth_b")
