"""GPU parity: layer counts from the CUDA path (through the C ABI) against the CPU oracle,
bit-exact (integer results: tolerance 0).  Sizes span many warp units and ragged tails;
the full-size workloads compare with stored oracle output (tests/golden/)."""

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
    vals = []
    for line in open(os.path.join(GOLDEN, name + ".txt")):
        if line.startswith("#") or not line.strip():
            continue
        r, c = line.split()
        assert int(r) == len(vals)
        vals.append(int(c))
    return vals


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


def test_s8_coxeter_full(cg):
    r = cg.growth(8, w.coxeter(8))
    assert r.status == 0
    assert r.layers == mahonian(8)
    assert r.layers == oracle.growth(8, w.coxeter(8))[0]


STRATS = ["hash", "bitmap", "auto"]


@pytest.mark.parametrize("strategy", STRATS)
def test_s11_lrx_full(cg, strategy):
    r = cg.growth(11, w.lrx(11), strategy=strategy)
    assert r.status == 0
    assert r.layers == golden("s11_lrx_growth")
    assert r.total == math.factorial(11)


@pytest.mark.parametrize("strategy", STRATS)
def test_s10_lx_directed(cg, strategy):
    r = cg.growth(10, w.lx(10), inverse_closed=False, strategy=strategy)
    assert r.layers == golden("s10_lx_growth")


@pytest.mark.parametrize("strategy", ["hash", "bitmap"])
@pytest.mark.parametrize("seed", range(24))
def test_random_sets_vs_oracle(cg, seed, strategy):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 10))
    k = int(rng.integers(1, 5))
    gens = w.random_perms(rng, n, k) if n > 1 else [[0]]
    if seed % 2 == 0:
        gens = w.inverse_closure(gens) or gens
    want, _ = oracle.growth(n, gens)
    got = cg.growth(n, gens, strategy=strategy)
    assert got.layers == want
    assert got.status == 0


@pytest.mark.parametrize("family", ["coxeter", "cyclic_coxeter", "all_transpositions", "star", "lrx",
                                    "lx", "pancake", "reversals", "transposons", "three_cycles",
                                    "cycles_01i_inv", "consecutive_3cycles_inv", "prefix_cycles"])
@pytest.mark.parametrize("n", [2, 3, 5, 7, 9])
@pytest.mark.parametrize("strategy", ["hash", "bitmap"])
def test_families_vs_oracle(cg, family, n, strategy):
    gens = w.FAMILIES[family](n)
    if not gens:
        pytest.skip("empty generating set")
    want, _ = oracle.growth(n, gens)
    assert cg.growth(n, gens, strategy=strategy).layers == want


def test_edge_cases(cg):
    assert cg.growth(1, [[0]]).layers == [1]
    assert cg.growth(4, [[0, 1, 2, 3]]).layers == [1]               # identity only
    assert cg.growth(2, [[1, 0]]).layers == [1, 1]
    g = w.coxeter(6)
    assert cg.growth(6, g + g).layers == mahonian(6)                  # duplicate rows
    c = w.cycle(16, list(range(16)))                                  # n = 16, cyclic group
    r = cg.growth(16, [c], inverse_closed=False)
    assert r.layers == [1] * 16
    r = cg.growth(16, w.coxeter(16), max_radius=6)                    # n = 16 keys use all 64 bits
    assert r.layers == mahonian(16)[:7] and r.status == 1


def test_radius_and_stop_limits(cg):
    m = mahonian(9)
    r = cg.growth(9, w.coxeter(9), max_radius=10)
    assert r.layers == m[:11] and r.status == 1
    r = cg.growth(9, w.coxeter(9), max_radius=0)
    assert r.layers == [1] and r.status == 1
    r = cg.growth(9, w.coxeter(9), stop_above=5000)
    assert r.status == 3 and r.layers[-1] > 5000 and max(r.layers[:-1]) <= 5000
    assert r.layers == m[:len(r.layers)]


@pytest.mark.parametrize("strategy", ["hash", "bitmap"])
def test_memcap_regrow_and_truncation(cg, strategy):
    want = golden("s11_lrx_growth")
    # grow-and-rebuild of the state array (and of the visited set) is exercised by n = 14: the
    # group order is too large to allocate up front, layers 0..7 hold 16.8M > 2^24 states
    r = cg.growth(14, w.pancake(14), max_radius=7, strategy=strategy)
    assert r.layers == golden("s14_pancake_layers")[:8]
    # a cap too small for the whole S11 growth: exact prefix, then CG_TRUNC_MEMCAP
    r = cg.growth(11, w.lrx(11), mem_cap=64 << 20, strategy=strategy)
    assert r.status == 2
    assert r.layers == want[:len(r.layers)] and len(r.layers) < len(want)


@pytest.mark.parametrize("strategy", ["hash", "bitmap"])
def test_last_layer_matches_oracle(cg, strategy):
    for n, gens in [(8, w.coxeter(8)), (7, w.reversals(7)), (8, w.lx(8)), (7, w.all_transpositions(7))]:
        g = cg.Growth(n, gens, keep_last=True, strategy=strategy)
        r = g.run()
        keys = np.sort(g.last_layer())
        want = oracle.layer_keys(n, gens, len(r.layers) - 1)
        assert np.array_equal(keys, want)
        g.close()


@pytest.mark.parametrize("kind,n,d,gens_text", [
    ("undirected", 10, 77, "(01)(23)(45)(68)(79); (45)(67)(89); (16)(24)(38)"),
    ("undirected", 11, 85, "(01)(23)(45)(67)(89); (13)(24)(56)(78)(9,10); (14)(23)"),
    ("directed", 11, 93, "(01)(23)(45)(67)(89); (1528)(47)(6,10)"),
    ("undirected", 12, 95, "(01)(23)(45)(67)(89)(10,11); (12)(35)(46)(78)(9,10); (36)(45)"),
    ("directed", 12, 106, "(01)(23)(45)(67)(89); (1,11,9,10)(04)(28)(36)"),
])
@pytest.mark.parametrize("strategy", ["hash", "bitmap"])
def test_published_max_diameters_gpu(cg, kind, n, d, gens_text, strategy):
    # Section 3.4 tables: the printed diameter and the layer sum n! (these sizes exceed what
    # the oracle finishes in seconds; the pins are the paper's numbers).
    gens = [w.from_cycles(n, t) for t in gens_text.split(";")]
    r = cg.growth(n, gens, inverse_closed=(kind == "undirected"), strategy=strategy)
    assert r.status == 0
    assert r.diameter == d
    assert r.total == math.factorial(n)


def test_batch_matches_oracle_and_single(cg):
    jobs = w.batch_groups(count=96)
    small = [j for j in jobs if j.n <= 8][:48]
    spec = [(j.n, j.gens, j.inverse_closed, -1) for j in small]
    with cg.Batch(spec) as b:
        res = b.run()
    for j, r in zip(small, res):
        want, _ = oracle.growth(j.n, j.gens)
        assert r.layers == want, j.name
        assert r.status == 0
    # the same job alone gives the same answer
    for j, r in list(zip(small, res))[:6]:
        assert cg.growth(j.n, j.gens).layers == r.layers


def test_batch_radius_caps_and_waves(cg):
    jobs = [(8, w.coxeter(8), True, r) for r in range(0, 12)] + [(7, w.lx(7), False, -1)]
    m = mahonian(8)
    with cg.Batch(jobs, mem_cap=8 << 20) as b:      # small budget: several waves
        res = b.run()
    for r, (n, g, inv, rad) in zip(res, jobs):
        if rad >= 0:
            assert r.layers == m[:rad + 1]
            assert r.status == 1
        else:
            assert r.layers == oracle.growth(7, w.lx(7))[0]


@pytest.mark.parametrize("wave_l2", [1 << 10, 256 << 10, 0, -1])
def test_batch_l2_waves_give_the_same_results(cg, wave_l2):
    # the L2 window only changes which jobs grow at the same time, never a result
    jobs = w.batch_groups(count=64)
    spec = [(j.n, j.gens, j.inverse_closed, -1) for j in jobs]
    with cg.Batch(spec, wave_l2=wave_l2) as b:
        res = b.run()
        launches = b.stats()["launches"]
    with cg.Batch(spec, wave_l2=-1) as b:
        ref = b.run()
    assert [r.layers for r in res] == [r.layers for r in ref]
    for j, r in list(zip(jobs, res))[:24:3]:
        assert r.layers == oracle.growth(j.n, j.gens)[0]
    # one persistent launch (plus its admission kernel) whatever the window: the cap only
    # changes how many jobs grow at once
    assert launches == 2


def test_step_expand_matches_gather(cg):
    # cg_expand (step K1 alone): t[i] = s[g[i]] for every generator and frontier state, laid out
    # generator-major, against the gather done by numpy indexing
    import torch
    from paper_2509_19162_gb300 import _cg
    rng = np.random.default_rng(5)
    for n, F in [(5, 1), (11, 1000), (16, 4099)]:
        perms = np.array([rng.permutation(n) for _ in range(F)], dtype=np.uint64)
        keys = (perms << (4 * np.arange(n, dtype=np.uint64))).sum(axis=1, dtype=np.uint64)
        gens = [list(rng.permutation(n)) for _ in range(3)]
        d_in = torch.tensor(keys.view(np.int64), device="cuda")
        d_out = torch.empty(3 * F, dtype=torch.int64, device="cuda")
        g = np.ascontiguousarray(np.array(gens, dtype=np.uint8))
        rc = _cg.cg_expand(n, 3, g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                           d_in.data_ptr(), F, d_out.data_ptr(), None)
        assert rc == 0
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint64).reshape(3, F)
        for j, gj in enumerate(gens):
            t = perms[:, gj]                                   # t[i] = s[g[i]]
            want = (t << (4 * np.arange(n, dtype=np.uint64))).sum(axis=1, dtype=np.uint64)
            assert np.array_equal(got[j], want)


def test_step_hash_insert_is_set_insert(cg):
    import torch
    from paper_2509_19162_gb300 import _cg
    rng = np.random.default_rng(9)
    slots = 1 << 16
    table = torch.empty(slots, dtype=torch.int64, device="cuda")
    assert _cg.cg_hash_clear(table.data_ptr(), slots, None) == 0
    seen = set()
    for N in (0, 1, 33, 5000, 20011):
        keys = rng.integers(0, 1 << 20, size=N, dtype=np.uint64)
        d_keys = torch.tensor(keys.view(np.int64), device="cuda")
        d_out = torch.empty(max(N, 1), dtype=torch.int64, device="cuda")
        d_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert _cg.cg_hash_insert(table.data_ptr(), slots, d_keys.data_ptr(), N, d_out.data_ptr(),
                                  d_cnt.data_ptr(), None) == 0
        torch.cuda.synchronize()
        c = int(d_cnt.item())
        new = np.sort(d_out[:c].cpu().numpy().view(np.uint64))
        want = np.array(sorted(set(int(x) for x in keys) - seen), dtype=np.uint64)
        assert np.array_equal(new, want)
        seen |= set(int(x) for x in keys)


def test_batch_with_hash_visited_sets(cg):
    # a job with n > 12 makes the whole batch use hash tables instead of rank bitmaps
    jobs = [(13, w.coxeter(13), True, 6), (9, w.lrx(9), True, -1), (7, w.lx(7), False, -1)]
    with cg.Batch(jobs) as b:
        res = b.run()
    assert res[0].layers == mahonian(13)[:7] and res[0].status == 1
    assert res[1].layers == oracle.growth(9, w.lrx(9))[0]
    assert res[2].layers == oracle.growth(7, w.lx(7))[0]


@pytest.mark.parametrize("strategy", ["bitmap", "hash", "sort"])
def test_config3_s14_pancake_full_size(cg, strategy):
    # Config 3 at full size: layers 0..10 (2.6e9 states in the last one) against oracle B.
    job = w.config_s14_pancake()
    r = cg.growth(job.n, job.gens, True, stop_above=job.stop_above, strategy=strategy)
    assert r.status == 3                                   # stopped above 2^31
    assert r.layers == golden("s14_pancake_layers_b")


def test_config4_full_batch_matches_oracle(cg):
    # Config 4 at full size: every one of the 4096 seeded groups, grown in one batch run, against
    # the oracle's growth vector of that group (tests/golden/batch4096_growth.txt)
    jobs = w.batch_groups()
    want = {}
    for line in open(os.path.join(GOLDEN, "batch4096_growth.txt")):
        if line.startswith("#"):
            continue
        f = [int(x) for x in line.split()]
        want[f[0]] = (f[1], f[2], f[3:])
    assert len(want) == len(jobs) == 4096
    spec = [(j.n, j.gens, j.inverse_closed, -1) for j in jobs]
    with cg.Batch(spec) as b:
        for _ in range(2):                         # the second run replays the resident plan
            res = b.run()
            for i, (j, r) in enumerate(zip(jobs, res)):
                n, k, layers = want[i]
                assert (n, k) == (j.n, j.k)
                assert r.status == 0 and r.layers == layers, f"group {i}"
