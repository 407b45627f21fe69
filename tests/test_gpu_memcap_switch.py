"""GPU: an undirected growth whose stored states outgrow mem_cap goes on with the sorted layer
step, which keeps only the last two layers (in an undirected graph the neighbours of layer r lie
in layers r-1, r and r+1).  The layers must equal the oracle's, before and after the switch."""

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

SORT = 2   # CG_STRATEGY_SORT


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available()
    import paper_2509_19162_gb300 as p
    p.build()
    return p


def test_s9_lrx_switches_and_completes(cg):
    # 362,880 states as keys (2.9 MB) do not fit 3300 KiB beside the 1 MiB reserve; the sorted
    # step needs at most 2.8 MB for any layer of S_9 LRX.  max_radius (beyond the diameter 36)
    # keeps AUTO off the bitmask sweep.
    gens = w.lrx(9)
    want, _ = oracle.growth(9, gens)
    with cg.Growth(9, gens, max_radius=40, mem_cap=3300 << 10, keep_last=True) as g:
        for _ in range(2):     # the second run on the handle starts from the key store again
            r = g.run()
            st = g.stats()
            assert r.status == 0 and r.layers == want
            assert st["switched_to_sort"] == 1 and st["strategy_used"] == SORT
            assert 0 < st["sort_from"] < len(want) - 1
            last = np.sort(g.last_layer())
            assert np.array_equal(last, oracle.layer_keys(9, gens, len(want) - 1))


def test_binary_coset_switches_and_completes(cg):
    # Schreier coset graph of LRX on the 705,432 binary strings of length 22 with eleven ones:
    # a hash table (the start has repeated values), tagged 1-bit keys
    gens = w.lrx(22)
    start = [0] * 11 + [1] * 11
    want, _ = oracle.growth(22, gens, start=start)
    with cg.Growth(22, gens, mem_cap=2500 << 10, start=start) as g:
        r = g.run()
        st = g.stats()
    assert r.status == 0 and r.layers == want
    assert st["switched_to_sort"] == 1 and 0 < st["sort_from"] < len(want) - 1


def test_sorted_step_truncates_exactly(cg):
    # at 1000 KiB the switch happens but the sorted step itself runs out later (the two largest
    # layers and the next one's buffer leave no room for candidates): an exact prefix
    gens = w.lrx(9)
    want, _ = oracle.growth(9, gens)
    with cg.Growth(9, gens, max_radius=40, mem_cap=1000 << 10) as g:
        r = g.run()
        st = g.stats()
    assert r.status == 2                      # CG_TRUNC_MEMCAP
    assert 1 < len(r.layers) < len(want) and r.layers == want[:len(r.layers)]
    assert st["switched_to_sort"] == 1
    # at 1600 KiB the sorted step completes: its largest steps (112,548 candidates, 1.9 MB at
    # once) run in key-range chunks beside the three layers
    with cg.Growth(9, gens, max_radius=40, mem_cap=1600 << 10) as g:
        r = g.run()
        assert r.status == 0 and r.layers == want and g.stats()["switched_to_sort"] == 1


def test_directed_set_keeps_the_truncation(cg):
    # LX is not closed under inverses: the two-layer step does not apply
    gens = w.lx(9)
    want, _ = oracle.growth(9, gens)
    with cg.Growth(9, gens, max_radius=60, mem_cap=2000 << 10) as g:
        r = g.run()
        st = g.stats()
    assert r.status == 2 and r.layers == want[:len(r.layers)] and len(r.layers) < len(want)
    assert st["switched_to_sort"] == 0 and st["strategy_used"] != SORT
