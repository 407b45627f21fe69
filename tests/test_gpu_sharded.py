"""GPU: the sharded growth (one graph over P ranks, one exchange per layer) run as P logical
ranks on one GPU in one process -- the owner partition (cg_shard_expand) and insert-if-absent
(cg_hash_insert) kernels with the exchange done as device copies.  The merged growth must equal
the oracle's; the partition must be the gather expansion grouped by owner."""

import ctypes

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


@pytest.mark.parametrize("P", [1, 2, 3, 5, 8])
def test_sharded_growth_equals_oracle(cg, P):
    from paper_2509_19162_gb300.sharded import sharded_growth_local
    assert sharded_growth_local(8, w.coxeter(8), P).layers == mahonian(8)
    for n, gens in [(9, w.lrx(9)), (8, w.lx(8)), (7, w.pancake(7))]:
        assert sharded_growth_local(n, gens, P).layers == oracle.growth(n, gens)[0]
    rng = np.random.default_rng(10 + P)
    gens = w.random_perms(rng, 7, 2)
    assert sharded_growth_local(7, gens, P).layers == oracle.growth(7, gens)[0]
    r = sharded_growth_local(10, w.coxeter(10), P, max_radius=9)
    assert r.layers == mahonian(10)[:10] and r.status == 1


def test_sharded_s11_lrx_four_ranks(cg):
    import os
    from paper_2509_19162_gb300.sharded import sharded_growth_local
    golden = os.path.join(os.path.dirname(__file__), "golden", "s11_lrx_growth.txt")
    want = [int(l.split()[1]) for l in open(golden) if not l.startswith("#")]
    assert sharded_growth_local(11, w.lrx(11), 4).layers == want


def test_shard_expand_groups_the_gather_by_owner(cg):
    import torch
    from paper_2509_19162_gb300 import _cg
    from paper_2509_19162_gb300.sharded import owner
    rng = np.random.default_rng(2)
    n, F, P = 10, 3001, 6
    perms = np.array([rng.permutation(n) for _ in range(F)], dtype=np.uint64)
    sh = (4 * np.arange(n)).astype(np.uint64)
    keys = (perms << sh).sum(axis=1, dtype=np.uint64)
    gens = [list(rng.permutation(n)) for _ in range(4)]
    g = np.ascontiguousarray(np.array(gens, dtype=np.uint8))
    d_in = torch.tensor(keys.view(np.int64), device="cuda")
    d_out = torch.empty(4 * F, dtype=torch.int64, device="cuda")
    counts = np.zeros(P, dtype=np.uint64)
    assert _cg.cg_shard_expand(n, 4, g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), d_in.data_ptr(), F, P,
                               d_out.data_ptr(), 4 * F,
                               counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), None) == 0
    got = d_out.cpu().numpy().view(np.uint64)
    want = np.concatenate([((perms[:, gj] << sh).sum(axis=1, dtype=np.uint64)) for gj in gens])
    assert int(counts.sum()) == 4 * F
    assert np.array_equal(np.sort(got), np.sort(want))
    o = 0
    for p in range(P):
        part = got[o:o + int(counts[p])]
        assert all(owner(int(x), P) == p for x in part[:: max(1, len(part) // 200)])
        o += int(counts[p])
    # a buffer too small is refused before any work
    assert _cg.cg_shard_expand(n, 4, g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), d_in.data_ptr(), F, P,
                               d_out.data_ptr(), 4 * F - 1,
                               counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), None) == _cg.CG_EINVAL
