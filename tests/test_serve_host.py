"""Host logic of the serving loop's admission (no GPU): the predicted states of a job bound the
states it can really reach by its radius cap, and the memory it is admitted with stays within
its share of the budget.  The bounds are checked against closed forms the paper states: the
Mahonian numbers for adjacent transpositions and the unsigned Stirling numbers of the first kind
for all transpositions (Section 3.3 table)."""

import math

import numpy as np
import pytest

import paper_2509_19162_gb300 as cgp

cgp.build()
from paper_2509_19162_gb300.serve import Server  # noqa: E402  (needs the built library)

import workloads as w  # noqa: E402

GiB = 1 << 30


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


@pytest.mark.parametrize("n", [8, 11, 13, 16])
@pytest.mark.parametrize("cap", [6, 9, 14, -1])
def test_prediction_bounds_the_reachable_states(n, cap):
    for gens, growth in ((w.coxeter(n), mahonian(n)), (w.all_transpositions(n), stirling_growth(n))):
        p = Server.predict(n, gens, True, cap, job_mem_cap=160 * GiB)
        reach = sum(growth[:cap + 1]) if cap >= 0 else sum(growth)
        assert p["states"] >= reach
        assert p["states"] <= math.factorial(n)
        if cap < 0:
            assert p["states"] == math.factorial(n)          # unlimited: the group order


def test_share_bounds_the_admitted_memory():
    for share in (1 << 20, 64 << 20, 2 * GiB):
        for n, gens, cap in [(16, w.coxeter(16), 60), (12, w.lrx(12), 40), (9, w.pancake(9), 6),
                             (10, w.all_transpositions(10), 9)]:
            p = Server.predict(n, gens, True, cap, job_mem_cap=share)
            assert 1 <= p["granted"] <= p["states"]
            assert p["bytes"] <= share + 256
    # small prediction: admitted with what it needs, not with the share
    p = Server.predict(8, w.coxeter(8), True, 2, job_mem_cap=2 * GiB)
    assert p["granted"] == p["states"] == 1 + 7 + 7 * 6 and p["bytes"] < (1 << 20)
    # S_12 whole: the rank bitmap (60 MB) stores more states in the share than a hash table
    p = Server.predict(12, w.lrx(12), True, -1, job_mem_cap=2 * GiB)
    assert p["granted"] > (2 * GiB) // 24


def test_prediction_rejects_bad_input():
    from paper_2509_19162_gb300 import _cg
    with pytest.raises(_cg.CgError):
        Server.predict(5, [[0, 1, 2, 3, 3]], True, 3)
    with pytest.raises(_cg.CgError):
        Server.predict(5, [[1, 2, 3, 4, 0]], True, 3)      # a 5-cycle without its inverse
