"""cg_growth_run_noalloc: the growth entry point for callers that cannot allocate device memory
(sandboxed or pool-capped code, processes that forbid cudaMalloc after start-up, plugins whose
host owns every allocation).  It keeps all of its buffers in one fixed array inside the library.

Checked through the C ABI against the allocating entry point (cg_growth_create / _run /
_destroy) on consecutive calls -- the fixed array keeps the previous call's contents, so a call
that forgot to clear it would show up in the second call -- and against the oracle and the
Mahonian numbers, with the tolerance of every growth test: exact layer counts (integers).  This
file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    import paper_2509_19162_gb300 as p
    p.build()
    from paper_2509_19162_gb300 import _cg
    return _cg


def mahonian(n):
    poly = np.array([1], dtype=object)
    for j in range(1, n + 1):
        poly = np.convolve(poly, np.ones(j, dtype=object))
    return [int(x) for x in poly]


def run_noalloc(lib, n, gens, inverse_closed, max_radius=-1, cap=4096, stream=None):
    g = np.ascontiguousarray(np.asarray(gens, dtype=np.uint8))
    out = np.zeros(cap, dtype=np.uint64)
    nl = ctypes.c_int(0)
    rc = lib.cg_growth_run_noalloc(n, len(gens), g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                   int(inverse_closed), int(max_radius), stream,
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap,
                                   ctypes.byref(nl))
    return rc, [int(x) for x in out[:nl.value]]


def run_allocating(lib, n, gens, inverse_closed, max_radius=-1, cap=4096):
    g = np.ascontiguousarray(np.asarray(gens, dtype=np.uint8))
    h = ctypes.c_void_p()
    assert lib.cg_growth_create(n, len(gens), g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                int(inverse_closed), int(max_radius), 0, ctypes.byref(h)) == 0
    out = np.zeros(cap, dtype=np.uint64)
    nl = ctypes.c_int(0)
    rc = lib.cg_growth_run(h, None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap,
                           ctypes.byref(nl))
    lib.cg_growth_destroy(h)
    return rc, [int(x) for x in out[:nl.value]]


# n = 16: keys use all 64 bits, so states carry no parent-edge tag
C16 = w.cycle(16, list(range(16)))
CASES = [
    (9, w.lrx(9), True, -1),          # 362,880 states: large table use first
    (8, w.coxeter(8), True, -1),      # then a smaller group over the previous call's contents
    (9, w.lx(9), False, -1),          # directed
    (10, w.lrx(10), True, 12),        # truncated growth of a group larger than the scratch
    (16, w.coxeter(16), True, 5),     # untagged 64-bit keys
    (16, [C16], False, -1),           # n = 16, cyclic group of order 16
]


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(lib):
    for n, gens, inv, rad in CASES + CASES[:2]:
        rc_a, got = run_noalloc(lib, n, gens, inv, rad)
        rc_b, want = run_allocating(lib, n, gens, inv, rad)
        assert rc_a == rc_b and rc_a >= 0
        assert got == want


def test_noalloc_matches_oracle_and_closed_forms(lib):
    assert run_noalloc(lib, 8, w.coxeter(8), True) == (0, mahonian(8))
    assert run_noalloc(lib, 16, w.coxeter(16), True, 5) == (lib.CG_TRUNC_RADIUS, mahonian(16)[:6])
    assert run_noalloc(lib, 16, [C16], False) == (0, [1] * 16)
    for n, gens, inv, rad in [(9, w.lrx(9), True, -1), (9, w.lx(9), False, -1),
                              (8, w.pancake(8) + w.pancake(8), True, -1),      # repeated rows
                              (7, w.all_transpositions(7), True, 4)]:
        rc, got = run_noalloc(lib, n, gens, inv, rad)
        want, orc = oracle.growth(n, gens, max_radius=rad)
        assert got == want and (rc == 0) == (orc == 0)


def test_noalloc_on_a_caller_stream(lib):
    import torch
    s = torch.cuda.Stream()
    for _ in range(2):
        rc, got = run_noalloc(lib, 9, w.lrx(9), True, stream=s.cuda_stream)
        assert rc == 0 and got == oracle.growth(9, w.lrx(9))[0]


def test_noalloc_rejects_problems_beyond_its_fixed_size(lib):
    rc, _ = run_noalloc(lib, 10, w.lrx(10), True)          # 3,628,800 states > 2^20
    assert rc == lib.CG_ETOOBIG
    rng = np.random.default_rng(3)
    many = [list(p) for p in {tuple(rng.permutation(8)) for _ in range(400)}][:300]
    rc, _ = run_noalloc(lib, 8, many, False)               # 300 distinct rows > 256
    assert rc == lib.CG_ETOOBIG
    rc, got = run_noalloc(lib, 8, [w.coxeter(8)[0]] * 300, True)   # one distinct row
    assert rc == 0 and got == [1, 1]
    # and the next call still works
    rc, got = run_noalloc(lib, 8, w.coxeter(8), True)
    assert rc == 0 and got == run_allocating(lib, 8, w.coxeter(8), True)[1]
