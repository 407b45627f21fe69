"""cg_growth_run_noalloc: the growth entry point for callers that cannot allocate device memory
(sandboxed or pool-capped code, processes that forbid cudaMalloc after start-up, plugins whose
host owns every allocation).  It keeps all of its buffers in one fixed array inside the library.

Checked through the C ABI against the allocating entry point (cg_growth_create / _run /
_destroy) on consecutive calls -- the fixed array keeps the previous call's contents, so a call
that forgot to clear it would show up in the second call -- with the tolerance of every growth
test: exact layer counts (integers).  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

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


def run_noalloc(lib, n, gens, inverse_closed, max_radius=-1, cap=4096):
    g = np.ascontiguousarray(np.asarray(gens, dtype=np.uint8))
    out = np.zeros(cap, dtype=np.uint64)
    nl = ctypes.c_int(0)
    rc = lib.cg_growth_run_noalloc(n, len(gens), g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                   int(inverse_closed), int(max_radius), None,
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


CASES = [
    (9, w.lrx(9), True, -1),          # 362,880 states: large table use first
    (8, w.coxeter(8), True, -1),      # then a smaller group over the previous call's contents
    (9, w.lx(9), False, -1),          # directed
    (10, w.lrx(10), True, 12),        # truncated growth of a group larger than the scratch
]


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(lib):
    for n, gens, inv, rad in CASES + CASES[:2]:
        rc_a, got = run_noalloc(lib, n, gens, inv, rad)
        rc_b, want = run_allocating(lib, n, gens, inv, rad)
        assert rc_a == rc_b and rc_a >= 0
        assert got == want


def test_noalloc_rejects_problems_beyond_its_fixed_size(lib):
    rc, _ = run_noalloc(lib, 10, w.lrx(10), True)          # 3,628,800 states > 2^20
    assert rc == lib.CG_ETOOBIG
    rc, _ = run_noalloc(lib, 8, [w.coxeter(8)[0]] * 300, True)  # more rows than it holds
    assert rc == lib.CG_ETOOBIG
    # and the next call still works
    rc, got = run_noalloc(lib, 8, w.coxeter(8), True)
    assert rc == 0 and got == run_allocating(lib, 8, w.coxeter(8), True)[1]
