"""CPU checks of the C ABI: the library builds, loads, exports every symbol include/*.h declares,
and its host-side logic (validation, inverse-closure check, group order) is right.  No call
here touches a GPU."""

import ctypes
import glob
import math
import os
import re

import numpy as np
import pytest

import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_19162_gb300 import build
    build()
    from paper_2509_19162_gb300 import _cg
    return _cg


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cg_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "cg_growth_create" in names and "cg_growth_run" in names
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in sorted(names):
        assert hasattr(so, name), f"{name} declared in include/ but not exported"
    # and the binding wraps every one of them under the same name
    for name in names:
        assert hasattr(lib, name), f"binding lacks {name}"


def test_header_constants_match_the_binding(lib):
    # every #define CG_* value of the header, under the same name in the binding
    found = 0
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        for m in re.finditer(r"^#define\s+(CG_[A-Z0-9_]+)\s+(-?\d+\b|\(1u << \d+\))", open(h).read(),
                             flags=re.M):
            name, text = m.group(1), m.group(2)
            value = 1 << int(text[7:-1]) if text.startswith("(1u") else int(text)
            assert getattr(lib, name, None) == value, f"{name} = {value} in the header"
            found += 1
    assert found >= 20


def test_prototype_arity_matches_the_binding(lib):
    # each entry point's argument count, as declared, against the ctypes argtypes
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "cg_growth.h")).read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(?:int|const char\*|uint64_t|size_t|void)\s+\**(cg_[a-z0-9_]+)\s*\(([^)]*)\)\s*;",
                         text):
        args = m.group(2).strip()
        protos[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    assert len(protos) >= 30
    for name, nargs in protos.items():
        assert name in lib.SIGNATURES, name
        assert len(lib.SIGNATURES[name][1]) == nargs, name


def test_stats_struct_matches_the_binding(lib):
    # field order and types of cg_growth_stats, as declared, against the ctypes mirror
    text = open(os.path.join(ROOT, "include", "cg_growth.h")).read()
    body = re.search(r"typedef struct cg_growth_stats \{(.*?)\} cg_growth_stats;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    ctype = {"double": ctypes.c_double, "int": ctypes.c_int, "uint64_t": ctypes.c_uint64}
    declared = [(m.group(2), ctype[m.group(1)])
                for m in re.finditer(r"\b(double|int|uint64_t)\s+(\w+)\s*;", body)]
    assert declared == list(lib.cg_growth_stats._fields_)


def test_strerror_names_every_code(lib):
    for code in (0, 1, 2, 3, -1, -2, -3, -4, -5, -6, -7):
        assert lib.strerror(code) != "unknown code"


def _create(lib, n, gens, inv=0, maxr=-1):
    g = np.ascontiguousarray(np.asarray(gens, dtype=np.uint8))
    h = ctypes.c_void_p()
    rc = lib.cg_growth_create(n, len(gens), g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              inv, maxr, 0, ctypes.byref(h))
    return rc, h


def test_create_validation(lib):
    assert _create(lib, 3, [[0, 0, 1]])[0] == lib.CG_EINVAL          # not a permutation
    assert _create(lib, 129, [list(range(129))])[0] == lib.CG_EINVAL   # n > 128
    assert _create(lib, 0, [[]])[0] == lib.CG_EINVAL
    assert _create(lib, 5, w.lx(5), inv=1)[0] == lib.CG_ENOTCLOSED
    rc, h = _create(lib, 5, w.lrx(5), inv=1)
    assert rc == 0 and h.value
    assert lib.cg_growth_set_option(h, 99, 0) == lib.CG_EINVAL
    assert lib.cg_growth_set_option(h, lib.CG_OPT_STRATEGY, 7) == lib.CG_EINVAL
    assert lib.cg_growth_set_option(h, lib.CG_OPT_SWEEP_ORDER, 3) == lib.CG_EINVAL
    assert lib.cg_growth_set_option(h, lib.CG_OPT_SWEEP_ORDER, -1) == lib.CG_EINVAL
    for order in (0, 1, 2):
        assert lib.cg_growth_set_option(h, lib.CG_OPT_SWEEP_ORDER, order) == 0
    assert lib.cg_growth_destroy(h) == 0
    assert lib.cg_growth_destroy(None) == 0
    # sort strategy needs an inverse-closed set
    rc, h = _create(lib, 5, w.lx(5), inv=0)
    assert lib.cg_growth_set_option(h, lib.CG_OPT_STRATEGY, lib.CG_STRATEGY_SORT) == lib.CG_EINVAL
    lib.cg_growth_destroy(h)


def test_set_start_validation(lib):
    rc, h = _create(lib, 5, w.lrx(5), inv=1)
    u8 = ctypes.POINTER(ctypes.c_uint8)
    bad = np.array([0, 1, 2, 3, 16], dtype=np.uint8)
    ok = np.array([0, 0, 1, 1, 1], dtype=np.uint8)
    assert lib.cg_growth_set_start(None, ok.ctypes.data_as(u8)) == lib.CG_EINVAL
    assert lib.cg_growth_set_start(h, bad.ctypes.data_as(u8)) == lib.CG_EINVAL
    assert lib.cg_growth_set_start(h, ok.ctypes.data_as(u8)) == 0
    assert lib.cg_growth_set_start(h, None) == 0
    lib.cg_growth_destroy(h)
    # n > 16: from the identity only up to n = 25 (5-bit elements in two words); longer vectors
    # from a start vector whose values fit n * width <= 128 bits
    rc, h = _create(lib, 40, [list(range(1, 40)) + [0]], inv=0)
    assert rc == 0
    out = np.zeros(8, dtype=np.uint64)
    nl = ctypes.c_int(0)
    assert lib.cg_growth_run(h, None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), 8,
                             ctypes.byref(nl)) == lib.CG_EINVAL          # identity of S_40
    four_bit = np.array([5] + [0] * 39, dtype=np.uint8)                    # 160 bits: too wide
    two_bit = np.array([3] + [0] * 39, dtype=np.uint8)                     # 80 bits: two words
    one_bit = np.array([1] * 20 + [0] * 20, dtype=np.uint8)                # 40 bits: one word
    assert lib.cg_growth_set_start(h, four_bit.ctypes.data_as(u8)) == lib.CG_EINVAL
    assert lib.cg_growth_set_start(h, two_bit.ctypes.data_as(u8)) == 0
    assert lib.cg_growth_key_words(h) == 2 and lib.cg_growth_key_width(h) == 2
    assert lib.cg_growth_set_start(h, one_bit.ctypes.data_as(u8)) == 0
    assert lib.cg_growth_key_words(h) == 1 and lib.cg_growth_key_width(h) == 1
    lib.cg_growth_destroy(h)
    # the identity of S_20: 5-bit elements, two words
    rc, h = _create(lib, 20, w.coxeter(20), inv=1)
    assert rc == 0 and lib.cg_growth_key_words(h) == 2 and lib.cg_growth_key_width(h) == 5
    lib.cg_growth_destroy(h)


def test_group_order_closed_forms(lib):
    from paper_2509_19162_gb300 import Growth
    for n in range(2, 17):
        assert Growth(n, w.coxeter(n)).order == math.factorial(n)
        if n >= 3:
            assert Growth(n, w.three_cycles(n) if n <= 9 else w.consecutive_3cycles_inv(n)).order \
                == math.factorial(n) // 2
    assert Growth(16, w.all_transpositions(16)).order == math.factorial(16)
    # identity / duplicate rows are ignored
    g = w.coxeter(6)
    assert Growth(6, g + g + [list(range(6))]).order == 720
    assert Growth(4, [[0, 1, 2, 3]]).order == 1


def test_group_order_matches_sympy(lib):
    sc = pytest.importorskip("sympy.combinatorics")
    from paper_2509_19162_gb300 import Growth
    rng = np.random.default_rng(99)
    for _ in range(60):
        n = int(rng.integers(2, 17))
        gens = w.random_perms(rng, n, int(rng.integers(1, 4)))
        if rng.integers(0, 2):
            # a subgroup: generators that fix the last points or move blocks
            m = int(rng.integers(1, n + 1))
            gens = [g[:m] + list(range(m, n)) if sorted(g[:m]) == list(range(m)) else g for g in gens]
        want = sc.PermutationGroup([sc.Permutation(g) for g in gens]).order()
        assert Growth(n, gens).order == want


def test_batch_create_validation(lib):
    from paper_2509_19162_gb300 import Batch
    jobs = [(n, w.coxeter(n), True, -1) for n in (3, 4, 5)]
    b = Batch(jobs)
    b.close()
    with pytest.raises(RuntimeError):
        Batch([(5, w.lx(5), True, -1)])


def test_server_host_logic(lib):
    from paper_2509_19162_gb300.serve import Server
    with Server(mem_budget=1 << 30, max_slots=4) as s:
        with pytest.raises(RuntimeError):
            s.submit(5, [[0, 0, 1, 2, 3]])                      # not a permutation
        with pytest.raises(RuntimeError):
            s.submit(5, w.lx(5), inverse_closed=True)          # not inverse-closed
        a = s.submit(4, [[0, 1, 2, 3]])                        # identity only: ends at once
        b = s.submit(6, w.coxeter(6), max_radius=0)            # radius 0: ends at once
        c = s.submit(6, w.coxeter(6))                          # queued
        assert s.load()[0] == 1
        assert sorted(s.finished()) == sorted([a, b])
        r = s.result(a)
        assert r.layers == [1] and r.status == 0
        assert s.result(b).status == 1
        with pytest.raises(RuntimeError):
            s.result(c)                                        # not run yet
