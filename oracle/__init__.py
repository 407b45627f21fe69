"""ORACLE (test infrastructure only): plain CPU growth of permutation Cayley graphs.

The computation lives in ``growth_ref.cpp`` (sequential breadth-first search over byte-array
permutations with a ``std::unordered_set`` visited set, Section 2.1 Def. "Growth" and the
BFS of Sections 3.1.2-3.1.3).  This module compiles it with the host C++ compiler and calls
it through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline / reference arm
may import this package.  The CUDA library never imports it, and it imports nothing from
the library.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "growth_ref.cpp")
_SRC_B = os.path.join(_HERE, "growth_bitmap_ref.cpp")
_LIB = os.path.join(_HERE, "libgrowth_ref.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libgrowth_ref.so (plain g++, -O2)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_B))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", tmp,
                               _SRC, _SRC_B])
        os.replace(tmp, _LIB)
    return _LIB


_PROGRESS = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.c_uint64)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.oracle_growth.argtypes = [ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_uint64, u64p, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]
            lib.oracle_growth.restype = ctypes.c_int
            lib.oracle_growth_from.argtypes = [ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_uint64, u64p, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)]
            lib.oracle_growth_from.restype = ctypes.c_int
            lib.oracle_layer_keys.argtypes = [ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int,
                                              u64p, ctypes.c_uint64, u64p]
            lib.oracle_layer_keys.restype = ctypes.c_int
            lib.oracle_distance.argtypes = [ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_int]
            lib.oracle_distance.restype = ctypes.c_int
            lib.oracle_growth_bitmap.argtypes = [ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int,
                                                 ctypes.c_uint64, ctypes.c_int, u64p, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int)]
            lib.oracle_growth_bitmap.restype = ctypes.c_int
            lib.oracle_growth_bitmask.argtypes = [ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int,
                                                  ctypes.c_uint64, ctypes.c_int, u64p, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_int), _PROGRESS]
            lib.oracle_growth_bitmask.restype = ctypes.c_int
            _lib = lib
    return _lib


def _gens_array(n: int, gens: Sequence[Sequence[int]]) -> np.ndarray:
    arr = np.ascontiguousarray(np.asarray(gens, dtype=np.uint8).reshape(len(gens), n))
    return arr


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def growth(n: int, gens: Sequence[Sequence[int]], two_layer: bool = False,
           max_radius: int = -1, stop_above: int = 0, start=None) -> Tuple[List[int], int]:
    """Growth vector gamma(0..R) and the return code (0 ended, 1 stopped by a limit), from the
    identity (n <= 32) or from the vector `start` (n <= 64 values in 0..15, repeats allowed)."""
    lib = _load()
    g = _gens_array(n, gens)
    cap = 4096
    out = np.zeros(cap, dtype=np.uint64)
    nl = ctypes.c_int(0)
    st = None
    if start is not None:
        st = np.ascontiguousarray(np.asarray(start, dtype=np.uint8))
    rc = lib.oracle_growth_from(n, len(gens), _ptr(g, ctypes.c_uint8),
                                _ptr(st, ctypes.c_uint8) if st is not None else None,
                                int(two_layer), int(max_radius), int(stop_above),
                                _ptr(out, ctypes.c_uint64), cap, ctypes.byref(nl))
    if rc < 0:
        raise ValueError(f"oracle_growth failed rc={rc}")
    return [int(x) for x in out[:nl.value]], rc


def growth_bitmap(n: int, gens: Sequence[Sequence[int]], max_radius: int = -1,
                  stop_above: int = 0, threads: int = 0) -> Tuple[List[int], int]:
    """Oracle B: the same growth with a visited bitmap over all n! permutations (n <= 14),
    expanded by `threads` host threads (0: all)."""
    lib = _load()
    g = _gens_array(n, gens)
    cap = 4096
    out = np.zeros(cap, dtype=np.uint64)
    nl = ctypes.c_int(0)
    rc = lib.oracle_growth_bitmap(n, len(gens), _ptr(g, ctypes.c_uint8), int(max_radius),
                                  int(stop_above), int(threads), _ptr(out, ctypes.c_uint64), cap,
                                  ctypes.byref(nl))
    if rc < 0:
        raise ValueError(f"oracle_growth_bitmap failed rc={rc}")
    return [int(x) for x in out[:nl.value]], rc


def growth_bitmask(n: int, gens: Sequence[Sequence[int]], max_radius: int = -1,
                   stop_above: int = 0, threads: int = 0, progress=None) -> Tuple[List[int], int]:
    """Oracle C: the same growth with the visited set and the current and next layers as bitmaps
    over all n! permutations (n <= 14; 3 n!/8 bytes of host memory).  progress(radius, size) is
    called after each layer when given."""
    lib = _load()
    g = _gens_array(n, gens)
    cap = 4096
    out = np.zeros(cap, dtype=np.uint64)
    nl = ctypes.c_int(0)
    cb = _PROGRESS(progress) if progress else _PROGRESS()
    rc = lib.oracle_growth_bitmask(n, len(gens), _ptr(g, ctypes.c_uint8), int(max_radius),
                                   int(stop_above), int(threads), _ptr(out, ctypes.c_uint64), cap,
                                   ctypes.byref(nl), cb)
    if rc < 0:
        raise ValueError(f"oracle_growth_bitmask failed rc={rc}")
    return [int(x) for x in out[:nl.value]], rc


def layer_keys(n: int, gens: Sequence[Sequence[int]], radius: int) -> np.ndarray:
    """Packed keys of layer ``radius`` (element i in bits [4i, 4i+4)), sorted ascending."""
    lib = _load()
    g = _gens_array(n, gens)
    cnt = ctypes.c_uint64(0)
    dummy = np.zeros(1, dtype=np.uint64)
    rc = lib.oracle_layer_keys(n, len(gens), _ptr(g, ctypes.c_uint8), radius,
                               _ptr(dummy, ctypes.c_uint64), 0, ctypes.byref(cnt))
    if rc == -3:
        return np.zeros(0, dtype=np.uint64)
    out = np.zeros(max(1, cnt.value), dtype=np.uint64)
    rc = lib.oracle_layer_keys(n, len(gens), _ptr(g, ctypes.c_uint8), radius,
                               _ptr(out, ctypes.c_uint64), cnt.value, ctypes.byref(cnt))
    if rc != 0:
        raise ValueError(f"oracle_layer_keys failed rc={rc}")
    return out[:cnt.value]


def distance(n: int, gens: Sequence[Sequence[int]], target: Sequence[int],
             max_radius: int = -1) -> int:
    """Word-metric distance of ``target`` from the identity (-1: not reached)."""
    lib = _load()
    g = _gens_array(n, gens)
    t = np.ascontiguousarray(np.asarray(target, dtype=np.uint8))
    rc = lib.oracle_distance(n, len(gens), _ptr(g, ctypes.c_uint8), _ptr(t, ctypes.c_uint8),
                             int(max_radius))
    if rc == -2:
        raise ValueError("oracle_distance: invalid input")
    return rc
