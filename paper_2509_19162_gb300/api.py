"""Python front end of the growth library (marshalling over the C ABI in _cg.py).

    >>> from paper_2509_19162_gb300 import growth
    >>> r = growth(8, coxeter_generators)          # runs on the current CUDA device
    >>> r.layers[:4], r.diameter

The computation is the growth of a permutation Cayley graph from the identity (Section 2.1,
Def. "Growth"), run entirely by the library's CUDA kernels.  PyTorch is optional: a
``torch.cuda.Stream`` may be passed as ``stream`` and ``use_torch_allocator()`` routes the
library's device allocations through PyTorch's caching allocator.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import _cg

STRATEGIES = {"auto": _cg.CG_STRATEGY_AUTO, "hash": _cg.CG_STRATEGY_HASH, "sort": _cg.CG_STRATEGY_SORT,
              "bitmap": _cg.CG_STRATEGY_BITMAP, "sweep": _cg.CG_STRATEGY_SWEEP}
SWEEP_ORDERS = {"auto": 0, "discovery": 1, "rank": 2}


@dataclass
class GrowthResult:
    layers: List[int]
    status: int

    @property
    def diameter(self) -> int:
        return len(self.layers) - 1

    @property
    def complete(self) -> bool:
        return self.status == _cg.CG_OK

    @property
    def total(self) -> int:
        return int(sum(self.layers))

    def statistics(self) -> dict:
        """Moments of the distance distribution P(d = r) = |S_r| / sum |S_r| (the growth
        columns of the paper's Section 3.3 table): mean, mode, variance, skewness and excess
        kurtosis.  Computed on the host from the exact layer sizes, with exact integer sums."""
        from fractions import Fraction
        N = sum(self.layers)
        if N == 0:
            return {}
        m1 = Fraction(sum(r * c for r, c in enumerate(self.layers)), N)
        var = Fraction(sum((r - m1) ** 2 * c for r, c in enumerate(self.layers)), N)
        m3 = Fraction(sum((r - m1) ** 3 * c for r, c in enumerate(self.layers)), N)
        m4 = Fraction(sum((r - m1) ** 4 * c for r, c in enumerate(self.layers)), N)
        mode = max(range(len(self.layers)), key=lambda r: (self.layers[r], -r))
        out = {"mean": float(m1), "mode": mode, "variance": float(var),
               "skewness": 0.0, "kurtosis": 0.0, "diameter": self.diameter}
        if var > 0:
            out["skewness"] = float(m3) / float(var) ** 1.5
            out["kurtosis"] = float(m4 / (var * var)) - 3.0
        return out


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    h = getattr(stream, "cuda_stream", None)
    if h is not None:
        return int(h)
    raise TypeError("stream must be None, an int handle or a torch.cuda.Stream")


def _gens_bytes(n: int, gens: Sequence[Sequence[int]]) -> np.ndarray:
    arr = np.asarray(gens, dtype=np.int64)
    if arr.ndim != 2 or arr.shape[1] != n:
        raise ValueError(f"gens must be k x {n}")
    if arr.min(initial=0) < 0 or arr.max(initial=0) > 255:
        raise ValueError("generator entries out of range")
    return np.ascontiguousarray(arr.astype(np.uint8))


def _is_inverse_closed(gens: Sequence[Sequence[int]]) -> bool:
    s = {tuple(int(x) for x in g) for g in gens}
    for g in s:
        inv = [0] * len(g)
        for i, v in enumerate(g):
            inv[v] = i
        if tuple(inv) not in s:
            return False
    return True


class Growth:
    """One growth job (cg_growth_create ... cg_growth_destroy)."""

    def __init__(self, n: int, gens: Sequence[Sequence[int]], inverse_closed: Optional[bool] = None,
                 max_radius: int = -1, mem_cap: int = 0, strategy: str = "auto",
                 stop_above: int = 0, keep_last: bool = False, start: Optional[Sequence[int]] = None):
        """n, gens: one-line permutations of 0..n-1 (t[i] = s[g[i]]).  inverse_closed: None
        detects it.  max_radius < 0: no limit.  mem_cap: bytes every device buffer of the job
        fits in (0: the library default); an undirected growth whose stored states outgrow it
        goes on with the sorted two-layer step.  strategy: one of STRATEGIES.  stop_above > 0:
        stop after the first layer with more states.  keep_last: keep the last layer for
        last_layer().  start: a central state (n values in 0..15, repeats allowed) to grow the
        orbit of, i.e. a Schreier coset graph; None grows the Cayley graph from the identity."""
        g = _gens_bytes(n, gens)
        if inverse_closed is None:
            inverse_closed = _is_inverse_closed(gens)
        self._gens = g
        h = ctypes.c_void_p()
        _cg.check(_cg.cg_growth_create(int(n), int(g.shape[0]),
                                       g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                       int(bool(inverse_closed)), int(max_radius), int(mem_cap),
                                       ctypes.byref(h)), "cg_growth_create")
        self._h = h
        self.n = n
        self.k = g.shape[0]
        if strategy not in STRATEGIES:
            raise ValueError(f"strategy must be one of {sorted(STRATEGIES)}")
        _cg.check(_cg.cg_growth_set_option(h, _cg.CG_OPT_STRATEGY, STRATEGIES[strategy]),
                  "cg_growth_set_option(strategy)")
        if stop_above:
            _cg.check(_cg.cg_growth_set_option(h, _cg.CG_OPT_STOP_ABOVE, int(stop_above)),
                      "cg_growth_set_option(stop_above)")
        if keep_last:
            _cg.check(_cg.cg_growth_set_option(h, _cg.CG_OPT_KEEP_LAST, 1),
                      "cg_growth_set_option(keep_last)")
        if start is not None:
            self.set_start(start)
        self._cap = 1024
        self._out = np.zeros(self._cap, dtype=np.uint64)

    @property
    def order(self) -> int:
        return int(_cg.cg_growth_group_order(self._h))

    def run(self, stream=None) -> GrowthResult:
        nl = ctypes.c_int(0)
        while True:
            rc = _cg.cg_growth_run(self._h, _stream_handle(stream),
                                   self._out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                   self._cap, ctypes.byref(nl))
            if rc == _cg.CG_EINVAL and nl.value > self._cap:
                self._cap = nl.value
                self._out = np.zeros(self._cap, dtype=np.uint64)
                continue
            break
        _cg.check(rc, "cg_growth_run")
        return GrowthResult([int(x) for x in self._out[:nl.value]], rc)

    def set_start(self, start: Optional[Sequence[int]]) -> None:
        """Grow from the central state `start` (n values in 0..15, repeats allowed: a Schreier
        coset graph), or from the identity when None."""
        if start is None:
            _cg.check(_cg.cg_growth_set_start(self._h, None), "cg_growth_set_start")
            return
        st = np.ascontiguousarray(np.asarray(start, dtype=np.int64))
        if st.shape != (self.n,) or st.min(initial=0) < 0 or st.max(initial=0) > 15:
            raise ValueError("start must hold n values in 0..15")
        st8 = st.astype(np.uint8)
        _cg.check(_cg.cg_growth_set_start(self._h, st8.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
                  "cg_growth_set_start")

    def set_grid(self, blocks: int) -> None:
        """Blocks of the persistent launch (0 = library default)."""
        _cg.check(_cg.cg_growth_set_option(self._h, _cg.CG_OPT_GRID, int(blocks)), "set_grid")

    def set_ilp(self, ilp: int) -> None:
        """Generators probed together per thread (1..4; 0 = library default)."""
        _cg.check(_cg.cg_growth_set_option(self._h, _cg.CG_OPT_ILP, int(ilp)), "set_ilp")

    def set_sweep_order(self, order: str) -> None:
        """Sweep strategy: the order in which a round takes a layer's nonempty blocks.

        "auto" (rank order for dense layers, else order of discovery), "discovery" or "rank".
        The layers are the same in every order."""
        if order not in SWEEP_ORDERS:
            raise ValueError(f"sweep order must be one of {sorted(SWEEP_ORDERS)}")
        _cg.check(_cg.cg_growth_set_option(self._h, _cg.CG_OPT_SWEEP_ORDER, SWEEP_ORDERS[order]),
                  "set_sweep_order")

    def stats(self) -> dict:
        st = _cg.cg_growth_stats()
        _cg.check(_cg.cg_growth_get_stats(self._h, ctypes.byref(st)), "cg_growth_get_stats")
        return {f: getattr(st, f) for f, _ in st._fields_}

    def last_layer(self) -> np.ndarray:
        """Packed keys of the last layer: shape (count,) uint64, or (count, 2) (low, high word)
        for keys of more than 64 bits (key_words == 2)."""
        cnt = ctypes.c_uint64(0)
        _cg.cg_growth_last_layer(self._h, None, 0, ctypes.byref(cnt))
        words = self.key_words
        out = np.zeros(max(1, cnt.value) * words, dtype=np.uint64)
        _cg.check(_cg.cg_growth_last_layer(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                           cnt.value, ctypes.byref(cnt)), "cg_growth_last_layer")
        if words == 2:
            return out[:2 * cnt.value].reshape(cnt.value, 2)
        return out[:cnt.value]

    @property
    def key_words(self) -> int:
        """64-bit words per packed key (2 for vectors of more than 64 bits)."""
        return int(_cg.cg_growth_key_words(self._h))

    @property
    def key_width(self) -> int:
        """Bits per element of the packed keys (4 for permutations; 1 or 2 for narrow vectors)."""
        return int(_cg.cg_growth_key_width(self._h))

    def last_layer_vectors(self) -> np.ndarray:
        """The last layer as an array of shape (count, n): the unpacked states."""
        keys = self.last_layer()
        w = self.key_width
        if keys.ndim == 2:                     # two words: element i at bits [w i, w i + w)
            out = np.zeros((keys.shape[0], self.n), dtype=np.uint8)
            for i in range(self.n):
                b = w * i
                v = np.zeros(keys.shape[0], dtype=np.uint64)
                for q in range(w):
                    bit = b + q
                    word = keys[:, bit // 64]
                    v |= ((word >> np.uint64(bit % 64)) & np.uint64(1)) << np.uint64(q)
                out[:, i] = v.astype(np.uint8)
            return out
        shifts = (w * np.arange(self.n, dtype=np.uint64)).astype(np.uint64)
        return ((keys[:, None] >> shifts[None, :]) & np.uint64((1 << w) - 1)).astype(np.uint8)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _cg.cg_growth_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def growth(n: int, gens: Sequence[Sequence[int]], inverse_closed: Optional[bool] = None,
           max_radius: int = -1, mem_cap: int = 0, strategy: str = "auto", stop_above: int = 0,
           stream=None, start: Optional[Sequence[int]] = None) -> GrowthResult:
    """Growth vector |S_0|, |S_1|, ... of the Cayley graph of <gens> from the identity, or of
    the Schreier coset graph of the orbit of `start`."""
    with Growth(n, gens, inverse_closed, max_radius, mem_cap, strategy, stop_above, start=start) as g:
        return g.run(stream)


class Batch:
    """Many independent growth jobs run together (cg_batch_create ... cg_batch_destroy)."""

    VISITED = {"auto": _cg.CG_STRATEGY_AUTO, "hash": _cg.CG_STRATEGY_HASH, "bitmap": _cg.CG_STRATEGY_BITMAP}

    def __init__(self, jobs, mem_cap: int = 0, wave_l2: Optional[int] = None, ilp: int = 0,
                 grid: int = 0, visited: str = "auto", graph: bool = True, max_active: int = 0,
                 unit: int = 4):
        """jobs: sequence of (n, gens, inverse_closed, max_radius).
        wave_l2: cap on the summed visited-set bytes of the jobs grown at once (None or 0: half
        of L2; -1: no cap).  ilp, grid: kernel variant and blocks of the launch (0: library
        choice).  visited: "auto", "hash" or "bitmap".  graph: capture a whole run as a CUDA
        graph (default).  max_active: most jobs grown at once (0: library choice).  unit:
        frontier states per warp work unit, in multiples of 32 (1, 2, 4 or 8; default 4)."""
        self.njobs = len(jobs)
        ns = np.array([j[0] for j in jobs], dtype=np.int32)
        ks = np.array([len(j[1]) for j in jobs], dtype=np.int32)
        blobs = [_gens_bytes(j[0], j[1]).ravel() for j in jobs]
        offs = np.zeros(self.njobs, dtype=np.uint64)
        if self.njobs:
            offs[1:] = np.cumsum([b.size for b in blobs])[:-1]
        flat = np.ascontiguousarray(np.concatenate(blobs) if blobs else np.zeros(1, np.uint8))
        inv = np.array([int(bool(j[2])) for j in jobs], dtype=np.int32)
        rad = np.array([int(j[3]) for j in jobs], dtype=np.int32)
        self._keep = (ns, ks, flat, offs, inv, rad)
        h = ctypes.c_void_p()
        ip = ctypes.POINTER(ctypes.c_int)
        _cg.check(_cg.cg_batch_create(self.njobs, ns.ctypes.data_as(ip), ks.ctypes.data_as(ip),
                                      flat.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                      offs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                      inv.ctypes.data_as(ip), rad.ctypes.data_as(ip), int(mem_cap),
                                      ctypes.byref(h)), "cg_batch_create")
        self._h = h
        self._out = None
        self.set_options(wave_l2=wave_l2 or 0, ilp=ilp, grid=grid, visited=visited, graph=graph,
                         max_active=max_active, unit=unit)

    def set_options(self, wave_l2: Optional[int] = None, ilp: Optional[int] = None,
                    grid: Optional[int] = None, visited: Optional[str] = None,
                    graph: Optional[bool] = None, max_active: Optional[int] = None,
                    unit: Optional[int] = None) -> None:
        """Change launch settings (None: unchanged); see __init__."""
        opts = []
        if max_active is not None:
            opts.append((_cg.CG_OPT_BATCH_ACTIVE, int(max_active)))
        if unit is not None:
            opts.append((_cg.CG_OPT_UNIT, int(unit)))
        if wave_l2 is not None:
            opts.append((_cg.CG_OPT_BATCH_WAVE_L2, int(wave_l2)))
        if ilp is not None:
            opts.append((_cg.CG_OPT_ILP, int(ilp)))
        if grid is not None:
            opts.append((_cg.CG_OPT_GRID, int(grid)))
        if visited is not None:
            if visited not in self.VISITED:
                raise ValueError(f"visited must be one of {sorted(self.VISITED)}")
            opts.append((_cg.CG_OPT_BATCH_VISITED, self.VISITED[visited]))
        if graph is not None:
            opts.append((_cg.CG_OPT_GRAPH, int(bool(graph))))
        for o, v in opts:
            _cg.check(_cg.cg_batch_set_option(self._h, o, v), "cg_batch_set_option")

    def set_wave_l2(self, nbytes: int) -> None:
        """Cap on the summed visited-set bytes of the jobs grown in one launch (0: half of L2,
        -1: no cap)."""
        self.set_options(wave_l2=nbytes)

    def stats(self) -> dict:
        st = _cg.cg_growth_stats()
        _cg.check(_cg.cg_batch_get_stats(self._h, ctypes.byref(st)), "cg_batch_get_stats")
        return {f: getattr(st, f) for f, _ in st._fields_}

    def run(self, stream=None, cap: int = 512) -> List[GrowthResult]:
        if self._out is None or self._out[0].shape[1] != cap:
            self._out = (np.zeros((self.njobs, cap), dtype=np.uint64), np.zeros(self.njobs, dtype=np.int32),
                         np.zeros(self.njobs, dtype=np.int32))
        out, nl, stv = self._out
        ip = ctypes.POINTER(ctypes.c_int)
        rc = _cg.cg_batch_run(self._h, _stream_handle(stream),
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap,
                              nl.ctypes.data_as(ip), stv.ctypes.data_as(ip))
        _cg.check(rc, "cg_batch_run")
        nls = nl.tolist()
        sts = stv.tolist()
        return [GrowthResult(out[j, :nls[j]].tolist(), sts[j]) for j in range(self.njobs)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _cg.cg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shard(items, rank: int, world: int):
    """The share of `items` that rank `rank` of `world` runs (round-robin): independent growth
    jobs shard across GPUs with no exchange step."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    return items[rank::world]


def unshard(parts, total: int):
    """Inverse of shard: parts[r] is rank r's results in its own order; returns them in the
    original item order."""
    world = len(parts)
    out = [None] * total
    for r, part in enumerate(parts):
        for i, x in enumerate(part):
            out[r + i * world] = x
    return out


_torch_alloc_refs = None


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _torch_alloc_refs
    if not enable:
        _cg.check(_cg.cg_set_allocator(_cg.ALLOC_FN(), _cg.FREE_FN(), None), "cg_set_allocator")
        _torch_alloc_refs = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _cg.ALLOC_FN(_alloc), _cg.FREE_FN(_free)
    _torch_alloc_refs = (a, f)
    _cg.check(_cg.cg_set_allocator(a, f, None), "cg_set_allocator")
