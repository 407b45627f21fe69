"""Serving loop over the library's continuous-batching server (cg_server_* in the C ABI).

``Server`` wraps one native server: jobs are submitted to a host queue, admitted into device
slots by predicted memory, and advanced a few layer steps at a time, all admitted jobs together
in one persistent launch per step.  ``serve_stream`` drives it with a stream of jobs arriving at
given times (a Poisson process in the serving workload) and reports each job's latency from its
arrival to the end of the step in which it finished.
"""

from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import _cg
from .api import GrowthResult, _gens_bytes, _is_inverse_closed, _stream_handle


class Server:
    def __init__(self, mem_budget: int = 0, max_slots: int = 256, job_mem_cap: int = 0,
                 rounds_per_step: int = 8):
        h = ctypes.c_void_p()
        _cg.check(_cg.cg_server_create(int(mem_budget), int(max_slots), int(job_mem_cap),
                                       int(rounds_per_step), ctypes.byref(h)), "cg_server_create")
        self._h = h

    def submit(self, n: int, gens: Sequence[Sequence[int]], inverse_closed: Optional[bool] = None,
               max_radius: int = -1) -> int:
        g = _gens_bytes(n, gens)
        if inverse_closed is None:
            inverse_closed = _is_inverse_closed(gens)
        jid = ctypes.c_uint64(0)
        _cg.check(_cg.cg_server_submit(self._h, int(n), int(g.shape[0]),
                                       g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                       int(bool(inverse_closed)), int(max_radius), ctypes.byref(jid)),
                  "cg_server_submit")
        return int(jid.value)

    @staticmethod
    def predict(n: int, gens: Sequence[Sequence[int]], inverse_closed: Optional[bool] = None,
                max_radius: int = -1, job_mem_cap: int = 160 << 24) -> Dict[str, int]:
        """Admission plan of a job under the per-job share job_mem_cap (bytes; the server's default
        share is its budget / 64): predicted states up to the radius cap, states granted, the
        device bytes it is admitted with, its visited set ("hash" or "bitmap"), and whether the
        server grows it alone (predicted to fill the GPU: CG_SERVER_SOLO_STATES states or more).
        Host only."""
        g = _gens_bytes(n, gens)
        if inverse_closed is None:
            inverse_closed = _is_inverse_closed(gens)
        st, gr, by = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
        vis = ctypes.c_int(0)
        _cg.check(_cg.cg_server_predict(int(n), int(g.shape[0]), g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                        int(bool(inverse_closed)), int(max_radius), int(job_mem_cap),
                                        ctypes.byref(st), ctypes.byref(gr), ctypes.byref(by), ctypes.byref(vis)),
                  "cg_server_predict")
        return {"states": int(st.value), "granted": int(gr.value), "bytes": int(by.value),
                "visited": "bitmap" if vis.value == _cg.CG_STRATEGY_BITMAP else "hash",
                "alone": int(st.value) >= _cg.CG_SERVER_SOLO_STATES}

    def step(self, stream=None):
        a = ctypes.c_int(0)
        f = ctypes.c_int(0)
        _cg.check(_cg.cg_server_step(self._h, _stream_handle(stream), ctypes.byref(a), ctypes.byref(f)),
                  "cg_server_step")
        return a.value, f.value

    def finished(self) -> List[int]:
        out = np.zeros(4096, dtype=np.uint64)
        ids: List[int] = []
        while True:
            c = ctypes.c_int(0)
            _cg.check(_cg.cg_server_finished(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                             len(out), ctypes.byref(c)), "cg_server_finished")
            ids.extend(int(x) for x in out[:c.value])
            if c.value < len(out):
                return ids

    def result(self, job_id: int) -> GrowthResult:
        cap = 4096
        out = np.zeros(cap, dtype=np.uint64)
        nl = ctypes.c_int(0)
        st = ctypes.c_int(0)
        _cg.check(_cg.cg_server_result(self._h, int(job_id), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                       cap, ctypes.byref(nl), ctypes.byref(st)), "cg_server_result")
        return GrowthResult([int(x) for x in out[:nl.value]], int(st.value))

    def load(self):
        q = ctypes.c_int(0)
        a = ctypes.c_int(0)
        u = ctypes.c_uint64(0)
        _cg.check(_cg.cg_server_load(self._h, ctypes.byref(q), ctypes.byref(a), ctypes.byref(u)),
                  "cg_server_load")
        return q.value, a.value, u.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _cg.cg_server_destroy(self._h)
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


@dataclass
class StreamReport:
    results: List[GrowthResult]
    latency_s: List[float]
    arrival_s: List[float]
    makespan_s: float
    steps: int
    max_active: int
    mean_active: float
    extra: Dict = field(default_factory=dict)

    @property
    def jobs_per_s(self) -> float:
        return len(self.results) / self.makespan_s if self.makespan_s > 0 else float("inf")

    def percentile_ms(self, q: float) -> float:
        return float(np.percentile(np.asarray(self.latency_s) * 1000.0, q))


def serve_stream(jobs, arrivals_s: Sequence[float], server: Server, stream=None,
                 realtime: bool = True) -> StreamReport:
    """Submit jobs[i] at arrivals_s[i] seconds after the start (sorted ascending) and step the
    server until every job has ended.  jobs: objects with n, gens, inverse_closed, max_radius.
    With realtime=False every job arrives at time 0 (a closed batch)."""
    N = len(jobs)
    arr = list(arrivals_s) if realtime else [0.0] * N
    id_of: Dict[int, int] = {}
    done: Dict[int, GrowthResult] = {}
    lat = [0.0] * N
    t0 = time.perf_counter()
    i = 0
    steps = 0
    max_active = 0
    active_sum = 0
    while len(done) < N:
        now = time.perf_counter() - t0
        while i < N and arr[i] <= now:
            j = jobs[i]
            jid = server.submit(j.n, j.gens, j.inverse_closed, j.max_radius)
            id_of[jid] = i
            i += 1
        active, _ = server.step(stream)
        steps += 1
        max_active = max(max_active, active)
        active_sum += active
        t_end = time.perf_counter() - t0
        for jid in server.finished():
            idx = id_of[jid]
            done[idx] = server.result(jid)
            lat[idx] = t_end - arr[idx]
        queued, act, _ = server.load()
        if act == 0 and queued == 0 and i < N and len(done) < N:
            wait = arr[i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.05))
    makespan = (time.perf_counter() - t0) - (arr[0] if N else 0.0)
    return StreamReport([done[k] for k in range(N)], lat, arr, makespan, steps, max_active,
                        active_sum / max(steps, 1))
