"""Autotuner for the launch settings of batched and single growths.

The library's defaults are rules (kernel variant from the generator count, blocks from
co-residency, jobs grown at once capped by half of L2 and at 2048, work units of 128 frontier
states, rank bitmap for dense groups of n <= 12).
The tuner times the actual workload under alternative settings and keeps the fastest, one knob at
a time (coordinate descent from the defaults), and records the winner in a JSON table keyed by a
signature of the workload and the device, so that later runs of the same kind of workload start
from it.

Every candidate setting gives the same results (the settings change how the work is laid out on
the GPU, never what is computed); the tuner checks that, and rejects a setting whose results
differ.
"""

import hashlib
import json
import os
import time
from typing import Callable, Dict, List, Optional, Sequence

from . import _cg, api

MiB = 1 << 20

# Knobs and their candidate values, in the order they are tuned.  "grid" is in blocks per SM
# (the library caps it at co-residency).
BATCH_KNOBS = (
    ("visited", ("auto", "hash", "bitmap")),
    ("ilp", (0, 1, 2, 3, 4)),
    ("grid_per_sm", (0, 4, 3, 2, 1)),
    ("wave_l2", (0, 16 * MiB, 32 * MiB, 96 * MiB, -1)),
    ("max_active", (0, 256, 512, 2048)),
    ("unit", (4, 1, 2, 8)),
    ("graph", (True, False)),
)

GROWTH_KNOBS = (
    ("strategy", ("auto", "bitmap", "hash", "sweep", "sort")),
    ("ilp", (0, 1, 2, 3, 4)),
    ("grid_per_sm", (0, 4, 3, 2, 1)),
)


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def _sm_count() -> int:
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def batch_signature(jobs: Sequence, device: Optional[str] = None) -> str:
    """Workload key of a batch: the multiset of (n, k, inverse_closed, max_radius) and the device."""
    hist: Dict[str, int] = {}
    for j in jobs:
        key = f"{j[0]}/{len(j[1])}/{int(bool(j[2]))}/{int(j[3])}"
        hist[key] = hist.get(key, 0) + 1
    text = json.dumps(sorted(hist.items())) + "|" + (device or _device_name())
    return "batch:" + hashlib.sha256(text.encode()).hexdigest()[:16]


def growth_signature(n: int, gens: Sequence[Sequence[int]], device: Optional[str] = None, **limits) -> str:
    text = json.dumps([n, [list(map(int, g)) for g in gens], sorted(limits.items())]) + "|" + \
        (device or _device_name())
    return "growth:" + hashlib.sha256(text.encode()).hexdigest()[:16]


def coordinate_descent(knobs, measure: Callable[[dict], Optional[float]], start: Optional[dict] = None):
    """Tune one knob at a time: for each knob in order, try every value with the others fixed at
    the best so far, keep the fastest.  measure(settings) returns seconds, or None when the
    setting is not applicable.  Returns (best settings, best time, trials)."""
    best = dict(start or {name: values[0] for name, values in knobs})
    best_t = measure(best)
    if best_t is None:
        raise ValueError("the starting settings are not applicable")
    trials = [(dict(best), best_t)]
    for name, values in knobs:
        for v in values:
            if v == best[name]:
                continue
            cand = dict(best)
            cand[name] = v
            t = measure(cand)
            if t is None:
                continue
            trials.append((dict(cand), t))
            if t < best_t:
                best, best_t = cand, t
    return best, best_t, trials


class TuneTable:
    """A JSON file of tuned settings: {signature: {"settings": ..., "seconds": ..., ...}}."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.entries: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def get(self, signature: str) -> Optional[dict]:
        e = self.entries.get(signature)
        return dict(e["settings"]) if e else None

    def put(self, signature: str, settings: dict, seconds: float, default_seconds: float,
            trials: List) -> None:
        self.entries[signature] = {"settings": settings, "seconds": seconds,
                                   "default_seconds": default_seconds, "trials": len(trials)}
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def batch_options(settings: dict, sms: int) -> dict:
    """Batch.set_options arguments of a settings dict."""
    return {"visited": settings["visited"], "ilp": settings["ilp"],
            "grid": settings["grid_per_sm"] * sms, "wave_l2": settings["wave_l2"],
            "max_active": settings.get("max_active", 0), "unit": settings.get("unit", 4),
            "graph": settings["graph"]}


def _time_runs(run: Callable[[], object], reps: int) -> float:
    import torch
    run()                      # first run plans (and, with graphs, captures)
    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best


def tune_batch(jobs: Sequence, stream=None, reps: int = 2, table: Optional[TuneTable] = None,
               mem_cap: int = 0, cap: int = 512) -> dict:
    """Tune the launch settings of a batch (jobs as for api.Batch) on the batch itself.
    Returns {"settings", "options", "seconds", "default_seconds", "trials", "signature"}; the
    winner is stored in `table` when one is given."""
    sms = _sm_count()
    ref = {}

    with api.Batch(jobs, mem_cap=mem_cap) as b:
        def measure(settings):
            try:
                b.set_options(**batch_options(settings, sms))
                res = [r.layers for r in b.run(stream, cap=cap)]
            except _cg.CgError:
                return None
            if "layers" not in ref:
                ref["layers"] = res
            elif res != ref["layers"]:
                raise RuntimeError(f"settings {settings} changed the results")
            return _time_runs(lambda: b.run(stream, cap=cap), reps)

        best, best_t, trials = coordinate_descent(BATCH_KNOBS, measure)
    default_t = trials[0][1]
    sig = batch_signature(jobs)
    if table is not None:
        table.put(sig, best, best_t, default_t, trials)
    return {"settings": best, "options": batch_options(best, sms), "seconds": best_t,
            "default_seconds": default_t, "trials": len(trials), "signature": sig}


def tune_growth(n: int, gens, inverse_closed: Optional[bool] = None, max_radius: int = -1,
                stop_above: int = 0, mem_cap: int = 0, stream=None, reps: int = 2,
                table: Optional[TuneTable] = None) -> dict:
    """Tune the strategy, kernel variant and blocks of one growth by running it."""
    sms = _sm_count()
    ref = {}

    def measure(settings):
        try:
            g = api.Growth(n, gens, inverse_closed, max_radius, mem_cap, settings["strategy"], stop_above)
        except (_cg.CgError, ValueError):
            return None
        try:
            if settings["ilp"]:
                g.set_ilp(settings["ilp"])
            if settings["grid_per_sm"]:
                g.set_grid(settings["grid_per_sm"] * sms)
            layers = g.run(stream).layers
            if "layers" not in ref:
                ref["layers"] = layers
            elif layers != ref["layers"]:
                raise RuntimeError(f"settings {settings} changed the results")
            return _time_runs(lambda: g.run(stream), reps)
        except _cg.CgError:
            return None
        finally:
            g.close()

    best, best_t, trials = coordinate_descent(GROWTH_KNOBS, measure)
    default_t = trials[0][1]
    sig = growth_signature(n, gens, max_radius=max_radius, stop_above=stop_above)
    if table is not None:
        table.put(sig, best, best_t, default_t, trials)
    return {"settings": best, "seconds": best_t, "default_seconds": default_t,
            "trials": len(trials), "signature": sig}
