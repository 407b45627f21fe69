#!/usr/bin/env python
"""Benchmark of the GB300 growth library: neighbour states generated + deduplicated per second.

One step = one complete growth of the workload through the library's C ABI (default: S_11 with
the LRX generators, 39,916,800 states, 56 layers, every layer expanded).  `value` is timed on the
device (CUDA events on the run's stream, inputs resident: the handle and its buffers exist before
the timed region); `e2e` is the same metric through the public Python call `growth()` with host
inputs and outputs, host<->device copies inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload s11_lrx|s8_coxeter|s14_pancake|batch]
    python bench.py --impl reference ...     # the CPU oracle on a bounded sample, same metric

Multi-GPU (torchrun): every rank grows its own replica of the workload (the growth of one graph
has no partition without an exchange step; the library runs one GPU), value = all ranks' work /
max-over-ranks time, scaling "weak".
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "neighbour states/sec generated+deduped"
UNIT = "neighbours/s"
L2_BYTES = 129 * 1024 * 1024


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_record(kernel_name, workload, settings=None):
    """The committed ncu record of `kernel_name` on `workload` (profiles/traffic.json), or None
    when there is none, the kernel's sources changed since it was taken, or it was taken under
    other launch settings."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel_name)
        if not rec or rec.get("workload") != workload:
            return None
        if "settings" in rec and rec["settings"] != (settings or rec["settings"]):
            return None
        h = hashlib.sha256()
        for src in rec["kernel_sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        return rec if h.hexdigest() == rec["kernel_sources_sha256"] else None
    except Exception:
        return None


def issue_roofline(kernel_name, workload, kernel_ms, sm_mhz, settings=None):
    """Warp instructions issued per second against the SMs' issue rate (4 schedulers per SM, one
    warp instruction per scheduler per clock, at the SM clock sampled during the run), from the
    instruction count of the committed ncu record; None without a current record."""
    rec = measured_record(kernel_name, workload, settings)
    if not rec or "warp_instructions" not in rec or not kernel_ms:
        return None
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_mhz or 2070.0
    peak = sms * 4 * mhz * 1e6 / 1e12
    achieved = rec["warp_instructions"] / (kernel_ms / 1000.0) / 1e12
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "T warp-instr/s",
            "frac": achieved / peak, "warp_instructions": rec["warp_instructions"],
            "peak_source": f"{sms} SMs x 4 schedulers x {mhz:.0f} MHz (sampled)"}


def measured_traffic(kernel_name, workload, settings=None):
    """DRAM bytes per launch of `kernel_name` on `workload` from its committed ncu record
    (measured_record), or None without a current record."""
    rec = measured_record(kernel_name, workload, settings)
    return rec["dram_bytes"] if rec else None


def with_dram_rate(roof):
    """Add the DRAM rate the committed ncu traffic implies at the kernel time measured here
    (traffic_gbs, and traffic_frac of the same peak) to a roofline record that has both."""
    t, ms = roof.get("traffic"), roof.get("kernel_ms")
    if t and ms:
        roof["traffic_gbs"] = t / (ms / 1e3) / 1e9
        roof["traffic_frac"] = roof["traffic_gbs"] / roof["peak"]
    return roof


def algorithmic_bytes(layers, k, complete):
    """Bytes the layer steps must move (per-step model B_r): read the frontier (8 F_r), write and
    read back each candidate key (16 k F_r), read layers r and r-1 for the set difference
    (8 (F_r + F_{r-1})), write the new layer (8 F_{r+1})."""
    expanded = len(layers) if complete else len(layers) - 1
    total = 0
    for r in range(expanded):
        F = layers[r]
        Fm = layers[r - 1] if r > 0 else 0
        Fp = layers[r + 1] if r + 1 < len(layers) else 0
        total += 8 * F + 16 * k * F + 8 * (F + Fm) + 8 * Fp
    return total


def neighbours(layers, k, complete):
    """The metric's unit count: the graph's edges out of every expanded layer, k * sum F_r."""
    expanded = len(layers) if complete else len(layers) - 1
    return k * sum(layers[:expanded])


def generated_candidates(n, gens, layers, complete, skips_parent):
    """Candidates the kernels actually generate and probe.  The key-list strategies (bitmap and
    hash) store a state found through generator g with the tag of g's inverse and do not expand
    that edge (it leads back to the parent): when every distinct generator's inverse is in the
    set among its first 15 rows and n <= 15, each state after the first skips one generator.
    None when only some generators have their inverse there (the count depends on the path)."""
    expanded = len(layers) if complete else len(layers) - 1
    rows = []
    for g in gens:
        t = tuple(int(x) for x in g)
        if t != tuple(range(n)) and t not in rows:
            rows.append(t)
    k = len(rows)
    total = k * sum(layers[:expanded])
    if not skips_parent or n > 15 or expanded == 0:
        return total
    def inv(t):
        r = [0] * len(t)
        for i, v in enumerate(t):
            r[v] = i
        return tuple(r)
    tagged = [inv(t) in rows[:15] for t in rows]
    if all(tagged):
        return total - sum(layers[1:expanded])
    return total if not any(tagged) else None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def combine_ranks(total_ms, units):
    """Job-wide figures of a multi-rank run: the slowest rank's time (MAX) and all ranks' work
    (SUM), over the default process group (NCCL on GPUs, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def get_workload(name):
    if name == "s11_lrx":
        return wl.config_s11_lrx()
    if name == "s8_coxeter":
        return wl.config_s8_coxeter()
    if name == "s14_pancake":
        return wl.config_s14_pancake()
    if ":" in name:
        # any named family, full growth: e.g. "pancake:14" (the whole of S_14), "coxeter:13";
        # a third field "bin" grows the orbit of the binary vector 0^(n/2) 1^(n - n/2) (the
        # "Bin" Schreier coset graph), e.g. "lrx:32:bin"
        parts = name.split(":")
        fam, n = parts[0], int(parts[1])
        gens = wl.FAMILIES[fam](n)
        if len(parts) > 2 and parts[2] == "bin":
            return wl.GrowthJob(n, gens, wl.is_inverse_closed(gens), name=f"Bin{n}-{fam}-k{len(gens)}-full",
                                family=fam, start=wl.binary_start(n))
        return wl.GrowthJob(n, gens, wl.is_inverse_closed(gens), name=f"S{n}-{fam}-k{len(gens)}-full",
                            family=fam)
    raise ValueError(name)


# --------------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)

# Bounded samples of each workload for the oracle: the growth up to this radius (the oracle
# expands layers 0..R-1).  About 10-20 s of one host core for S_11 LRX.
ORACLE_SAMPLE_RADIUS = {"s11_lrx": 32, "s8_coxeter": -1, "s14_pancake": 6}
REFERENCE_STEP_RADIUS = {"s11_lrx": 28, "s8_coxeter": -1, "s14_pancake": 5}


def oracle_sample(job, radius):
    import oracle
    t0 = time.perf_counter()
    layers, rc = oracle.growth(job.n, job.gens, max_radius=radius, start=job.start)
    dt = time.perf_counter() - t0
    complete = (rc == 0)
    return neighbours(layers, job.k, complete), dt, layers, complete


def sample_radius(job, budget_s):
    """Largest radius whose oracle growth ends within about budget_s (for workloads without a
    fixed sample): radii are tried in order until one takes more than a quarter of the budget."""
    import oracle
    R = 1
    while True:
        t0 = time.perf_counter()
        _, rc = oracle.growth(job.n, job.gens, max_radius=R, start=job.start)
        if rc == 0:
            return -1
        if time.perf_counter() - t0 > budget_s / 4:
            return R
        R += 1


def cpu_baseline(wname, job):
    R = ORACLE_SAMPLE_RADIUS[wname] if wname in ORACLE_SAMPLE_RADIUS else sample_radius(job, 20.0)
    nb, dt, layers, complete = oracle_sample(job, R)
    return {"value": nb / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{job.name}: growth to radius {len(layers) - 1} "
                      f"({'complete' if complete else 'expanding layers 0..%d' % (len(layers) - 2)}), "
                      f"{nb} neighbours in {dt:.2f} s, single-threaded unordered_set BFS",
            "host_nproc": os.cpu_count()}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    job = get_workload(args.workload)
    R = (REFERENCE_STEP_RADIUS[args.workload] if args.workload in REFERENCE_STEP_RADIUS
         else sample_radius(job, 10.0))
    for _ in range(args.warmup):
        oracle_sample(job, R)
    total_nb, total_t = 0, 0.0
    last = None
    for _ in range(args.steps):
        nb, dt, layers, complete = oracle_sample(job, R)
        total_nb += nb
        total_t += dt
        last = (layers, complete)
    value = total_nb / total_t
    sample = (f"{job.name}: growth to radius {len(last[0]) - 1} per step "
              f"({'complete' if last[1] else 'expanding layers 0..%d' % (len(last[0]) - 2)})")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
           "data": "synthetic", "config": {"workload": job.name, "n": job.n, "k": job.k},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# --------------------------------------------------------------------------------------------
# GPU arm

def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2509_19162_gb300 as cg
    cg.build()
    from paper_2509_19162_gb300 import _cg  # noqa: F401  (load the library)

    job = get_workload(args.workload)
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")

    handle = cg.Growth(job.n, job.gens, job.inverse_closed, job.max_radius,
                       stop_above=job.stop_above, keep_last=False, strategy=args.strategy,
                       start=job.start)
    handle.set_sweep_order(args.sweep_order)
    # warm-up (also allocates the job's buffers: inputs resident before the timed region)
    res = None
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            res = handle.run(stream)
    complete = res.status == 0
    layers = res.layers
    nb_step = neighbours(layers, job.k, complete)
    bytes_step = algorithmic_bytes(layers, job.k, complete)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    sampler = ClockSampler(local) if rank == 0 or world == 1 else None
    barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kernel_ms = 0.0
    launches = 0
    st0 = handle.stats()
    strat_name = {1: "hash", 2: "sort", 3: "bitmap", 4: "sweep"}.get(st0["strategy_used"], "?")
    variant = st0["probe_variant"]
    # kernel names as ncu prints them: the single-job bitmap kernel with one generator in
    # flight is compiled per n (last template argument), every other variant has 0 there
    per_n = job.n if (strat_name == "bitmap" and variant == 17 and 2 <= job.n <= 14) else 0
    # the sweep's block order changes its memory traffic: its ncu record names the order
    launch_settings = {"sweep_order": args.sweep_order} if strat_name == "sweep" else None
    kernel_name = {"sort": "radix sort / merge-path kernels",
                   "sweep": f"sweep_grow_kernel<{min(variant, 2)}, {job.n}>"}.get(
        strat_name, f"hash_grow_kernel<{variant & 7}, {variant >> 3}, 0, {per_n}>")
    for i in range(args.steps):
        flush.zero_()                               # evict L2 between timed steps
        torch.cuda.synchronize()
        ev[i][0].record(stream)
        r = handle.run(stream)
        ev[i][1].record(stream)
        st = handle.stats()
        kernel_ms += st["kernel_ms"]
        launches += st["launches"]
        if r.layers != layers:
            raise RuntimeError("layer counts changed between steps")
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    units_all = nb_step * args.steps
    if world > 1:
        total_ms, units_all = combine_ranks(total_ms, units_all)
    value = units_all / (total_ms / 1000.0)

    # end to end through the public API: create + run + destroy with host inputs/outputs (the
    # timed handle's buffers are released first: a growth may size them to the memory cap)
    handle.close()
    e2e_times = []
    h2d = d2h = 0
    for i in range(max(1, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with cg.Growth(job.n, job.gens, job.inverse_closed, job.max_radius,
                       stop_above=job.stop_above, strategy=args.strategy, start=job.start) as g:
            g.set_sweep_order(args.sweep_order)
            r = g.run(stream)
            st = g.stats()
        e2e_times.append(time.perf_counter() - t0)
        h2d, d2h = st["h2d_bytes"], st["d2h_bytes"]
        if r.layers != layers:
            raise RuntimeError("e2e layer counts differ")
    e2e_value = world * nb_step / statistics.median(e2e_times)

    peak, peak_kind = load_peaks()
    kern_ms_per = kernel_ms / args.steps
    achieved = bytes_step / (kern_ms_per / 1000.0) / 1e9

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": job.name, "n": job.n, "k": job.k, "states": sum(layers),
                   "layers": len(layers), "neighbours_per_step": nb_step,
                   "generated_per_step": generated_candidates(job.n, job.gens, layers, complete,
                                                              strat_name in ("bitmap", "hash")),
                   "counting": "value and roofline count k * sum F_r neighbours (every edge out of "
                               "every expanded layer) and the algorithmic bytes of that growth; "
                               "generated_per_step is what the kernel expands after skipping each "
                               "state's parent edge",
                   "strategy": strat_name + {
                       "sort": " (sorted layers: expand, radix sort, merge-path difference)",
                       "sweep": " (bitmaps over S_n for the visited set and layers; one persistent "
                                "cooperative launch)"}.get(
                       strat_name, " (visited set; one persistent cooperative launch)"),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   **(launch_settings or {})},
        "roofline_issue": issue_roofline(kernel_name, job.name, kern_ms_per,
                                         (clocks or {}).get("sm_mhz"), launch_settings),
        "roofline": with_dram_rate({
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": measured_traffic(kernel_name, job.name, launch_settings),
            "kernel": kernel_name,
            "kernel_ms": kern_ms_per, "algorithmic_bytes": bytes_step,
            "peak_source": peak_kind}),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "api": "paper_2509_19162_gb300.Growth(...).run()"},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, job)
    if world == 1 and not args.no_extra and args.workload == "s11_lrx" and args.strategy == "auto":
        out["extra"] = extra_configs(cg, stream, flush)
    print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------------------------
# Config 4: 4096 independent random groups, one persistent launch per batch run

def measure_batch(cg, spec, stream, flush, steps, warmup, autotune=True, tune_table=None):
    """Time batched runs of `spec` (jobs as for Batch): optionally autotuned first (outside the
    timed region), then `warmup` untimed and `steps` timed runs with L2 flushed between them."""
    import torch
    tuned = None
    if autotune:
        from paper_2509_19162_gb300 import tune
        t0 = time.perf_counter()
        table = tune.TuneTable(tune_table) if tune_table else None
        tuned = tune.tune_batch(spec, stream=stream, table=table)
        tuned["tuning_s"] = time.perf_counter() - t0
    batch = cg.Batch(spec, **(tuned["options"] if tuned else {}))
    res = None
    for _ in range(max(1, warmup)):
        res = batch.run(stream)
    layers = [r.layers for r in res]
    total_ms, kernel_ms, launches = 0.0, 0.0, 0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = batch.run(stream)
        b.record(stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
        st = batch.stats()
        kernel_ms += st["kernel_ms"]
        launches += st["launches"]
        if [r.layers for r in out] != layers:
            raise RuntimeError("batched layer counts changed between steps")
    variant = batch.stats()["probe_variant"]
    batch.close()
    return {"layers": layers, "statuses": [r.status for r in res], "total_ms": total_ms,
            "kernel_ms": kernel_ms, "launches": launches, "variant": variant, "tuned": tuned}


def one_at_a_time(cg, jobs, stream, mem_cap=0, strategies=None, per_job=None):
    """Jobs run one after another through growth() on the same GPU: (layers, seconds).  per_job:
    a list that receives each job's seconds."""
    import torch
    strategies = strategies or ["auto"] * len(jobs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = []
    for j, s in zip(jobs, strategies):
        t = time.perf_counter()
        out.append(cg.growth(j.n, j.gens, j.inverse_closed, j.max_radius, mem_cap=mem_cap, strategy=s,
                             stream=stream).layers)
        if per_job is not None:
            per_job.append(time.perf_counter() - t)
    return out, time.perf_counter() - t0


def run_batch(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2509_19162_gb300 as cg
    cg.build()
    jobs_all = wl.batch_groups()
    jobs = cg.shard(jobs_all, rank, world)        # the groups shard across ranks, no exchange
    spec = [(j.n, j.gens, j.inverse_closed, -1) for j in jobs]
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    m = measure_batch(cg, spec, stream, flush, args.steps, args.warmup, not args.no_autotune,
                      args.tune_table)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    layers, tuned, launches = m["layers"], m["tuned"], m["launches"]
    nb_step = sum(len(j.gens) * sum(l) for j, l in zip(jobs, layers))
    bytes_step = sum(algorithmic_bytes(l, len(j.gens), True) for j, l in zip(jobs, layers))
    total_ms = m["total_ms"]
    if world > 1:
        total_ms, nb_all = combine_ranks(total_ms, nb_step)
    else:
        nb_all = nb_step
    value = nb_all * args.steps / (total_ms / 1000.0)
    jobs_per_s = len(jobs_all) * args.steps / (total_ms / 1000.0)
    # end to end: create + run + destroy from host inputs
    t0 = time.perf_counter()
    with cg.Batch(spec) as b2:
        b2.run(stream)
        est = b2.stats()
    e2e_s = time.perf_counter() - t0
    # one at a time, same GPU, first 512 groups of this rank's share (same results required)
    sample = jobs[:512]
    single, one_s = one_at_a_time(cg, sample, stream)
    if single != layers[:len(sample)]:
        raise RuntimeError("one-at-a-time results differ from the batched results")
    peak, peak_kind = load_peaks()
    kms = m["kernel_ms"] / args.steps
    achieved = bytes_step / (kms / 1000.0) / 1e9
    variant = m["variant"]
    if rank != 0:
        return 0
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"batched-{len(jobs_all)}-random-groups-seed{wl.BATCH_SEED}",
                   "groups": len(jobs_all), "states": sum(sum(l) for l in layers),
                   "neighbours_per_step": nb_step, "jobs_per_s": jobs_per_s,
                   "one_at_a_time_jobs_per_s": len(sample) / one_s,
                   "batched_over_one_at_a_time": jobs_per_s / (len(sample) / one_s),
                   "autotune": None if not tuned else {
                       "settings": tuned["settings"], "tuned_ms": tuned["seconds"] * 1e3,
                       "default_ms": tuned["default_seconds"] * 1e3, "trials": tuned["trials"],
                       "tuning_s": tuned["tuning_s"]},
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "groups sharded over ranks" if world > 1 else "single GPU"},
        "roofline": with_dram_rate({
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": measured_traffic(f"hash_grow_kernel<{variant & 7}, {variant >> 3}, 1, 0>",
                                        f"batched-{len(jobs_all)}-random-groups-seed{wl.BATCH_SEED}",
                                        tuned["settings"] if tuned else None),
            "kernel": f"hash_grow_kernel<{variant & 7}, {variant >> 3}, 1, 0> (multi-job, one "
                      f"persistent launch per batch run admitting the jobs by the L2 window)",
            "kernel_ms": kms, "algorithmic_bytes": bytes_step, "peak_source": peak_kind}),
        "e2e": {"value": nb_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": est["h2d_bytes"],
                "d2h_bytes_per_step": est["d2h_bytes"], "api": "paper_2509_19162_gb300.Batch(...).run()"},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(out))
    return 0


# --------------------------------------------------------------------------------------------
# Config 5: Poisson stream of growth jobs through the continuous-batching server

SERVE_BUDGET = 160 << 30


def measure_serve(cg, jobs, stream, rates=(1.0, 2.0), slots=512, rounds=8, job_mem=0, lam_sample=200):
    """Serve `jobs` at multiples of the one-at-a-time capacity lambda_1 (measured first on the
    same GPU, each job alone with the same per-job share).  job_mem = 0: the server's default
    share of the 160 GiB budget (budget / 64).  Returns (lambda_1, [one summary per rate])."""
    import numpy as np
    from paper_2509_19162_gb300.serve import Server, serve_stream
    share = job_mem or SERVE_BUDGET // 64
    plans = [Server.predict(j.n, j.gens, j.inverse_closed, j.max_radius, job_mem_cap=share) for j in jobs]
    over = [i for i, p in enumerate(plans) if p["granted"] < p["states"]]
    sample = jobs[:lam_sample]
    # each job alone with the memory and the visited set the server gives it (no hand-off to
    # the sorted step, which the server does not make either)
    strat = [p["visited"] for p in plans[:lam_sample]]
    one_at_a_time(cg, sample[:10], stream, mem_cap=share, strategies=strat[:10])
    per_job = []
    alone, one_s = one_at_a_time(cg, sample, stream, mem_cap=share, strategies=strat, per_job=per_job)
    lam1 = len(sample) / one_s
    # where one-at-a-time time goes: jobs the server grows alone (each fills the GPU) and the
    # jobs it batches -- and those batched jobs alone against served together (all queued at once)
    solo = [p["alone"] for p in plans]
    small = [j for j, a in zip(jobs, solo) if not a]
    small_alone_s = []
    one_at_a_time(cg, small, stream, mem_cap=share,
                  strategies=[p["visited"] for p, a in zip(plans, solo) if not a], per_job=small_alone_s)
    with Server(mem_budget=SERVE_BUDGET, max_slots=slots, job_mem_cap=share, rounds_per_step=rounds) as srv:
        t0 = time.perf_counter()
        serve_stream(small, [0.0] * len(small), srv, stream, realtime=False)
        small_served_s = time.perf_counter() - t0
    split = {"sample_jobs": len(sample),
             "sample_alone_s_grown_alone_by_server": sum(t for t, a in zip(per_job, solo) if a),
             "sample_alone_s_batched_by_server": sum(t for t, a in zip(per_job, solo) if not a),
             "jobs_grown_alone_by_server": sum(solo), "jobs_batched_by_server": len(small),
             "batched_jobs_one_at_a_time_s": sum(small_alone_s),
             "batched_jobs_served_together_s": small_served_s}
    out = []
    for mult in rates:
        lam = lam1 * mult
        arr = [j.arrival / lam for j in jobs]
        with Server(mem_budget=SERVE_BUDGET, max_slots=slots, job_mem_cap=share,
                    rounds_per_step=rounds) as srv:
            sampler = ClockSampler(0)
            sampler.start()
            rep = serve_stream(jobs, arr, srv, stream)
            clocks = sampler.stop()
        statuses = [r.status for r in rep.results]
        memcap_ended = [i for i, st in enumerate(statuses) if st == 2]
        for a, r in zip(alone, rep.results):           # the same growth alone and in the mix
            m = min(len(a), len(r.layers))
            if a[:m] != r.layers[:m]:
                raise RuntimeError("a served job's layers differ from the same job grown alone")
        out.append({
            "rate": f"{mult:g} x one-at-a-time capacity", "arrival_rate_jobs_per_s": lam,
            "jobs_per_s": rep.jobs_per_s, "makespan_s": rep.makespan_s,
            "latency_ms": {"p50": rep.percentile_ms(50), "p99": rep.percentile_ms(99),
                           "mean": float(np.mean(rep.latency_s) * 1000.0)},
            "server_steps": rep.steps, "max_active": rep.max_active, "mean_active": rep.mean_active,
            "ended": {"complete": statuses.count(0), "radius_cap": statuses.count(1),
                      "mem_cap": statuses.count(2)},
            # every job stopped by memory is one whose predicted states exceed its share
            "mem_cap_all_predicted_over_share": set(memcap_ended) <= set(over),
            "clocks": clocks})
    return lam1, {"jobs": len(jobs), "job_share_bytes": share, "budget_bytes": SERVE_BUDGET,
                  "predicted_over_share": len(over), "predicted_over_share_ids": over[:50],
                  "time_split": split}, out


def run_serve(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import paper_2509_19162_gb300 as cg
    cg.build()
    jobs = wl.serve_stream(count=args.serve_jobs)
    stream = torch.cuda.Stream()
    lam1, info, rates = measure_serve(cg, jobs, stream, rates=(1.0, 2.0, 4.0), slots=args.serve_slots,
                                      rounds=args.serve_rounds, job_mem=args.serve_job_mem << 20)
    for r in rates:
        print(json.dumps({
            "metric": "jobs/sec + p50/p99 latency (serving)", "value": r["jobs_per_s"], "unit": "jobs/s",
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": r["makespan_s"] * 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"serving-{len(jobs)}-jobs-seed{wl.SERVE_SEED}", **info,
                       "slots": args.serve_slots, "rounds_per_step": args.serve_rounds,
                       **{k: v for k, v in r.items() if k not in ("jobs_per_s", "latency_ms", "clocks")}},
            "latency_ms": r["latency_ms"], "one_at_a_time_jobs_per_s": lam1, "clocks": r["clocks"]}))
    return 0


# --------------------------------------------------------------------------------------------
# The other configurations, measured briefly beside the default line (its `extra`)

def quick_growth(cg, job, stream, flush, steps=3, warmup=2):
    """A few timed runs of one growth: rate, time per run, kernel time and its HBM fraction."""
    import torch
    with cg.Growth(job.n, job.gens, job.inverse_closed, job.max_radius, stop_above=job.stop_above,
                   start=job.start) as g:
        for _ in range(warmup):
            r = g.run(stream)
        ms, kms = [], []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r2 = g.run(stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            kms.append(g.stats()["kernel_ms"])
            if r2.layers != r.layers:
                raise RuntimeError("layer counts changed between steps")
        st = g.stats()
    complete = r.status == 0
    nb = neighbours(r.layers, job.k, complete)
    peak, _ = load_peaks()
    t, kt = statistics.median(ms), statistics.median(kms)
    return {"workload": job.name, "value": nb / (t / 1000.0), "unit": UNIT, "ms_per_step": t,
            "kernel_ms": kt, "layers": len(r.layers), "states": sum(r.layers), "status": r.status,
            "strategy": {1: "hash", 2: "sort", 3: "bitmap", 4: "sweep"}.get(st["strategy_used"], "?"),
            "roofline_frac": algorithmic_bytes(r.layers, job.k, complete) / (kt / 1000.0) / 1e9 / peak,
            "steps": steps}


def extra_configs(cg, stream, flush):
    """Configs 1, 3, 4 and 5 measured briefly (the default line's value stays config 2)."""
    out = {"config1": quick_growth(cg, wl.config_s8_coxeter(), stream, flush, steps=10, warmup=3),
           "config3": quick_growth(cg, wl.config_s14_pancake(), stream, flush, steps=3, warmup=1)}
    jobs = wl.batch_groups()
    spec = [(j.n, j.gens, j.inverse_closed, -1) for j in jobs]
    m = measure_batch(cg, spec, stream, flush, steps=3, warmup=2, autotune=False)
    single, one_s = one_at_a_time(cg, jobs[:256], stream)
    if single != m["layers"][:256]:
        raise RuntimeError("one-at-a-time results differ from the batched results")
    t = m["total_ms"] / 3
    jps = len(jobs) / (t / 1000.0)
    out["config4"] = {"workload": f"batched-{len(jobs)}-random-groups-seed{wl.BATCH_SEED}",
                      "value": sum(len(j.gens) * sum(l) for j, l in zip(jobs, m["layers"])) / (t / 1000.0),
                      "unit": UNIT, "ms_per_step": t, "jobs_per_s": jps,
                      "one_at_a_time_jobs_per_s": 256 / one_s,
                      "batched_over_one_at_a_time": jps / (256 / one_s),
                      "launches_per_run": m["launches"] // 3, "settings": "library defaults",
                      "all_complete": all(s == 0 for s in m["statuses"])}
    sjobs = wl.serve_stream(count=1000)
    lam1, info, rates = measure_serve(cg, sjobs, stream, rates=(1.0, 2.0), lam_sample=100)
    out["config5"] = {"workload": f"serving-first-1000-of-20000-jobs-seed{wl.SERVE_SEED}", **info,
                      "one_at_a_time_jobs_per_s": lam1,
                      "rates": [{k: v for k, v in r.items() if k != "clocks"} for r in rates]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="s11_lrx",
                    help="s11_lrx | s8_coxeter | s14_pancake | batch | serve | <family>:<n> "
                         "(full growth of a named family, e.g. pancake:14)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload: skip the brief runs of configs 1, 3, 4 and 5 (extra)")
    ap.add_argument("--strategy", default="auto", choices=["auto", "hash", "bitmap", "sort", "sweep"],
                    help="visited-set strategy of the single-job workloads")
    ap.add_argument("--sweep-order", default="auto", choices=["auto", "discovery", "rank"],
                    help="sweep strategy: order in which a round takes a layer's blocks")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batch workload: run with the library's default launch settings")
    ap.add_argument("--tune-table", default=None, help="JSON file to record tuned settings in")
    ap.add_argument("--serve-jobs", type=int, default=20000)
    ap.add_argument("--serve-job-mem", type=int, default=0,
                    help="per-job device memory share, MiB (0: the server default, budget / 64)")
    ap.add_argument("--serve-slots", type=int, default=512)
    ap.add_argument("--serve-rounds", type=int, default=8)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        if args.workload in ("batch", "serve"):
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle arm covers the single-growth workloads"}))
            return 0
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
