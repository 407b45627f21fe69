"""GPU tests of the serving loop: every job's growth is the same alone and in the mix, jobs that
arrive while others are on the GPU are admitted as slots and memory free up, and the memory
budget bounds what is admitted."""

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


def small_stream(count=160, seed=7):
    return w.serve_stream(seed=seed, count=count, n_range=(6, 10))


def test_stream_results_equal_alone(cg):
    from paper_2509_19162_gb300.serve import Server, serve_stream
    jobs = small_stream()
    arr = [j.arrival * 0.0005 for j in jobs]          # 2000 jobs/s offered load
    with Server(mem_budget=8 << 30, max_slots=64, job_mem_cap=512 << 20, rounds_per_step=4) as s:
        rep = serve_stream(jobs, arr, s)
    assert rep.max_active > 1                       # work of several jobs overlapped
    for j, r in zip(jobs, rep.results):
        alone = cg.growth(j.n, j.gens, j.inverse_closed, max_radius=j.max_radius)
        assert r.status in (0, 1, 2)
        if r.status == 2:                           # stopped by its memory cap: exact prefix
            assert r.layers == alone.layers[:len(r.layers)]
        else:
            assert r.layers == alone.layers and r.status == alone.status
    for j, r in list(zip(jobs, rep.results))[:25]:
        if j.n <= 8:
            want, rc = oracle.growth(j.n, j.gens, max_radius=j.max_radius)
            assert r.layers == want


def test_budget_limits_admission(cg):
    from paper_2509_19162_gb300.serve import Server, serve_stream
    jobs = [j for j in small_stream(count=40, seed=11) if j.n <= 8][:12]
    with Server(mem_budget=1, max_slots=16, job_mem_cap=64 << 20, rounds_per_step=2) as s:
        rep = serve_stream(jobs, [0.0] * len(jobs), s, realtime=False)
    assert rep.max_active == 1                      # nothing fits beside a running job
    for j, r in zip(jobs, rep.results):
        assert r.layers == cg.growth(j.n, j.gens, j.inverse_closed, max_radius=j.max_radius).layers


def test_late_arrivals_join_running_jobs(cg):
    from paper_2509_19162_gb300.serve import Server
    big = (9, w.lrx(9), True, -1)                   # 36 layers: 18 steps of 2 rounds
    with Server(max_slots=8, rounds_per_step=2) as s:
        a = s.submit(*big[:2], big[2], big[3])
        s.step()                                    # a is on the GPU
        b = s.submit(8, w.coxeter(8), True, -1)     # arrives while a runs
        seen_both = False
        done = {}
        while len(done) < 2:
            active, _ = s.step()
            seen_both |= active == 2
            for jid in s.finished():
                done[jid] = s.result(jid)
        assert seen_both
        assert done[b].layers == oracle.growth(8, w.coxeter(8))[0]
        assert done[a].layers == oracle.growth(9, w.lrx(9))[0] and done[a].status == 0


def test_jobs_that_fill_the_gpu_are_grown_alone(cg):
    # S_11 LRX (39.9M states predicted) is grown by the single-job kernels when it reaches the
    # head of the queue; the small jobs queued around it are batched, in order
    import os
    from paper_2509_19162_gb300.serve import Server
    golden = os.path.join(os.path.dirname(__file__), "golden", "s11_lrx_growth.txt")
    want = [int(l.split()[1]) for l in open(golden) if not l.startswith("#")]
    assert Server.predict(11, w.lrx(11), True, -1)["states"] >= 1 << 24
    with Server(max_slots=8, rounds_per_step=4) as s:
        ids = [s.submit(8, w.coxeter(8), True, -1), s.submit(11, w.lrx(11), True, -1),
               s.submit(7, w.pancake(7), True, -1)]
        done = {}
        while len(done) < 3:
            s.step()
            for jid in s.finished():
                done[jid] = s.result(jid)
    assert done[ids[1]].layers == want and done[ids[1]].status == 0
    assert done[ids[0]].layers == oracle.growth(8, w.coxeter(8))[0]
    assert done[ids[2]].layers == oracle.growth(7, w.pancake(7))[0]


def _mahonian(n):
    poly = np.array([1], dtype=object)
    for j in range(1, n + 1):
        poly = np.convolve(poly, np.ones(j, dtype=object))
    return [int(x) for x in poly]


def _stirling_growth(n):
    c = [[0] * (n + 1) for _ in range(n + 1)]
    c[0][0] = 1
    for m in range(1, n + 1):
        for j in range(1, m + 1):
            c[m][j] = c[m - 1][j - 1] + (m - 1) * c[m - 1][j]
    return [c[n][n - r] for r in range(n)]


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name + ".txt")
    return [int(l.split()[1]) for l in open(path) if not l.startswith("#") and l.strip()]


def test_serving_stream_full_n_range_against_closed_forms(cg):
    # Config 5's own recipe (n = 8..16, five families, radius caps up to the family's diameter
    # bound), first 240 jobs of the seeded stream, all arriving at once.  Every job's layers are
    # exact: Coxeter jobs are Mahonian prefixes, all-transpositions jobs Stirling prefixes, jobs
    # with n <= 10 the oracle's growth to the same radius, S_11..S_13 LRX / pancake jobs prefixes
    # of the stored oracle growths; a job stopped by memory reports an exact prefix.
    from paper_2509_19162_gb300.serve import Server, serve_stream
    jobs = w.serve_stream(count=240)
    assert {j.n for j in jobs} >= set(range(11, 17))
    with Server(mem_budget=96 << 30, max_slots=256, job_mem_cap=256 << 20, rounds_per_step=4) as s:
        rep = serve_stream(jobs, [0.0] * len(jobs), s, realtime=False)
    stored = {("lrx", 11): _golden("s11_lrx_growth"), ("lrx", 12): _golden("s12_lrx_growth_b"),
              ("pancake", 12): _golden("s12_pancake_growth_b"),
              ("pancake", 13): _golden("s13_pancake_growth")}
    checked_closed = 0
    for j, r in zip(jobs, rep.results):
        assert r.status in (0, 1, 2), j.name
        if r.status == 1:
            assert len(r.layers) == j.max_radius + 1, j.name
        want = None
        if j.family == "coxeter":
            want = _mahonian(j.n)
        elif j.family == "all_transpositions":
            want = _stirling_growth(j.n)
        elif (j.family, j.n) in stored:
            want = stored[(j.family, j.n)]
        if want is not None:
            checked_closed += j.n >= 11
            if r.status == 0:
                assert r.layers == want, j.name
            else:
                assert r.layers == want[:len(r.layers)], j.name
        elif j.n <= 10:
            full, rc = oracle.growth(j.n, j.gens, max_radius=j.max_radius)
            assert r.layers == full[:len(r.layers)], j.name
            if r.status != 2:
                assert r.layers == full, j.name
        else:                                       # no closed form: the same job alone
            alone = cg.growth(j.n, j.gens, j.inverse_closed, max_radius=j.max_radius,
                              mem_cap=256 << 20)
            m = min(len(alone.layers), len(r.layers))
            assert r.layers[:m] == alone.layers[:m], j.name
    assert checked_closed >= 40
