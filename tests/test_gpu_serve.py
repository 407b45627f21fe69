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
    big = (11, w.lrx(11), True, -1)
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
        assert sum(done[a].layers) == 39916800 and done[a].status == 0
