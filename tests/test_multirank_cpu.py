"""The multi-GPU host logic on CPU ranks (gloo, world size 2): independent growth jobs shard
across ranks with no exchange step, every job runs exactly once, results reassemble in job
order, and the job-wide figures are the slowest rank's time and the sum of all ranks' work."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        import workloads as w
        from paper_2509_19162_gb300.api import shard
        jobs = [j for j in w.batch_groups(count=40) if j.n <= 7]
        mine = shard(jobs, rank, world)
        res = [oracle.growth(j.n, j.gens)[0] for j in mine]
        gathered = [None] * world
        dist.all_gather_object(gathered, res)
        work = sum(len(j.gens) * sum(r) for j, r in zip(mine, res))
        t, u = bench.combine_ranks(total_ms=10.0 * (rank + 1), units=work)
        q.put((rank, gathered, t, u, work))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_shard_batch_jobs():
    import oracle
    import workloads as w
    from paper_2509_19162_gb300.api import unshard
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    jobs = [j for j in w.batch_groups(count=40) if j.n <= 7]
    want = [oracle.growth(j.n, j.gens)[0] for j in jobs]
    total_work = sum(len(j.gens) * sum(r) for j, r in zip(jobs, want))
    for rank, gathered, t, u, work in outs:
        assert unshard(gathered, len(jobs)) == want      # every job once, in order
        assert t == 20.0                                 # slowest rank's time
        assert u == total_work                           # all ranks' work
