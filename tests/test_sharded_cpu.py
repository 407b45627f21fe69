"""The sharded growth's layer loop (one graph over P ranks, one exchange per layer) on CPU ranks:
gloo, world size 2 and 3.  Each rank runs the library's driver (grow_sharded with the
torch.distributed exchange: counts, then keys, as all-to-all; one all-reduce per layer); the
rank's device work -- partition of its frontier's candidates by owner and insert-if-absent
into its share of the visited states -- is stood in for by a host fake defined here (the CUDA
kernels run in the GPU tests).  The merged growth must equal the oracle's."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

M1 = np.uint64(0xff51afd7ed558ccd)
M2 = np.uint64(0xc4ceb9fe1a85ec53)


def mix64(k):
    # the 64-bit MurmurHash3 finaliser, as published, on numpy uint64 arrays
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        k = k ^ (k >> np.uint64(33))
        k = k * M1
        k = k ^ (k >> np.uint64(33))
        k = k * M2
        k = k ^ (k >> np.uint64(33))
    return k


def fake_owner(key, P):
    return int(mix64(np.array([key], dtype=np.uint64))[0] % np.uint64(P))


class FakeShardOps:
    """Host stand-in for ShardOps (same methods): keys in CPU int64 tensors."""

    def __init__(self, n, gens, P):
        import torch
        self.torch = torch
        self.n, self.P = n, P
        self.gens = np.asarray(gens, dtype=np.int64)
        self.seen = set()

    def empty(self):
        return self.torch.empty(0, dtype=self.torch.int64)

    def keys(self, values):
        return self.torch.tensor(np.asarray(values, dtype=np.uint64).view(np.int64))

    def partition(self, frontier):
        keys = frontier.numpy().view(np.uint64)
        sh = (4 * np.arange(self.n)).astype(np.uint64)
        digits = (keys[:, None] >> sh[None, :]) & np.uint64(15)
        cand = [((digits[:, g] << sh[None, :]).sum(axis=1, dtype=np.uint64)) for g in self.gens]
        cand = np.concatenate(cand) if cand else np.zeros(0, np.uint64)
        own = (mix64(cand) % np.uint64(self.P)).astype(np.int64)
        order = np.argsort(own, kind="stable")
        counts = np.bincount(own, minlength=self.P)
        return self.torch.tensor(cand[order].view(np.int64)), [int(c) for c in counts]

    def insert(self, keys):
        new = []
        for x in keys.numpy().view(np.uint64).tolist():
            if x not in self.seen:
                self.seen.add(x)
                new.append(x)
        return self.keys(new), len(new)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


CASES = [("coxeter", 7, None), ("lrx", 7, None), ("pancake", 6, 4), ("random", 6, None)]


def _gens(name, n):
    import workloads as w
    if name == "random":
        rng = np.random.default_rng(4)
        return w.random_perms(rng, n, 3)          # a directed set
    return w.FAMILIES[name](n)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2509_19162_gb300.sharded import TorchExchange, grow_sharded
        out = []
        for name, n, rad in CASES:
            ex = TorchExchange()
            ops = FakeShardOps(n, _gens(name, n), world)
            r = grow_sharded(n, [ops], ex, -1 if rad is None else rad, owner_of=fake_owner)
            out.append((r.layers, r.status, len(ops.seen)))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_growth_on_cpu_ranks_equals_oracle(world):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for i, (name, n, rad) in enumerate(CASES):
        want, rc = oracle.growth(n, _gens(name, n), max_radius=-1 if rad is None else rad)
        stored = 0
        for r in range(world):
            layers, status, seen = outs[r][i]
            assert layers == want, (name, r)            # every rank reports the merged growth
            assert status == (1 if rc == 1 else 0)
            stored += seen
        assert stored == sum(want)                      # each state owned by exactly one rank


def test_owner_is_the_published_hash():
    # the library's owner function is mix64(key) mod P with the MurmurHash3 finaliser
    from paper_2509_19162_gb300.sharded import owner
    rng = np.random.default_rng(8)
    for key in rng.integers(0, 2 ** 63, size=200, dtype=np.uint64).tolist() + [0, 0x76543210]:
        for P in (1, 2, 3, 8, 1000):
            assert owner(key, P) == fake_owner(key, P)
