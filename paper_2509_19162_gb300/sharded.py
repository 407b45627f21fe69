"""Growth of one Cayley graph sharded over P ranks, one exchange per layer (the BFS layer step of
Sections 3.1.2-3.1.3 split by an owner hash, owner(t) = mix64(t) mod P).

Per layer, every rank
  1. expands its share of layer r and groups the candidates by owner (cg_shard_expand, CUDA);
  2. sends each owner its candidates -- one all-to-all of packed keys (counts first);
  3. keeps the received candidates absent from its share of the visited states
     (cg_hash_insert into its own open-addressing table, CUDA): its share of layer r+1;
and |L_{r+1}| is the sum over ranks (one all-reduce).  No rank ever holds another's states.

The driver runs the ranks a process holds: one under torch.distributed (`TorchExchange`, NCCL on
GPUs), or P logical ranks on one GPU in one process (`LocalExchange`), which runs the same
kernels and the same exchange layout with the transfers done as device copies.
"""

from __future__ import annotations

import ctypes
import math
from typing import List, Optional, Sequence

import numpy as np

from . import _cg
from .api import GrowthResult, _gens_bytes, _is_inverse_closed


def owner(key: int, P: int) -> int:
    """Rank that owns packed state `key` among P ranks."""
    return int(_cg.check(_cg.cg_shard_owner(int(key), int(P)), "cg_shard_owner"))


def identity_key(n: int) -> int:
    return sum(i << (4 * i) for i in range(n))


class ShardOps:
    """The device work of one rank: its visited-state table, the owner partition of its
    frontier's candidates and the insert-if-absent of what it receives (CUDA kernels through the
    C ABI; torch tensors hold the device memory)."""

    def __init__(self, n: int, gens: Sequence[Sequence[int]], P: int, table_slots: int, device=None,
                 stream=None):
        import torch
        self.torch = torch
        self.n, self.P = n, P
        self.gens = _gens_bytes(n, gens)
        self.k = self.gens.shape[0]
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.stream = stream
        self.slots = 1 << max(10, int(table_slots - 1).bit_length())
        self.table = torch.empty(self.slots, dtype=torch.int64, device=self.device)
        _cg.check(_cg.cg_hash_clear(self.table.data_ptr(), self.slots, self._st()), "cg_hash_clear")
        self.stored = 0

    def _st(self):
        return None if self.stream is None else int(self.stream.cuda_stream)

    def empty(self):
        return self.torch.empty(0, dtype=self.torch.int64, device=self.device)

    def keys(self, values: Sequence[int]):
        a = np.asarray(values, dtype=np.uint64).view(np.int64)
        return self.torch.tensor(a, device=self.device)

    def partition(self, frontier):
        """Candidates of the frontier grouped by owner, and the count for each owner."""
        F = int(frontier.numel())
        out = self.torch.empty(max(1, self.k * F), dtype=self.torch.int64, device=self.device)
        counts = np.zeros(self.P, dtype=np.uint64)
        _cg.check(_cg.cg_shard_expand(self.n, self.k, self.gens.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                      frontier.data_ptr() if F else None, F, self.P, out.data_ptr(),
                                      out.numel(), counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                      self._st()), "cg_shard_expand")
        return out[:self.k * F], [int(c) for c in counts]

    def insert(self, keys):
        """Insert-if-absent into this rank's share of the visited states: the new ones, in a
        device tensor, form its share of the next layer."""
        N = int(keys.numel())
        out = self.torch.empty(max(1, N), dtype=self.torch.int64, device=self.device)
        cnt = self.torch.zeros(1, dtype=self.torch.int64, device=self.device)
        _cg.check(_cg.cg_hash_insert(self.table.data_ptr(), self.slots, keys.data_ptr() if N else None, N,
                                     out.data_ptr(), cnt.data_ptr(), self._st()), "cg_hash_insert")
        if self.stream is not None:
            self.stream.synchronize()
        else:
            self.torch.cuda.synchronize(self.device)
        c = int(cnt.item())
        if c < 0 or c > N:              # the insert ran out of table (count set to all ones)
            raise _cg.CgError(_cg.CG_ENOMEM, "sharded growth: a rank's visited table is full")
        self.stored += c
        return out[:c], c


class LocalExchange:
    """P logical ranks in one process (one GPU): the all-to-all is a regrouping of device
    slices, the all-reduce a sum."""

    def __init__(self, P: int):
        self.P = P
        self.ranks = list(range(P))

    def alltoall(self, sends):
        import torch
        recv = []
        offs = []
        for keys, counts in sends:
            o = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
            offs.append(o)
        for q in range(self.P):
            parts = [keys[int(o[q]):int(o[q + 1])] for (keys, _), o in zip(sends, offs)]
            recv.append(torch.cat(parts) if parts else sends[0][0][:0])
        return recv

    def allreduce(self, values):
        return int(sum(values))


class TorchExchange:
    """One rank per process over a torch.distributed process group (NCCL on GPUs, gloo on the
    host): counts first, then the keys, as all_to_all_single with split sizes."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.P = dist.get_world_size(group)
        self.ranks = [dist.get_rank(group)]

    def alltoall(self, sends):
        import torch
        (keys, counts), = sends
        dev = keys.device
        c_send = torch.tensor(counts, dtype=torch.int64, device=dev)
        c_recv = torch.empty(self.P, dtype=torch.int64, device=dev)
        self.dist.all_to_all_single(c_recv, c_send, group=self.group)
        rc = [int(x) for x in c_recv.tolist()]
        out = torch.empty(sum(rc), dtype=keys.dtype, device=dev)
        self.dist.all_to_all_single(out, keys.contiguous(), output_split_sizes=rc,
                                    input_split_sizes=list(counts), group=self.group)
        return [out]

    def allreduce(self, values):
        import torch
        dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor([int(sum(values))], dtype=torch.int64, device=dev)
        self.dist.all_reduce(t, group=self.group)
        return int(t.item())


def grow_sharded(n: int, shards: List, exchange, max_radius: int = -1, owner_of=None) -> GrowthResult:
    """The layer loop over the ranks this process holds (`shards[i]` is rank
    exchange.ranks[i]): the rank that owns the identity starts with it; every layer is one
    partition, one exchange, one insert and one sum.  owner_of(key, P) defaults to the library's."""
    owner_of = owner_of or owner
    P = exchange.P
    start = identity_key(n)
    o = owner_of(start, P)
    frontiers = []
    for r, ops in zip(exchange.ranks, shards):
        if r == o:
            f, c = ops.insert(ops.keys([start]))
            assert c == 1
        else:
            f = ops.empty()
        frontiers.append(f)
    layers = [1]
    status = _cg.CG_OK
    while True:
        if max_radius >= 0 and len(layers) - 1 >= max_radius:
            status = _cg.CG_TRUNC_RADIUS
            break
        sends = [ops.partition(f) for ops, f in zip(shards, frontiers)]
        recv = exchange.alltoall(sends)
        new = [ops.insert(keys) for ops, keys in zip(shards, recv)]
        frontiers = [f for f, _ in new]
        total = exchange.allreduce([c for _, c in new])
        if total == 0:
            break
        layers.append(total)
    return GrowthResult(layers, status)


def _table_slots(n, gens, P, order=None):
    if order is None:
        from .api import Growth
        with Growth(n, gens, _is_inverse_closed(gens)) as g:
            order = g.order
    # load about 0.4 on an even share, with room for the imbalance of the owner hash
    per = order / P
    return int(2.5 * (per + 6 * math.sqrt(per) + 64))


def sharded_growth(n: int, gens: Sequence[Sequence[int]], max_radius: int = -1, group=None,
                   stream=None) -> GrowthResult:
    """Growth of <gens> from the identity with this process as one rank of `group` (a
    torch.distributed process group over the GPUs, one rank per GPU)."""
    ex = TorchExchange(group)
    ops = ShardOps(n, gens, ex.P, _table_slots(n, gens, ex.P), stream=stream)
    return grow_sharded(n, [ops], ex, max_radius)


def sharded_growth_local(n: int, gens: Sequence[Sequence[int]], P: int, max_radius: int = -1,
                         stream=None) -> GrowthResult:
    """The same growth with P logical ranks on the current GPU (one process)."""
    slots = _table_slots(n, gens, P)
    ex = LocalExchange(P)
    shards = [ShardOps(n, gens, P, slots, stream=stream) for _ in range(P)]
    return grow_sharded(n, shards, ex, max_radius)
