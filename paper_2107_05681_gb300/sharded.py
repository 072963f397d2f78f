"""One array sorted by the bitonic network across the ranks of a process
group, one shard per rank (the whole-array network does not shard without an
exchange step; this is that exchange).

Rank r holds elements r*n .. r*n + n - 1 of an array of G*n (G = group
size, a power of two).  The schedule is the one darm.h documents for the
shard entry points: every rank sorts its shard through stages k <= n with
the whole array's comparator directions; then for every stage k = 2n .. G*n
each layer j >= n pairs rank r with rank r ^ (j / n) - the two swap their
shards over the process group and each keeps its side of every pair - and
the layers j < n run on the shard.  The compute of every step runs in the
library's kernels (`DeviceOps`); this module only orders the steps and moves
shards between ranks with torch.distributed (NCCL between GPUs).  The steps
are injected (`ops`, `exchange`) so that the same schedule can be driven by
other implementations of the three steps.
"""
from __future__ import annotations


class DeviceOps:
    """The three steps on this rank's device, through the C ABI."""

    def __init__(self, variant="melded", stream=None):
        self.variant = variant
        self.stream = stream

    def sort_shard(self, keys, vals, shard, nshards, descending):
        import paper_2107_05681_gb300 as darm
        darm.sort_shard(keys, vals, shard, nshards, descending, self.variant, self.stream)

    def exchange(self, keys, vals, peer_keys, peer_vals, shard, nshards, log2k, log2j,
                 descending):
        import paper_2107_05681_gb300 as darm
        darm.exchange_shard(keys, vals, peer_keys, peer_vals, shard, nshards, log2k, log2j,
                            descending, self.stream)

    def merge_shard(self, keys, vals, shard, nshards, log2k, descending):
        import paper_2107_05681_gb300 as darm
        darm.merge_shard(keys, vals, shard, nshards, log2k, descending, self.variant,
                         self.stream)


def p2p_exchange(keys, vals, peer, group=None):
    """Swap this rank's shard with `peer`'s over the process group; returns
    the peer's (keys, vals) in new buffers of this rank's device."""
    import torch
    import torch.distributed as dist
    pk = torch.empty_like(keys)
    pv = None if vals is None else torch.empty_like(vals)
    ops = [dist.P2POp(dist.isend, keys, peer, group), dist.P2POp(dist.irecv, pk, peer, group)]
    if vals is not None:
        ops += [dist.P2POp(dist.isend, vals, peer, group), dist.P2POp(dist.irecv, pv, peer, group)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return pk, pv


def schedule(n: int, nshards: int):
    """The steps after the shard sort: [(log2k, [log2j, ...]), ...] - for
    every stage above the shard, its exchange layers, highest first."""
    m = n.bit_length() - 1
    M = (n * nshards).bit_length() - 1
    return [(p, list(range(p - 1, m - 1, -1))) for p in range(m + 1, M + 1)]


def partner(shard: int, n: int, log2j: int) -> int:
    """The shard rank `shard` meets in layer 2^log2j (>= n)."""
    return shard ^ ((1 << log2j) // n)


def sharded_sort(keys, vals=None, group=None, descending=False, ops=None, exchange=None):
    """Sort the array whose shard this rank holds (keys/vals), in place.
    `ops` runs the three steps (default: this device's kernels); `exchange`
    moves shards between ranks (default: torch.distributed send/recv)."""
    import torch.distributed as dist
    nshards = dist.get_world_size(group)
    shard = dist.get_rank(group)
    n = keys.numel()
    if n < 2 or n & (n - 1) or nshards & (nshards - 1):
        raise ValueError("shard length and rank count must be powers of two")
    ops = ops or DeviceOps()
    exchange = exchange or (lambda k, v, peer: p2p_exchange(k, v, peer, group))
    ops.sort_shard(keys, vals, shard, nshards, descending)
    for log2k, layers in schedule(n, nshards):
        for log2j in layers:
            pk, pv = exchange(keys, vals, partner(shard, n, log2j))
            ops.exchange(keys, vals, pk, pv, shard, nshards, log2k, log2j, descending)
        ops.merge_shard(keys, vals, shard, nshards, log2k, descending)
