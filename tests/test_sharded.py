"""The sharded sort's schedule across ranks, on CPU: gloo ranks (2 and 4)
each hold one shard and run paper_2107_05681_gb300.sharded.sharded_sort with
its real exchange (torch.distributed send/recv); the three per-shard steps
are a numpy restatement of Fig. 1's layers on global indices (this test's
own, no GPU).  The shards together must equal the oracle's sort of the whole
array, payload order included."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import torch.distributed as dist
import oracle, synth
from paper_2107_05681_gb300 import sharded

class CpuOps:
    # Fig. 1's layers restricted to one shard: element i of shard s is
    # element s*n + i of the array; stage 2^p pairs i with i ^ 2^q and is
    # ascending where bit p of the array index is clear (descending flips
    # every comparator); a swap needs a strict inequality.
    def layer(self, k, v, base, p, q, desc):
        n = k.numel()
        lo = np.nonzero((np.arange(n) >> q) & 1 == 0)[0]
        hi = lo | (1 << q)
        kn, vn = k.numpy(), None if v is None else v.numpy()
        asc = (((base + lo) >> p) & 1 == 0) ^ desc
        a, b = kn[lo].copy(), kn[hi].copy()
        swap = np.where(asc, b < a, b > a)
        kn[lo], kn[hi] = np.where(swap, b, a), np.where(swap, a, b)
        if vn is not None:
            va, vb = vn[lo].copy(), vn[hi].copy()
            vn[lo], vn[hi] = np.where(swap, vb, va), np.where(swap, va, vb)
    def sort_shard(self, k, v, shard, nshards, desc):
        m = k.numel().bit_length() - 1
        for p in range(1, m + 1):
            for q in range(p - 1, -1, -1):
                self.layer(k, v, shard * k.numel(), p, q, desc)
    def exchange(self, k, v, pk, pv, shard, nshards, log2k, log2j, desc):
        n = k.numel()
        peer = shard ^ ((1 << log2j) // n)
        asc = (((shard * n) >> log2k) & 1 == 0) ^ desc
        kn, pkn = k.numpy(), pk.numpy()
        lower, upper = (kn, pkn) if shard < peer else (pkn, kn)
        swap = (upper < lower) if asc else (upper > lower)
        new_k = np.where(swap, pkn, kn)
        if v is not None:
            v.numpy()[:] = np.where(swap, pv.numpy(), v.numpy())
        kn[:] = new_k
    def merge_shard(self, k, v, shard, nshards, log2k, desc):
        m = k.numel().bit_length() - 1
        for q in range(m - 1, -1, -1):
            self.layer(k, v, shard * k.numel(), log2k, q, desc)

dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
for n, desc, mod in ((64, False, 7), (256, True, 5), (1024, False, 1 << 30)):
    keys = synth.uniform_u32(77 + n, n * world) % np.uint32(mod)
    vals = np.arange(n * world, dtype=np.uint32)
    k = torch.from_numpy(keys[rank * n:(rank + 1) * n].copy())
    v = torch.from_numpy(vals[rank * n:(rank + 1) * n].copy())
    sharded.sharded_sort(k, v, descending=desc, ops=CpuOps())
    got = [None] * world
    dist.all_gather_object(got, (k.numpy().copy(), v.numpy().copy()))
    if rank == 0:
        ek, ev = oracle.bitonic_sort(keys, vals, desc=desc)
        gk = np.concatenate([g[0] for g in got])
        gv = np.concatenate([g[1] for g in got])
        assert np.array_equal(gk, ek), (n, desc, "keys")
        assert np.array_equal(gv, ev), (n, desc, "payload")
dist.barrier()
dist.destroy_process_group()
print("rank", rank, "ok")
"""


@pytest.mark.parametrize("world,port", [(2, 29531), (4, 29533)])
def test_sharded_sort_over_gloo_ranks_equals_the_oracle(tmp_path, world, port):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
               WORLD_SIZE=str(world))
    procs = []
    for r in range(world):
        e = dict(env, RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=e, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err[-3000:]
        assert "ok" in out


def test_schedule_and_partners():
    from paper_2107_05681_gb300 import sharded
    # 4 shards of 8: stages 16 and 32; stage 16 has layer 8, stage 32 layers 16, 8
    assert sharded.schedule(8, 4) == [(4, [3]), (5, [4, 3])]
    assert [sharded.partner(s, 8, 3) for s in range(4)] == [1, 0, 3, 2]
    assert [sharded.partner(s, 8, 4) for s in range(4)] == [2, 3, 0, 1]
    assert sharded.schedule(16, 1) == []
