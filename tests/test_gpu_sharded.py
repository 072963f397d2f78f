"""GPU parity of the shard building blocks (darm_bitonic_sort_shard,
darm_bitonic_exchange, darm_bitonic_merge_shard): G shards of one array
held as G buffers of this one GPU, driven through the sharded schedule
(the exchange being a copy of the peer's buffer taken before the layer), and
the shards together equal the oracle's sort of the whole array.  No kernel
waits on another: every step is a plain launch over local buffers."""
import numpy as np
import pytest

import oracle
import synth
from paper_2107_05681_gb300 import sharded
from tests.gpu_util import assert_equal, to_dev, total_order_u32

pytestmark = pytest.mark.gpu


def _run(darm, shards, vals, desc, variant):
    import torch
    G = len(shards)
    n = shards[0].numel()
    ops = sharded.DeviceOps(variant)
    for r in range(G):
        ops.sort_shard(shards[r], None if vals is None else vals[r], r, G, desc)
    for log2k, layers in sharded.schedule(n, G):
        for log2j in layers:
            before = [s.clone() for s in shards]
            vbefore = None if vals is None else [v.clone() for v in vals]
            for r in range(G):
                p = sharded.partner(r, n, log2j)
                ops.exchange(shards[r], None if vals is None else vals[r], before[p],
                             None if vals is None else vbefore[p], r, G, log2k, log2j, desc)
        for r in range(G):
            ops.merge_shard(shards[r], None if vals is None else vals[r], r, G, log2k, desc)
    torch.cuda.synchronize()


@pytest.mark.parametrize("variant", ["melded", "divergent"])
@pytest.mark.parametrize("G,m", [(2, 15), (4, 16), (8, 15)])
@pytest.mark.parametrize("desc", [False, True])
def test_key_value_shards(darm, G, m, variant, desc):
    n = 1 << m
    keys = synth.uniform_u32(1500 + G + m, n * G) % np.uint32(3000)
    vals = np.arange(n * G, dtype=np.uint32)
    shards = [to_dev(keys[r * n:(r + 1) * n]) for r in range(G)]
    vs = [to_dev(vals[r * n:(r + 1) * n]) for r in range(G)]
    _run(darm, shards, vs, desc, variant)
    ek, ev = oracle.bitonic_sort(keys, vals, desc=desc)
    assert_equal("keys", np.concatenate([s.cpu().numpy() for s in shards]), ek)
    assert_equal("payload", np.concatenate([v.cpu().numpy() for v in vs]), ev)


@pytest.mark.parametrize("desc", [False, True])
def test_float_and_u64_shards(darm, desc):
    G, n = 4, 1 << 16
    kf = synth.cfg3_f32(0xDA2C0003, n * G)
    shards = [to_dev(kf[r * n:(r + 1) * n]) for r in range(G)]
    _run(darm, shards, None, desc, "melded")
    ek, _ = oracle.bitonic_sort(kf, None, desc=desc)
    got = np.concatenate([s.cpu().numpy() for s in shards])
    assert_equal("f32 keys", total_order_u32(got), total_order_u32(ek))
    ku = synth.uniform_u64(1510, n * G) % np.uint64(5000)
    vals = np.arange(n * G, dtype=np.uint32)
    shards = [to_dev(ku[r * n:(r + 1) * n]) for r in range(G)]
    vs = [to_dev(vals[r * n:(r + 1) * n]) for r in range(G)]
    _run(darm, shards, vs, desc, "melded")
    ek, ev = oracle.bitonic_sort(ku, vals, desc=desc)
    assert_equal("u64 keys", np.concatenate([s.cpu().numpy() for s in shards]), ek)
    assert_equal("u64 payload", np.concatenate([v.cpu().numpy() for v in vs]), ev)


def test_one_shard_is_the_whole_sort(darm):
    import torch
    keys = synth.uniform_u32(1520, 1 << 16) % np.uint32(100)
    vals = np.arange(1 << 16, dtype=np.uint32)
    k, v = to_dev(keys), to_dev(vals)
    darm.sort_shard(k, v, 0, 1, descending=True)
    torch.cuda.synchronize()
    ek, ev = oracle.bitonic_sort(keys, vals, desc=True)
    assert_equal("keys", k.cpu().numpy(), ek)
    assert_equal("payload", v.cpu().numpy(), ev)


def test_shard_arguments_are_checked(darm):
    k = to_dev(np.zeros(1 << 15, np.uint32))
    with pytest.raises(darm.DarmError):
        darm.sort_shard(k, None, 4, 4)          # shard outside the array
    with pytest.raises(darm.DarmError):
        darm.merge_shard(k, None, 0, 4, 15)     # stage not above the shard
    with pytest.raises(darm.DarmError):
        darm.merge_shard(to_dev(np.zeros(1 << 12, np.uint32)), None, 0, 4, 13)  # one tile
    with pytest.raises(darm.DarmError):
        darm.exchange_shard(k, None, k, None, 0, 4, 16, 16)  # layer not below the stage
