"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle,
bit-exact on keys and on payload order under duplicate keys."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_equal, gpu_sort, total_order_u32

pytestmark = pytest.mark.gpu

VARIANTS = ["divergent", "melded"]


def _check(darm, keys, vals, desc, variant):
    ek, ev = oracle.bitonic_sort(keys, vals, desc=desc)
    gk, gv = gpu_sort(darm, keys, vals, desc=desc, variant=variant)
    assert_equal("keys", gk, ek)
    if vals is not None:
        assert_equal("payload", gv, ev)


@pytest.mark.parametrize("variant", VARIANTS)
def test_cfg1_single_block_4096(darm, variant):
    """4096 uniform uint32 keys, ascending, one thread block."""
    keys = synth.cfg1_keys()
    _check(darm, keys, None, False, variant)
    _check(darm, keys, np.arange(keys.size, dtype=np.uint32), False, variant)
    p, launches, tile = darm.plan_info(darm.U32, 4096, False, variant)
    assert (p, launches, tile) == (1, 1, 4096)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("desc", [False, True])
@pytest.mark.parametrize("m", list(range(1, 17)) + [18, 20])
def test_u32_kv_all_sizes(darm, m, desc, variant):
    """Every power of two up to 2^16 (tile, register and window boundaries),
    plus multi-tile sizes; heavy duplicates so payload order is tested."""
    n = 1 << m
    keys = synth.uniform_u32(1000 + m, n) % np.uint32(max(2, n // 8))
    vals = np.arange(n, dtype=np.uint32)
    _check(darm, keys, vals, desc, variant)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m", [1, 2, 5, 9, 13, 14, 15, 17, 19, 21])
def test_u32_keys_only(darm, m, variant):
    n = 1 << m
    keys = synth.uniform_u32(2000 + m, n)
    _check(darm, keys, None, False, variant)
    _check(darm, keys, None, True, variant)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m", [3, 10, 12, 13, 16, 18])
def test_u64_kv(darm, m, variant):
    n = 1 << m
    keys = synth.uniform_u64(3000 + m, n)
    idx = np.arange(0, n, 3)
    keys[idx] = keys[(idx + 1) % n]  # duplicates
    vals = np.arange(n, dtype=np.uint32)
    for desc in (False, True):
        _check(darm, keys, vals, desc, variant)
    _check(darm, keys, None, False, variant)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("m", [4, 11, 15, 17])
def test_f32_total_order(darm, m, variant):
    n = 1 << m
    x = synth.cfg3_f32(4000 + m, n, dup_frac=0.02, zeros_each=max(1, n // 32))
    for desc in (False, True):
        _check(darm, x, None, desc, variant)
        _check(darm, x, np.arange(n, dtype=np.uint32), desc, variant)


@pytest.mark.parametrize("variant", VARIANTS)
def test_buffers_16_byte_aligned_only(darm, variant):
    """Key and payload pointers 16 bytes past a 256-byte boundary: the merge
    pass's 256-bit stores must fall back to 128-bit ones and the result stay
    exact."""
    import torch

    n = 1 << 17
    keys = synth.uniform_u32(91, n) % np.uint32(1 << 12)
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.bitonic_sort(keys, vals)
    pad = np.zeros(4, dtype=np.uint32)
    kb = torch.from_numpy(np.concatenate([pad, keys])).cuda()
    vb = torch.from_numpy(np.concatenate([pad, vals])).cuda()
    K, V = kb[4:], vb[4:]
    assert K.data_ptr() % 32 == 16 and V.data_ptr() % 32 == 16
    darm.sort(K, V, variant=variant)
    torch.cuda.synchronize()
    kh, vh = kb.cpu().numpy(), vb.cpu().numpy()
    assert_equal("keys", kh[4:], ek)
    assert_equal("payload", vh[4:], ev)
    assert not kh[:4].any() and not vh[:4].any()


def test_cross_variant_identity(darm):
    n = 1 << 17
    keys = synth.uniform_u32(77, n) % np.uint32(64)
    vals = np.arange(n, dtype=np.uint32)
    outs = [gpu_sort(darm, keys, vals, variant=v) for v in ("divergent", "melded", "auto")]
    for k, v in outs[1:]:
        assert_equal("keys", k, outs[0][0])
        assert_equal("payload", v, outs[0][1])


def test_edge_cases(darm):
    import torch
    # n = 0 and n = 1 are no-ops
    for n in (0, 1):
        k = torch.from_numpy(np.full(n, 7, np.uint32)).cuda()
        darm.sort(k)
        assert k.cpu().numpy().tolist() == [7] * n
    # not a power of two
    k = torch.from_numpy(np.zeros(6, np.uint32)).cuda()
    with pytest.raises(darm.DarmError) as e:
        darm.sort(k)
    assert e.value.status == darm.ERR_NOT_POW2
    # misaligned pointer
    k = torch.from_numpy(np.zeros(33, np.uint32)).cuda()
    with pytest.raises(darm.DarmError) as e:
        darm.sort(k[1:])
    assert e.value.status == darm.ERR_INVALID_ARG
    # all-equal keys keep the identity payload
    n = 1 << 15
    keys = np.full(n, 5, np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    _, gv = gpu_sort(darm, keys, vals)
    assert_equal("payload", gv, vals)


@pytest.mark.parametrize("skew", [False, True])
def test_cfg2_kv_2pow24_full(darm, skew):
    """Key-value sort of 2^24 uint32 keys (uniform / rand mod 16) with payload
    = index: every key and payload against the oracle."""
    keys, vals = synth.cfg2_kv(skew=skew)
    ek, ev = oracle.bitonic_sort(keys, vals)
    for variant in VARIANTS:
        gk, gv = gpu_sort(darm, keys, vals, variant=variant)
        assert_equal("keys", gk, ek)
        assert_equal("payload", gv, ev)


def test_cfg3_f32_2pow26_full(darm):
    """2^26 float32 keys: the sorted key sequence is unique, so the result must
    equal the keys sorted by their totalOrder words (every element checked),
    and equal for both variants."""
    x = synth.cfg3_f32()
    order = np.argsort(total_order_u32(x), kind="stable")
    expect = x[order].view(np.uint32)
    for variant in VARIANTS:
        gk, _ = gpu_sort(darm, x, None, variant=variant)
        assert_equal("keys", gk.view(np.uint32), expect)
    # a sampled comparison with the oracle network itself on a 2^20 slice
    sl = x[: 1 << 20]
    ek, _ = oracle.bitonic_sort(sl)
    gk, _ = gpu_sort(darm, sl, None, variant="melded")
    assert_equal("keys", gk.view(np.uint32), ek.view(np.uint32))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("case", ["u32_kv_22_desc", "u32_keys_23", "f32_22_desc", "u64_kv_22",
                                  "u64_kv_22_desc"])
def test_split_whole_array_sorts(darm, case, variant):
    """Arrays of 2^22 elements and more run their two halves' tile passes and
    stages below the final one concurrently on two streams, then the final
    stage over the whole array: keys and payload order under ties against
    the oracle's single network, ascending and descending, every key kind."""
    kind, *rest = case.split("_")
    desc = rest[-1] == "desc"
    m = int(rest[-2] if desc else rest[-1])
    n = 1 << m
    hv = "kv" in rest
    if kind == "u64":
        keys = synth.uniform_u64(6100 + m, n) % np.uint64(n // 8)
    elif kind == "f32":
        keys = synth.cfg3_f32(0xDA2C0003, n)
    else:
        keys = synth.uniform_u32(6200 + m, n) % np.uint32(n // 8)
    vals = np.arange(n, dtype=np.uint32) if hv else None
    ek, ev = oracle.bitonic_sort(keys, vals, desc=desc)
    gk, gv = gpu_sort(darm, keys, vals, desc=desc, variant=variant)
    if kind == "f32":
        assert_equal("keys", total_order_u32(gk), total_order_u32(ek))
    else:
        assert_equal("keys", gk, ek)
    if hv:
        assert_equal("payload", gv, ev)
    assert darm.device_status() == 0


def test_host_buffer_sort(darm):
    n = 1 << 16
    keys = synth.uniform_u32(91, n) % np.uint32(100)
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.bitonic_sort(keys, vals, desc=True)
    k, v = keys.copy(), vals.copy()
    darm.sort_host(k, v, descending=True)
    assert_equal("keys", k, ek)
    assert_equal("payload", v, ev)


@pytest.mark.parametrize("case", ["kv_asc", "kv_desc", "f32_desc", "u64_kv", "kv_22"])
def test_host_sort_chunked_overlap(darm, case):
    """Host buffers of 2^20 or more elements are copied in 8 chunks whose
    first stages run while later chunks are still being copied; the result
    must equal the whole-array network's, payload order included."""
    m = 22 if case == "kv_22" else 20
    n = 1 << m
    desc = case.endswith("desc")
    if case == "f32_desc":
        keys = synth.cfg3_f32(4100, n, dup_frac=0.02, zeros_each=64)
    elif case == "u64_kv":
        keys = synth.uniform_u64(4101, n) % np.uint64(1 << 40)
    else:
        keys = synth.uniform_u32(4102 + m, n) % np.uint32(n // 4)
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.bitonic_sort(keys, vals, desc=desc)
    k, v = keys.copy(), vals.copy()
    darm.sort_host(k, v, descending=desc)
    assert_equal("keys", k.view(np.uint32) if k.dtype == np.float32 else k,
                 ek.view(np.uint32) if ek.dtype == np.float32 else ek)
    assert_equal("payload", v, ev)


def test_launch_counter_counts_kernels(darm):
    import torch
    before = darm.launch_count()
    k = torch.from_numpy(synth.uniform_u32(5, 1 << 20)).cuda()
    darm.sort(k)
    torch.cuda.synchronize()
    passes, launches, _ = darm.plan_info(darm.U32, 1 << 20, False)
    assert darm.launch_count() - before == launches
    assert darm.device_status() == darm.OK


def test_autotune_then_auto_variant(darm, tmp_path):
    """The tuner's choice (tile size, window depth, form per pass kind) is
    persisted, reloaded and gives the same bit-exact result."""
    db = str(tmp_path / "tune.db")
    n = 1 << 18
    darm.autotune(darm.U32, n, True, db)
    lines = open(db).read().split("\n")
    assert len([ln for ln in lines if ln.strip()]) == 1
    darm.load_tune_db(db)
    keys = synth.uniform_u32(61, n) % np.uint32(1000)
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.bitonic_sort(keys, vals)
    gk, gv = gpu_sort(darm, keys, vals, variant="auto")
    assert_equal("keys", gk, ek)
    assert_equal("payload", gv, ev)
