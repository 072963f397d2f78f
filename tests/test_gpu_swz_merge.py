"""GPU parity of the passes that stream 32-bit keys (no payload) through
shared memory with TMA tensor copies and work on them in place: the
swizzled merge pass (tiles of 2^13 and 2^14 keys in the 128-byte swizzled
layout) and the two-window pass (blocks of 16 consecutive keys x 2 windows
of 5 bits, round 1 pair-swapped in half of each warp), against the oracle,
bit-exact, both directions, through the device and host-buffer entry
points."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_equal, gpu_sort, total_order_u32

pytestmark = pytest.mark.gpu

# key kind, payload, log2 n, log2 tile, E (tile), E (window), window threads,
# windows per pass, staging buffers (3: swizzled in place), forms, time,
# shuffle stages
_LINE = "0 0 {m} {t} 5 5 8 2 3 1 1 1 0.0 1"


@pytest.fixture(params=[13, 14])
def swz_tuned(darm, tmp_path, request):
    t = request.param
    db = str(tmp_path / f"swz{t}.db")
    with open(db, "w") as f:
        for m in range(t + 1, 27):
            f.write(_LINE.format(m=m, t=t) + "\n")
    darm.reset_tunings()
    darm.load_tune_db(db)
    yield darm, t
    darm.reset_tunings()


def _assert_swz_plan(darm, dtype, n, t):
    merges = [L for L in darm.plan_dump(dtype, n, False, "melded",
                                        tuning=(t, 5, 5, 8, 2, 3, 1)) if L["kind"] == 2]
    assert merges and all(L["tma"] == 3 for L in merges), [L["tma"] for L in merges]


@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("m", [15, 17, 20, 22])
@pytest.mark.parametrize("desc", [False, True])
def test_keys_only(swz_tuned, m, variant, desc):
    """Several tiles per CTA (2^22 keys: 256 or 512 tiles on 152 SMs, a
    ragged last wave) and fewer tiles than SMs (2^15)."""
    darm, t = swz_tuned
    n = 1 << m
    keys = synth.uniform_u32(1300 + m, n) % np.uint32(max(4, n // 8))
    _assert_swz_plan(darm, darm.U32, n, t)
    ek, _ = oracle.bitonic_sort(keys, None, desc=desc)
    gk, _ = gpu_sort(darm, keys, None, desc=desc, variant=variant)
    assert_equal("keys", gk, ek)


@pytest.mark.parametrize("desc", [False, True])
def test_float_keys_key_map_in_last_merge(swz_tuned, desc):
    """The last merge pass undoes the float key map (and the descending
    complement) before its bulk store."""
    darm, t = swz_tuned
    keys = synth.cfg3_f32(0xDA2C0003, 1 << 21)
    _assert_swz_plan(darm, darm.F32, keys.size, t)
    ek, _ = oracle.bitonic_sort(keys, None, desc=desc)
    gk, _ = gpu_sort(darm, keys, None, desc=desc)
    assert_equal("keys", total_order_u32(gk), total_order_u32(ek))


def test_host_buffers(swz_tuned):
    """Host-buffer sorts run the final stage's last merges per chunk: the
    tensor map then covers one chunk from its own base."""
    darm, t = swz_tuned
    keys = synth.uniform_u32(0x5A11, 1 << 23)
    ek, _ = oracle.bitonic_sort(keys, None)
    hk = keys.copy()
    darm.sort_host(hk)
    assert_equal("keys", hk, ek)


def test_default_plan_uses_it(darm):
    """With tensor maps available the default plan of 2^26 keys runs its
    merge passes in place (the full-size parity tests cover that plan)."""
    darm.reset_tunings()
    merges = [L for L in darm.plan_dump(darm.F32, 1 << 26, False, "melded") if L["kind"] == 2]
    assert len(merges) == 12 and all(L["tma"] == 3 for L in merges)
    assert darm.device_status() == 0


@pytest.mark.parametrize("desc", [False, True])
@pytest.mark.parametrize("dtype", ["u32", "f32"])
def test_tma_two_window_passes(darm, desc, dtype):
    """2^24 keys with the default plan: two-window passes of six to ten
    layers streamed by TMA (the ten-layer one runs the pair-swapped lowest
    layer), swizzled merges."""
    darm.reset_tunings()
    n = 1 << 24
    code = darm.U32 if dtype == "u32" else darm.F32
    plan = darm.plan_dump(code, n, False, "melded")
    w2t = [L for L in plan if L["win2"] == 2]
    assert w2t and any(L["rounds"][1]["cnt"] == 5 for L in w2t), [L["win2"] for L in plan]
    if dtype == "u32":
        keys = synth.uniform_u32(0x2A0E, n) % np.uint32(n // 4)
        ek, _ = oracle.bitonic_sort(keys, None, desc=desc)
        gk, _ = gpu_sort(darm, keys, None, desc=desc)
        assert_equal("keys", gk, ek)
    else:
        keys = synth.cfg3_f32(0xDA2C0003, n)
        ek, _ = oracle.bitonic_sort(keys, None, desc=desc)
        gk, _ = gpu_sort(darm, keys, None, desc=desc)
        assert_equal("keys", total_order_u32(gk), total_order_u32(ek))
    assert darm.device_status() == 0


_KV = "0 1 {m} {t} 4 4 8 2 3 1 1 1 0.0 1"


@pytest.fixture(params=[12, 13])
def swz_kv_tuned(darm, tmp_path, request):
    t = request.param
    db = str(tmp_path / f"swzkv{t}.db")
    with open(db, "w") as f:
        for m in range(t + 1, 27):
            f.write(_KV.format(m=m, t=t) + "\n")
    darm.reset_tunings()
    darm.load_tune_db(db)
    yield darm, t
    darm.reset_tunings()


@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("m", [14, 17, 21])
@pytest.mark.parametrize("desc", [False, True])
def test_key_value_in_place_merge(swz_kv_tuned, m, variant, desc):
    """Key-value merges in place (keys and payloads in two swizzled
    buffers): payload order under heavy ties is the network's, bit for bit."""
    darm, t = swz_kv_tuned
    n = 1 << m
    merges = [L for L in darm.plan_dump(darm.U32, n, True, variant,
                                        tuning=(t, 4, 4, 8, 2, 3, 1)) if L["kind"] == 2]
    assert merges and all(L["tma"] == 3 for L in merges)
    keys = synth.uniform_u32(2100 + m, n) % np.uint32(max(4, n // 64))
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.bitonic_sort(keys, vals, desc=desc)
    gk, gv = gpu_sort(darm, keys, vals, desc=desc, variant=variant)
    assert_equal("keys", gk, ek)
    assert_equal("payload", gv, ev)


def test_key_value_in_place_merge_host_buffers(swz_kv_tuned):
    darm, t = swz_kv_tuned
    n = 1 << 22
    keys = synth.uniform_u32(0x5A12, n) % np.uint32(1 << 12)
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.bitonic_sort(keys, vals)
    hk, hv = keys.copy(), vals.copy()
    darm.sort_host(hk, hv)
    assert_equal("keys", hk, ek)
    assert_equal("payload", hv, ev)


@pytest.mark.parametrize("case", [("u32", 15, 14), ("kv", 13, 12), ("kv", 14, 12)])
@pytest.mark.parametrize("m", [16, 21])
@pytest.mark.parametrize("desc", [False, True])
def test_merge_tile_smaller_than_tile(darm, tmp_path, case, m, desc):
    """Merge passes on tiles smaller than the tile pass's: the window passes
    of every stage above the tile also take the bits in between (keys with a
    2^15-key tile pass and 2^14-key merges; pairs with 2^13- or 2^14-pair
    tile passes and 2^12-pair merges)."""
    kind, t, tm = case
    hv = kind == "kv"
    db = str(tmp_path / "tm.db")
    with open(db, "w") as f:
        for mm in range(t + 1, 27):
            if hv:
                f.write(f"0 1 {mm} {t} 4 4 8 2 3 1 1 1 0.0 1 0 {tm}\n")
            else:
                f.write(f"0 0 {mm} {t} 5 5 8 2 3 1 1 1 0.0 1 0 {tm}\n")
    darm.reset_tunings()
    darm.load_tune_db(db)
    try:
        n = 1 << m
        plan = darm.plan_dump(darm.U32, n, hv, "melded",
                              tuning=(t, 4 if hv else 5, 4 if hv else 5, 8, 2, 3, 1, tm))
        assert plan[0]["b"] == t and all(L["b"] == tm for L in plan if L["kind"] == 2)
        keys = synth.uniform_u32(4400 + m + t, n) % np.uint32(max(4, n // 16))
        vals = np.arange(n, dtype=np.uint32) if hv else None
        ek, ev = oracle.bitonic_sort(keys, vals, desc=desc)
        gk, gv = gpu_sort(darm, keys, vals, desc=desc)
        assert_equal("keys", gk, ek)
        if hv:
            assert_equal("payload", gv, ev)
        assert darm.device_status() == 0
    finally:
        darm.reset_tunings()
