"""GPU parity of the tile pass with shuffle stages (stages 2E .. 32E across
the lanes of a warp by __shfl_xor_sync, both forms) against the oracle:
bit-exact keys and payload order under ties, ascending and descending."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_equal, gpu_sort, total_order_u32

pytestmark = pytest.mark.gpu

# the library's default tunings of 32-bit keys, with the shuffle flag set:
# key kind, payload, log2 n, log2 tile, E (tile), E (window), window threads,
# windows per pass, staging buffers, forms, time, shuffle stages
_KEYS = "0 0 {m} 14 5 5 8 2 2 1 1 1 0.0 1"
_PAIRS = "0 1 {m} 12 4 4 8 2 1 1 1 1 0.0 1"


@pytest.fixture()
def shfl_tuned(darm, tmp_path):
    db = str(tmp_path / "shfl.db")
    with open(db, "w") as f:
        for m in range(12, 27):
            f.write(_KEYS.format(m=m) + "\n")
            f.write(_PAIRS.format(m=m) + "\n")
    darm.reset_tunings()
    darm.load_tune_db(db)
    yield darm
    darm.reset_tunings()


def _assert_shfl_plan(darm, dtype, n, has_vals, variant):
    lines = darm.plan_describe(dtype, n, has_vals, variant)
    assert lines[0].startswith("tile") and "~" in lines[0].split()[0], lines[0]


@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("m", [13, 14, 15, 17, 20])
@pytest.mark.parametrize("desc", [False, True])
def test_keys_only(shfl_tuned, m, variant, desc):
    darm = shfl_tuned
    n = 1 << m
    keys = synth.uniform_u32(900 + m, n) % np.uint32(max(4, n // 8))
    _assert_shfl_plan(darm, darm.U32, n, False, variant)
    ek, _ = oracle.bitonic_sort(keys, None, desc=desc)
    gk, _ = gpu_sort(darm, keys, None, desc=desc, variant=variant)
    assert_equal("keys", gk, ek)


@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("m", [12, 13, 16, 18])
@pytest.mark.parametrize("desc", [False, True])
def test_key_value_payload_order(shfl_tuned, m, variant, desc):
    darm = shfl_tuned
    n = 1 << m
    keys = synth.uniform_u32(950 + m, n) % np.uint32(64)  # heavy duplicates
    vals = np.arange(n, dtype=np.uint32)
    _assert_shfl_plan(darm, darm.U32, n, True, variant)
    ek, ev = oracle.bitonic_sort(keys, vals, desc=desc)
    gk, gv = gpu_sort(darm, keys, vals, desc=desc, variant=variant)
    assert_equal("keys", gk, ek)
    assert_equal("payload", gv, ev)


@pytest.mark.parametrize("variant", ["divergent", "melded"])
def test_float_keys(shfl_tuned, variant):
    darm = shfl_tuned
    keys = synth.cfg3_f32(0xDA2C0003, 1 << 20)
    _assert_shfl_plan(darm, darm.F32, keys.size, False, variant)
    ek, _ = oracle.bitonic_sort(keys, None)
    gk, _ = gpu_sort(darm, keys, None, variant=variant)
    assert_equal("keys", total_order_u32(gk), total_order_u32(ek))


_MERGE2 = "0 0 {m} 14 5 5 8 2 2 1 1 1 0.0 3"


@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("desc", [False, True])
def test_two_round_shuffle_merge(darm, tmp_path, variant, desc):
    """The merge pass in two rounds (its lane layers by shuffles), selected by
    bit 1 of the shuffle tuning field: the same network, bit for bit."""
    db = str(tmp_path / "merge2.db")
    with open(db, "w") as f:
        for m in range(15, 22):
            f.write(_MERGE2.format(m=m) + "\n")
    darm.reset_tunings()
    darm.load_tune_db(db)
    try:
        for m in (15, 18, 21):
            n = 1 << m
            lines = darm.plan_describe(darm.U32, n, False, variant)
            assert any(ln.startswith("merge") and "rounds=2" in ln for ln in lines), lines
            keys = synth.uniform_u32(980 + m, n) % np.uint32(n // 4)
            ek, _ = oracle.bitonic_sort(keys, None, desc=desc)
            gk, _ = gpu_sort(darm, keys, None, desc=desc, variant=variant)
            assert_equal("keys", gk, ek)
    finally:
        darm.reset_tunings()
