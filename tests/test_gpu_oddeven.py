"""GPU parity of the single-block odd-even merge sort network (both forms)
against the oracle, bit-exact on keys and on payload order under ties."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_equal, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("m", range(1, 13))
def test_all_sizes_with_ties(darm, m, variant):
    import torch
    n = 1 << m
    keys = synth.uniform_u32(700 + m, n) % np.uint32(max(2, n // 16))
    vals = np.arange(n, dtype=np.uint32)
    ek, ev, _ = oracle.oddeven_sort(keys, vals)
    k, v = to_dev(keys), to_dev(vals)
    darm.oddeven_sort_block(k, v, variant=variant)
    torch.cuda.synchronize()
    assert_equal("keys", k.cpu().numpy(), ek)
    assert_equal("payload", v.cpu().numpy(), ev)
    k = to_dev(keys)
    darm.oddeven_sort_block(k, variant=variant)
    torch.cuda.synchronize()
    assert_equal("keys only", k.cpu().numpy(), ek)


def test_uniform_4096_both_forms_identical(darm):
    import torch
    keys = synth.cfg1_keys()
    vals = np.arange(keys.size, dtype=np.uint32)
    ek, ev, _ = oracle.oddeven_sort(keys, vals)
    for variant in ("divergent", "melded", "auto"):
        k, v = to_dev(keys), to_dev(vals)
        darm.oddeven_sort_block(k, v, variant=variant)
        torch.cuda.synchronize()
        assert_equal(f"{variant} keys", k.cpu().numpy(), ek)
        assert_equal(f"{variant} payload", v.cpu().numpy(), ev)


def test_rejects_bad_sizes(darm):
    with pytest.raises(darm.DarmError):
        darm.oddeven_sort_block(to_dev(np.zeros(8192, np.uint32)))
    with pytest.raises(darm.DarmError):
        darm.oddeven_sort_block(to_dev(np.zeros(6, np.uint32)))
    k = to_dev(np.array([5], np.uint32))
    darm.oddeven_sort_block(k)  # n = 1: nothing to do
    assert k.cpu().numpy().tolist() == [5]


_BUCKET_CACHE = {}


def _oracle_buckets(keys, vals, bucket, tag):
    """Every bucket sorted on its own by the oracle network (computed once
    per input and shared by both kernel forms)."""
    if tag not in _BUCKET_CACHE:
        ek = np.empty_like(keys)
        ev = None if vals is None else np.empty_like(vals)
        for b in range(0, keys.size, bucket):
            bk, bv, _ = oracle.oddeven_sort(keys[b:b + bucket],
                                            None if vals is None else vals[b:b + bucket])
            ek[b:b + bucket] = bk
            if vals is not None:
                ev[b:b + bucket] = bv
        _BUCKET_CACHE.clear()
        _BUCKET_CACHE[tag] = (ek, ev)
    return _BUCKET_CACHE[tag]


def _first_bad_bucket(got, exp, bucket):
    bad = np.nonzero((got != exp).reshape(-1, bucket).any(axis=1))[0]
    return None if bad.size == 0 else int(bad[0])


@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("bucket", [2, 256, 4096])
def test_buckets_each_sorted_like_the_oracle(darm, bucket, variant):
    """One thread block per bucket: every bucket (all of them) equals the
    oracle's sort of that bucket alone, payload order included."""
    import torch
    n = 1 << 18
    keys = synth.uniform_u32(800 + bucket, n) % np.uint32(512)
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = _oracle_buckets(keys, vals, bucket, ("ties", bucket))
    k, v = to_dev(keys), to_dev(vals)
    darm.oddeven_sort_buckets(k, v, bucket=bucket, variant=variant)
    torch.cuda.synchronize()
    gk, gv = k.cpu().numpy(), v.cpu().numpy()
    assert _first_bad_bucket(gk, ek, bucket) is None, "keys differ in a bucket"
    assert _first_bad_bucket(gv, ev, bucket) is None, "payload differs in a bucket"
    assert_equal("keys", gk, ek)
    assert_equal("payload", gv, ev)


@pytest.mark.parametrize("variant", ["divergent", "melded"])
def test_oem26_full_size_every_bucket(darm, variant):
    """The bucketed odd-even workload at full size, as the benchmark runs it:
    2^26 uniform uint32 keys, 4096-key buckets, one thread block each; all
    16,384 buckets against the oracle."""
    import torch
    bucket = 4096
    keys = synth.uniform_u32(0xDA2C0006, 1 << 26)
    ek, _ = _oracle_buckets(keys, None, bucket, ("oem26", bucket))
    k = to_dev(keys)
    darm.oddeven_sort_buckets(k, bucket=bucket, variant=variant)
    torch.cuda.synchronize()
    gk = k.cpu().numpy()
    bad = _first_bad_bucket(gk, ek, bucket)
    assert bad is None, f"bucket {bad} differs from the oracle"


def test_bucket_arguments_are_checked(darm):
    k = to_dev(np.zeros(1 << 12, np.uint32))
    for bucket in (3, 8192):
        with pytest.raises(darm.DarmError):
            darm.oddeven_sort_buckets(k, bucket=bucket)
    with pytest.raises(darm.DarmError):
        darm.oddeven_sort_buckets(to_dev(np.zeros(6000, np.uint32)), bucket=4096)
