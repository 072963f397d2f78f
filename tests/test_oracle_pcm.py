"""Pins of the PCM oracle (Section VI-A: Batcher's odd-even merge sort over
buckets of sorted keys, merge-split comparators).  No GPU needed.

Nothing here retypes the oracle's loops: the pins are numpy's sort, the
permutation property, the 0-1 principle over buckets, two closed forms
(buckets of one key make PCM the plain odd-even network; one bucket is the
bucket sort alone), the recursive formulation, a stable two-bucket merge
(heapq.merge keeps the first input's elements first on ties) and hand
traces."""
import heapq
import itertools

import numpy as np
import pytest

import oracle
import synth


def _layouts():
    return [(n, s) for n in (2, 4, 8, 16, 64, 256, 1024) for s in (1, 2, 4, 16, 64)
            if s <= n]


@pytest.mark.parametrize("n,bucket", _layouts())
def test_keys_sorted_and_payload_a_permutation(n, bucket):
    keys = synth.uniform_u32(1200 + n + bucket, n) % np.uint32(max(2, n // 4))
    vals = np.arange(n, dtype=np.uint32)
    k, v = oracle.pcm_sort(keys, vals, bucket=bucket)
    assert np.array_equal(k, np.sort(keys))
    assert np.array_equal(np.sort(v), vals)
    assert np.array_equal(keys[v], k)


def test_zero_one_principle_over_buckets():
    """Every 0/1 input of up to 16 keys, for every bucket count and size,
    comes out sorted (a merge-split network over sorted buckets sorts if
    the underlying comparator network does)."""
    for n in (4, 8, 16):
        for bucket in (1, 2, 4):
            if bucket > n:
                continue
            for bits in itertools.product((0, 1), repeat=n):
                k, _ = oracle.pcm_sort(np.array(bits, np.uint32), bucket=bucket)
                assert np.all(k[1:] >= k[:-1]), (n, bucket, bits)


@pytest.mark.parametrize("m", [1, 3, 6, 10])
def test_buckets_of_one_key_are_the_odd_even_network(m):
    """A merge-split of two one-key buckets keeps the lower bucket's key first
    on ties: the strict compare-exchange of the odd-even network."""
    n = 1 << m
    keys = synth.uniform_u32(1300 + m, n) % np.uint32(4)
    vals = np.arange(n, dtype=np.uint32)
    k1, v1 = oracle.pcm_sort(keys, vals, bucket=1)
    k2, v2, _ = oracle.oddeven_sort(keys, vals)
    assert np.array_equal(k1, k2) and np.array_equal(v1, v2)


def test_one_bucket_is_the_bucket_sort():
    keys = synth.uniform_u32(1310, 256) % np.uint32(8)
    vals = np.arange(256, dtype=np.uint32)
    k1, v1 = oracle.pcm_sort(keys, vals, bucket=256)
    k2, v2, _ = oracle.oddeven_sort(keys, vals)
    assert np.array_equal(k1, k2) and np.array_equal(v1, v2)


def test_two_buckets_are_a_stable_merge_of_the_sorted_buckets():
    for seed in range(5):
        keys = synth.uniform_u32(1320 + seed, 128) % np.uint32(6)
        vals = np.arange(128, dtype=np.uint32)
        a = oracle.oddeven_sort(keys[:64], vals[:64])
        b = oracle.oddeven_sort(keys[64:], vals[64:])
        merged = list(heapq.merge(zip(a[0].tolist(), a[1].tolist()),
                                  zip(b[0].tolist(), b[1].tolist()), key=lambda kv: kv[0]))
        k, v = oracle.pcm_sort(keys, vals, bucket=64)
        assert k.tolist() == [x[0] for x in merged]
        assert v.tolist() == [x[1] for x in merged]


@pytest.mark.parametrize("n,bucket", [(16, 2), (64, 4), (256, 8), (1024, 16), (4096, 64)])
def test_payload_order_matches_recursive_formulation(n, bucket):
    keys = synth.uniform_u32(1330 + n, n) % np.uint32(5)
    vals = np.arange(n, dtype=np.uint32)
    k1, v1 = oracle.pcm_sort(keys, vals, bucket=bucket)
    k2, v2 = oracle.pcm_sort(keys, vals, bucket=bucket, recursive=True)
    assert np.array_equal(k1, k2) and np.array_equal(v1, v2)


def test_hand_traces():
    # two buckets of two: bucket sorts [3,1] -> [1,3] (payload 1,0) and
    # [1,2] -> [1,2] (2,3); the merge-split takes bucket 0's 1 before bucket
    # 1's 1, then 2, then 3
    k, v = oracle.pcm_sort(np.array([3, 1, 1, 2], np.uint32), np.arange(4, dtype=np.uint32),
                           bucket=2)
    assert k.tolist() == [1, 1, 2, 3] and v.tolist() == [1, 2, 3, 0]
    # four buckets of two, keys 2 2 | 1 0 | 2 1 | 0 2: bucket sorts give
    # [2 2](0 1) [0 1](3 2) [1 2](5 4) [0 2](6 7); layer (0,1),(2,3):
    # [0 1](3 2) [2 2](0 1) [0 1](6 5) [2 2](4 7); layer (0,2),(1,3):
    # [0 0](3 6) [2 2](0 1) [1 1](2 5) [2 2](4 7); layer (1,2):
    # [1 1](2 5) [2 2](0 1)
    k, v = oracle.pcm_sort(np.array([2, 2, 1, 0, 2, 1, 0, 2], np.uint32),
                           np.arange(8, dtype=np.uint32), bucket=2)
    assert k.tolist() == [0, 0, 1, 1, 2, 2, 2, 2]
    assert v.tolist() == [3, 6, 2, 5, 0, 1, 4, 7]


def test_rejects_bad_layouts():
    for n, bucket in ((12, 4), (16, 3), (16, 32)):
        with pytest.raises(ValueError):
            oracle.pcm_sort(np.zeros(n, np.uint32), bucket=bucket)


def _pins_fail(mutant):
    fails = []
    for m in (3, 6):
        keys = synth.uniform_u32(1340 + m, 1 << m) % np.uint32(3)
        vals = np.arange(1 << m, dtype=np.uint32)
        k1, v1 = oracle.pcm_sort(keys, vals, bucket=1, mutant=mutant)
        k2, v2, _ = oracle.oddeven_sort(keys, vals)  # the real build
        if not (np.array_equal(k1, k2) and np.array_equal(v1, v2)):
            fails.append("one-key buckets")
            break
    k, v = oracle.pcm_sort(np.array([3, 1, 1, 2], np.uint32), np.arange(4, dtype=np.uint32),
                           bucket=2, mutant=mutant)
    if v.tolist() != [1, 2, 3, 0]:
        fails.append("hand trace")
    return fails


def test_pins_catch_planted_mistake():
    """Mutant 8 takes the upper bucket's key first on ties."""
    assert _pins_fail(8)
    assert not _pins_fail(0)
