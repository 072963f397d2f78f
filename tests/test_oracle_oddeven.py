"""Pins of the oracle's odd-even merge sort network (Batcher's network, the
base of the paper's PCM benchmark, Section VI-A).  No GPU needed."""
import itertools

import numpy as np
import pytest

import oracle
import synth


def test_zero_one_principle_all_inputs():
    """A comparator network sorts every input iff it sorts every 0/1 input:
    all 2^n 0/1 vectors for n = 2, 4, 8, 16."""
    for n in (2, 4, 8, 16):
        for bits in range(1 << n):
            k = np.array([(bits >> i) & 1 for i in range(n)], dtype=np.uint32)
            out, _, _ = oracle.oddeven_sort(k)
            ones = int(k.sum())
            assert not out[: n - ones].any() and out[n - ones:].all(), (n, bits)


@pytest.mark.parametrize("p", range(1, 13))
def test_comparator_count_closed_form(p):
    """Batcher's network on n = 2^p elements has (p^2 - p + 4) 2^(p-2) - 1
    comparators (Knuth, TAOCP vol. 3, 5.3.4); a dropped or extra condition
    in the loop nest changes the count."""
    n = 1 << p
    _, _, ncmp = oracle.oddeven_sort(np.zeros(n, np.uint32))
    expected = 1 if p == 1 else (p * p - p + 4) * (1 << (p - 2)) - 1
    assert ncmp == expected


@pytest.mark.parametrize("m", [3, 8, 12, 14])
def test_keys_sorted_and_payload_is_a_permutation(m):
    n = 1 << m
    keys = synth.uniform_u32(500 + m, n) % np.uint32(max(2, n // 8))
    vals = np.arange(n, dtype=np.uint32)
    k, v, _ = oracle.oddeven_sort(keys, vals)
    assert np.array_equal(k, np.sort(keys))
    assert np.array_equal(np.sort(v), vals)
    assert np.array_equal(keys[v], k)


@pytest.mark.parametrize("m", [2, 5, 9, 12])
def test_payload_order_matches_recursive_formulation(m):
    """Payload order under ties is fixed by the network: the iterative loop
    nest and Batcher's recursive sort/merge must agree element for element."""
    n = 1 << m
    keys = synth.uniform_u32(600 + m, n) % np.uint32(7)
    vals = np.arange(n, dtype=np.uint32)
    k1, v1, _ = oracle.oddeven_sort(keys, vals)
    k2, v2, _ = oracle.oddeven_sort(keys, vals, recursive=True)
    assert np.array_equal(k1, k2) and np.array_equal(v1, v2)


def test_equal_keys_never_move():
    """Strict swaps: all-equal keys leave the payload in index order."""
    for m in range(1, 11):
        n = 1 << m
        _, v, _ = oracle.oddeven_sort(np.full(n, 5, np.uint32), np.arange(n, dtype=np.uint32))
        assert np.array_equal(v, np.arange(n, dtype=np.uint32))


def test_small_hand_case():
    """n = 4 by hand: layers (0,1)(2,3) | (0,2)(1,3) | (1,2)."""
    k, v, ncmp = oracle.oddeven_sort(np.array([3, 1, 1, 0], np.uint32),
                                     np.arange(4, dtype=np.uint32))
    # (0,1): 1 3 | (2,3): 0 1  -> [1,3,0,1] vals [1,0,3,2]
    # (0,2): 0 .. 1 -> [0,3,1,1] vals [3,0,1,2]; (1,3): 1 .. 3 -> [0,1,1,3] vals [3,2,1,0]
    # (1,2): equal keys, no swap
    assert ncmp == 5
    assert k.tolist() == [0, 1, 1, 3] and v.tolist() == [3, 2, 1, 0]


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.oddeven_sort(np.arange(6, dtype=np.uint32))


def _pins_fail(mutant):
    """True when some pin of this file rejects an oracle built with a planted
    mistake (run on small cases)."""
    fails = []
    # comparator count
    for p in range(2, 7):
        _, _, ncmp = oracle.oddeven_sort(np.zeros(1 << p, np.uint32), mutant=mutant)
        if ncmp != (p * p - p + 4) * (1 << (p - 2)) - 1:
            fails.append("count")
            break
    # equal keys never move / payload order equals the recursive form
    for m in (3, 6):
        n = 1 << m
        keys = synth.uniform_u32(610 + m, n) % np.uint32(3)
        vals = np.arange(n, dtype=np.uint32)
        k1, v1, _ = oracle.oddeven_sort(keys, vals, mutant=mutant)
        k2, v2, _ = oracle.oddeven_sort(keys, vals, recursive=True)  # the real build
        if not (np.array_equal(k1, k2) and np.array_equal(v1, v2)):
            fails.append("recursive")
            break
    return fails


@pytest.mark.parametrize("mutant", [6, 7])
def test_pins_catch_planted_mistakes(mutant):
    """6: the same-block test dropped; 7: equal keys swapped."""
    assert _pins_fail(mutant), f"mutant {mutant} passed every odd-even pin"
    assert not _pins_fail(0)
