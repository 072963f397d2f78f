"""The rule by which batched segmented sorts leave work out (host logic in
batch.cu, checked here on the network itself, no GPU): in a segment of
capacity 2^c with `length` real elements, sentinel-padded, the tile pass
(stages 2 .. 2^t) writes the sentinel to every tile block that starts at or
beyond the length without running its comparators, and a later stage p
leaves out every aligned 2^p block that starts at or beyond the length,
except in the segment's last pass (the layers below 2^t of stage 2^c).  Fig.
1's network with those comparators removed must give the full network's
keys and payloads, ties included."""
import numpy as np
import pytest

SENT = 0xFFFFFFFF


def _network(keys, vals, length, t, skip):
    # Fig. 1 on one segment: k = 2 .. n, j = k/2 .. 1, partner i ^ j,
    # ascending when bit k of i is clear, strict swaps
    k = keys.copy()
    v = vals.copy()
    k[length:] = SENT
    v[length:] = SENT
    n = k.size
    c = n.bit_length() - 1
    p = 1
    while (1 << p) <= n:
        kk = 1 << p
        j = kk >> 1
        while j >= 1:
            for i in range(n):
                l = i ^ j
                if l <= i:
                    continue
                if skip:
                    if p <= t and c > t and (i >> t << t) >= length:
                        continue  # tile block wholly in padding
                    last_pass = (p == c and j < (1 << t))
                    if p > t and not last_pass and (i >> p << p) >= length:
                        continue  # 2^p block of stage p wholly in padding
                asc = (i & kk) == 0
                if (k[l] < k[i]) if asc else (k[l] > k[i]):
                    k[i], k[l] = k[l], k[i]
                    v[i], v[l] = v[l], v[i]
            j >>= 1
        p += 1
    return k, v


@pytest.mark.parametrize("seed", range(6))
def test_left_out_comparators_move_nothing(seed):
    rng = np.random.default_rng(seed)
    for _ in range(8):
        c = int(rng.integers(3, 9))
        t = int(rng.integers(1, c + 1))
        n = 1 << c
        length = int(rng.choice([0, 1, n // 2, n // 2 + 1, n // 4 * 3, n, int(rng.integers(0, n + 1))]))
        keys = rng.integers(0, 5, n).astype(np.uint32)
        vals = np.arange(n, dtype=np.uint32)
        fk, fv = _network(keys, vals, length, t, skip=False)
        sk, sv = _network(keys, vals, length, t, skip=True)
        assert np.array_equal(fk, sk) and np.array_equal(fv, sv), (c, t, length)
        # the full network sorts: real keys first, ascending
        assert np.all(np.diff(fk.astype(np.int64)) >= 0)


def test_a_rule_that_skips_one_block_too_many_is_caught():
    """Leaving out the 2^p block that contains the length (start < length)
    changes the result."""
    rng = np.random.default_rng(7)
    n, t, length = 64, 2, 40
    keys = rng.integers(0, 100, n).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    fk, _ = _network(keys, vals, length, t, skip=False)

    def wrong(keys, vals):
        k = keys.copy()
        v = vals.copy()
        k[length:] = SENT
        v[length:] = SENT
        p = 1
        while (1 << p) <= n:
            kk = 1 << p
            j = kk >> 1
            while j >= 1:
                for i in range(n):
                    l = i ^ j
                    if l <= i:
                        continue
                    # off by one block: the block that holds the length too
                    if t < p < 6 and (i >> p << p) + (1 << p) > length:
                        continue
                    asc = (i & kk) == 0
                    if (k[l] < k[i]) if asc else (k[l] > k[i]):
                        k[i], k[l] = k[l], k[i]
                        v[i], v[l] = v[l], v[i]
                j >>= 1
            p += 1
        return k, v

    wk, _ = wrong(keys, vals)
    assert not np.array_equal(wk, fk)
