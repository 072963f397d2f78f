"""Pins of the oracle's synthetic divergent kernels (SB1-SB4 and their -R
variants, Section VI-A), traced by hand.  No GPU needed."""
import numpy as np
import pytest

import oracle


def _words_of_thread(d, t, blk=0):
    return [int(d[blk * 1024 + q * 256 + t]) for q in range(4)]


def test_zero_iterations_is_identity():
    d = np.arange(2048, dtype=np.uint32)
    for p in oracle.SB_PATTERNS:
        assert np.array_equal(oracle.sb_run(p, d, 0, 3), d)


def test_hand_traces_one_iteration_one_round():
    # data = 0, 1, 2, ...: thread t owns [t, 256 + t, 512 + t, 768 + t]
    d = np.arange(1024, dtype=np.uint32)
    # SB1, thread 0: j=0 second path s2=3*512+768=2304; j=1 first path
    # s1=3*256+2304=3072; j=2 second path s0=3*0+3072=3072; j=3 first path
    # s3=3*768+3072=5376
    assert _words_of_thread(oracle.sb_run("SB1", d, 1, 1), 0) == [3072, 3072, 2304, 5376]
    # SB4, thread 0: j=0 path 0 s0=3*0+256=256; j=1 path 1 s2=3*512+768=2304;
    # j=2 path 2 s0=3*256+256=1024; j=3 path 0 s3=3*768+1024=3328
    assert _words_of_thread(oracle.sb_run("SB4", d, 1, 1), 0) == [1024, 256, 2304, 3328]
    # SB4-R, thread 1 (s = 1, 257, 513, 769): j=0 path 1 s1=(5*257)^513=1796;
    # j=1 path 2 s3=7*769-1=5382; j=2 path 0 s2=3*513+5382=6921;
    # j=3 path 1 s0=(5*1)^1796=1793
    assert _words_of_thread(oracle.sb_run("SB4-R", d, 1, 1), 1) == [1793, 1796, 6921, 5382]


def test_hand_traces_if_then_regions():
    d = np.arange(1024, dtype=np.uint32)
    # SB2, thread 1 (s = 1, 257, 513, 769): j=0 path 0, s1 odd -> s0=3*1+257=260;
    # j=1 path 1 (a=3, b=0), s0=260 even -> skip; j=2 path 0, s3 odd ->
    # s2=3*513+769=2308; j=3 path 1 (a=1, b=2), s2 even -> skip
    assert _words_of_thread(oracle.sb_run("SB2", d, 1, 1), 1) == [260, 257, 2308, 769]
    # SB3, thread 2 (s = 2, 258, 514, 770): j=0 path 1 (a=2, b=3): s3 even;
    # s2&2 -> s3=3*770+514=2824.  j=1 path 0 (a=1, b=2): s2 even; s1&2 ->
    # s2=3*514+258=1800.  j=2 path 1 (a=0, b=1): s1 even; s0&2 ->
    # s1=3*258+2=776.  j=3 path 0 (a=3, b=0): s0 even; s3&2 == 0
    assert _words_of_thread(oracle.sb_run("SB3", d, 1, 1), 2) == [2, 776, 1800, 2824]
    # SB3-R, thread 2: as SB3 but path 0's second region is 7v - w:
    # j=1 -> s2=7*514-258=3340
    assert _words_of_thread(oracle.sb_run("SB3-R", d, 1, 1), 2) == [2, 776, 3340, 2824]


def test_hand_traces_sb1r_sb2r():
    # SB1-R, thread 1 of data = 0, 1, 2, ... (s = 1, 257, 513, 769); path 0
    # computes 3v + w, path 1 computes 5v ^ w.  j=0 path 0 (a=0, b=1):
    # s0=3*1+257=260; j=1 path 1 (a=3, b=0): s3=(5*769)^260=0xF05^0x104=3585;
    # j=2 path 0 (a=2, b=3): s2=3*513+3585=5124; j=3 path 1 (a=1, b=2):
    # s1=(5*257)^5124=0x505^0x1404=4353
    d = np.arange(1024, dtype=np.uint32)
    assert _words_of_thread(oracle.sb_run("SB1-R", d, 1, 1), 1) == [260, 4353, 5124, 3585]
    # thread 0 holding s = 1, 3, 5, 7 (every other word 0)
    d = np.zeros(1024, dtype=np.uint32)
    d[[0, 256, 512, 768]] = [1, 3, 5, 7]
    # SB1-R: j=0 path 1 (a=2, b=3): s2=(5*5)^7=25^7=30; j=1 path 0 (a=1, b=2):
    # s1=3*3+30=39; j=2 path 1 (a=0, b=1): s0=5^39=34; j=3 path 0 (a=3, b=0):
    # s3=3*7+34=55
    assert _words_of_thread(oracle.sb_run("SB1-R", d, 1, 1), 0) == [34, 39, 30, 55]
    # SB2-R: the same paths, each run only if s[b] is odd.  j=0 path 1, s3=7
    # odd: s2=30; j=1 path 0, s2=30 even: skip; j=2 path 1, s1=3 odd:
    # s0=5^3=6; j=3 path 0, s0=6 even: skip
    assert _words_of_thread(oracle.sb_run("SB2-R", d, 1, 1), 0) == [6, 3, 30, 7]
    # SB2 on the same data: path 1 computes 3v + w as well, so j=0 gives
    # s2=3*5+7=22 and the rest as above
    assert _words_of_thread(oracle.sb_run("SB2", d, 1, 1), 0) == [6, 3, 22, 7]


def test_blocks_are_independent():
    rng = np.random.default_rng(9)
    d = rng.integers(0, 2**32, 4096, dtype=np.uint64).astype(np.uint32)
    for p in oracle.SB_PATTERNS:
        whole = oracle.sb_run(p, d, 3, 4)
        parts = np.concatenate([oracle.sb_run(p, d[i:i + 1024], 3, 4) for i in range(0, 4096, 1024)])
        assert np.array_equal(whole, parts)


def test_identical_and_random_variants_differ():
    rng = np.random.default_rng(10)
    d = rng.integers(0, 2**32, 1024, dtype=np.uint64).astype(np.uint32)
    assert not np.array_equal(oracle.sb_run("SB1", d, 2, 2), oracle.sb_run("SB1-R", d, 2, 2))
    assert not np.array_equal(oracle.sb_run("SB4", d, 2, 2), oracle.sb_run("SB4-R", d, 2, 2))
    assert not np.array_equal(oracle.sb_run("SB2", d, 2, 2), oracle.sb_run("SB2-R", d, 2, 2))
    assert not np.array_equal(oracle.sb_run("SB3", d, 2, 2), oracle.sb_run("SB3-R", d, 2, 2))


def test_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.sb_run("SB1", np.zeros(1000, np.uint32), 1, 1)
