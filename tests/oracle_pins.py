"""Checks that pin the CPU oracle to facts outside itself.

Each check returns None when it holds and a short message when it fails, so
that the same checks run against the real oracle (tests/test_oracle.py) and
against builds of it with one planted mistake (tests/test_oracle_mutants.py).

Sources of truth used here, none of which is the oracle itself:
  * numpy's sort (a textbook sorting routine) for the key sequence;
  * the 0-1 principle (Knuth, TAOCP vol. 3, 5.3.4): a comparator network
    sorts every input iff it sorts every 0/1 input; brute force over all
    2^n inputs for n <= 16;
  * permutation invariants of the payload;
  * the independent recursive formulation for payload order under ties;
  * hand-worked traces of Fig. 1 on 4-element inputs (see the comments);
  * the mirror identity desc(x) == asc(~x) that follows from flipping every
    comparator;
  * IEEE-754 totalOrder for float keys.
"""
from __future__ import annotations

import numpy as np

import oracle
import synth


def _fail(msg):
    return msg


def check_sorted_like_numpy(mutant=0, seed=11):
    for m in range(0, 13):
        n = 1 << m
        keys = synth.uniform_u32(seed + m, n)
        for desc in (False, True):
            out, _ = oracle.bitonic_sort(keys, desc=desc, mutant=mutant)
            ref = np.sort(keys)
            if desc:
                ref = ref[::-1]
            if not np.array_equal(out, ref):
                return _fail(f"u32 keys differ from numpy sort at n={n} desc={desc}")
        keys64 = synth.uniform_u64(seed + 100 + m, n)
        out, _ = oracle.bitonic_sort(keys64, mutant=mutant)
        if not np.array_equal(out, np.sort(keys64)):
            return _fail(f"u64 keys differ from numpy sort at n={n}")
    return None


def check_payload_permutation(mutant=0, seed=12):
    for m in (1, 3, 6, 10, 13):
        n = 1 << m
        for skew in (False, True):
            keys = synth.uniform_u32(seed + m, n)
            if skew:
                keys = keys % np.uint32(5)
            vals = np.arange(n, dtype=np.uint32)
            for desc in (False, True):
                ko, vo = oracle.bitonic_sort(keys, vals, desc=desc, mutant=mutant)
                if not np.array_equal(np.sort(vo), vals):
                    return _fail(f"payload is not a permutation (n={n})")
                if not np.array_equal(ko, keys[vo]):
                    return _fail(f"payload does not travel with its key (n={n})")
    return None


def check_zero_one_principle(mutant=0, max_n=16):
    n = 2
    while n <= max_n:
        # all 2^n 0/1 vectors at once: row r holds the bits of r
        rows = np.arange(1 << n, dtype=np.uint32)
        bits = ((rows[:, None] >> np.arange(n, dtype=np.uint32)[None, :]) & 1).astype(np.uint32)
        ones = bits.sum(axis=1)
        for desc in (False, True):
            for r in range(bits.shape[0]):
                out, _ = oracle.bitonic_sort(bits[r], desc=desc, mutant=mutant)
                c = int(ones[r])
                if desc:
                    ok = out[:c].all() and not out[c:].any()
                else:
                    ok = (not out[:n - c].any()) and out[n - c:].all()
                if not ok:
                    return _fail(f"0/1 input {r:#x} of length {n} not sorted (desc={desc})")
        n *= 2
    return None


def check_recursive_agrees(mutant=0, seed=13):
    """Iterative (mutant build) versus recursive (always the real build)."""
    for m in (1, 2, 3, 5, 8, 11):
        n = 1 << m
        for mod in (2, 3, 16, 0):
            keys = synth.uniform_u32(seed + m * 7 + mod, n)
            if mod:
                keys = keys % np.uint32(mod)
            vals = np.arange(n, dtype=np.uint32)
            for desc in (False, True):
                ki, vi = oracle.bitonic_sort(keys, vals, desc=desc, mutant=mutant)
                kr, vr = oracle.bitonic_sort(keys, vals, desc=desc, recursive=True)
                if not (np.array_equal(ki, kr) and np.array_equal(vi, vr)):
                    return _fail(f"iterative != recursive at n={n} mod={mod} desc={desc}")
    return None


import os

_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                       "fig1_hand_traces.txt")


def load_hand_traces(path=_GOLDEN):
    """(keys, desc, expected keys, expected vals) rows worked by hand from
    Fig. 1; the derivations are in the fixture's comment header."""
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            d, kin, kout, vout = [c.strip() for c in line.split("|")]
            rows.append(([int(x) for x in kin.split()], d == "desc",
                         [int(x) for x in kout.split()], [int(x) for x in vout.split()]))
    return rows


HAND_TRACES = load_hand_traces()


def check_hand_traces(mutant=0):
    for keys, desc, ek, ev in HAND_TRACES:
        k = np.array(keys, dtype=np.uint32)
        v = np.arange(k.size, dtype=np.uint32)
        ko, vo = oracle.bitonic_sort(k, v, desc=desc, mutant=mutant)
        if ko.tolist() != ek or vo.tolist() != ev:
            return _fail(f"hand trace {keys} desc={desc}: got {ko.tolist()} {vo.tolist()}")
    return None


def check_all_equal_identity(mutant=0):
    for m in range(1, 12):
        n = 1 << m
        keys = np.full(n, 42, dtype=np.uint32)
        vals = np.arange(n, dtype=np.uint32)
        for desc in (False, True):
            _, vo = oracle.bitonic_sort(keys, vals, desc=desc, mutant=mutant)
            if not np.array_equal(vo, vals):
                return _fail(f"all-equal keys moved payload at n={n}")
    return None


def check_desc_mirror(mutant=0, seed=14):
    for m in (2, 4, 7, 10):
        n = 1 << m
        keys = synth.uniform_u32(seed + m, n) % np.uint32(9)
        vals = np.arange(n, dtype=np.uint32)
        kd, vd = oracle.bitonic_sort(keys, vals, desc=True, mutant=mutant)
        ka, va = oracle.bitonic_sort(~keys, vals, desc=False, mutant=mutant)
        if not (np.array_equal(kd, ~ka) and np.array_equal(vd, va)):
            return _fail(f"desc(x) != asc(~x) at n={n}")
    return None


def check_f32_total_order(mutant=0, seed=15):
    for m in (3, 9, 12):
        n = 1 << m
        x = synth.cfg3_f32(seed + m, n, dup_frac=0.05, zeros_each=max(1, n // 16))
        for desc in (False, True):
            out, _ = oracle.bitonic_sort(x, desc=desc, mutant=mutant)
            ref = np.sort(x)
            if desc:
                ref = ref[::-1]
            if not np.array_equal(out, ref):       # numeric order (0.0 == -0.0)
                return _fail(f"f32 order differs from numpy at n={n}")
            zeros = out[out == 0]
            neg = np.signbit(zeros)
            # totalOrder: every -0.0 precedes every +0.0 (reversed when descending)
            expect = np.sort(neg)[::-1] if not desc else np.sort(neg)
            if not np.array_equal(neg, expect):
                return _fail(f"signed zeros out of totalOrder at n={n}")
            if np.count_nonzero(neg) != np.count_nonzero(np.signbit(x[x == 0])):
                return _fail("signed zeros lost")
    return None


def check_segmented(mutant=0, seed=16):
    segs = synth.cfg4_segments(seed, num_segments=40, min_len=1, max_len=700,
                               mixed_dirs=True)
    ko, vo = oracle.segmented_sort(segs.keys, segs.vals, segs.offsets, segs.lengths,
                                   desc_per_seg=segs.desc, mutant=mutant)
    for s in range(segs.num_segments):
        a, b = int(segs.offsets[s]), int(segs.offsets[s + 1])
        ln = int(segs.lengths[s])
        d = bool(segs.desc[s])
        real = segs.keys[a:a + ln]
        sent = np.uint32(0 if d else 0xFFFFFFFF)
        ref = np.concatenate([np.sort(real), np.full(b - a - ln, sent, np.uint32)])
        if d:
            ref = np.concatenate([np.sort(real)[::-1], np.full(b - a - ln, sent, np.uint32)])
        if not np.array_equal(ko[a:b], ref):
            return _fail(f"segment {s} keys wrong")
        pv = vo[a:b]
        realv = np.sort(pv[pv != 0xFFFFFFFF])
        if not np.array_equal(realv, np.arange(ln, dtype=np.uint32)):
            return _fail(f"segment {s} payload not a permutation of its real elements")
    return None


ALL_CHECKS = [
    check_sorted_like_numpy,
    check_payload_permutation,
    check_zero_one_principle,
    check_recursive_agrees,
    check_hand_traces,
    check_all_equal_identity,
    check_desc_mirror,
    check_f32_total_order,
    check_segmented,
]


def run_all(mutant=0, fast=False):
    """Return the list of (check name, message) that failed."""
    failures = []
    for chk in ALL_CHECKS:
        if fast and chk is check_zero_one_principle:
            msg = chk(mutant=mutant, max_n=8)
        else:
            msg = chk(mutant=mutant)
        if msg is not None:
            failures.append((chk.__name__, msg))
    return failures

