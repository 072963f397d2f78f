"""Bounds and network checks of every whole-array plan, on the CPU.

The planner's launch lists (darm_plan_dump, no device needed) are replayed
through the kernels' index arithmetic (tests/plan_emulator.py): each round
must touch every element exactly once, stay inside the array and inside the
launch's shared memory, pair registers whose elements differ in one index
bit, and the whole plan must run Fig. 1's layers in Fig. 1's order.  This
stands in for a bounds-checking tool on the GPU."""
import numpy as np
import pytest

import paper_2107_05681_gb300 as darm
from tests import plan_emulator as em

KINDS = [(darm.U32, 4, False), (darm.U32, 4, True), (darm.F32, 4, False), (darm.U64, 8, False),
         (darm.U64, 8, True)]


@pytest.mark.parametrize("dtype,kb,hv", KINDS)
def test_default_plans_every_size_enumerated(dtype, kb, hv):
    for m in range(1, 18):
        n = 1 << m
        for variant in ("melded", "divergent"):
            plan = darm.plan_dump(dtype, n, hv, variant)
            em.check_plan(plan, n, kb, hv, full=True)


@pytest.mark.parametrize("dtype,kb,hv,m", [(darm.U32, 4, True, 24), (darm.F32, 4, False, 26),
                                           (darm.U32, 4, False, 28), (darm.U64, 8, True, 24),
                                           (darm.U32, 4, True, 31)])
def test_full_size_plans_bit_linear(dtype, kb, hv, m):
    """The benchmark's workloads (2^24 key-value pairs, 2^26 float keys) and
    the largest arrays the library accepts."""
    plan = darm.plan_dump(dtype, 1 << m, hv, "melded")
    em.check_plan(plan, 1 << m, kb, hv, full=False, rng=np.random.default_rng(m))


def _tuner_candidates(hv):
    base_t, base_e1 = (13, 4) if hv else (14, 5)
    for t in (base_t - 1, base_t, base_t + 1):
        for e1 in (base_e1 - 1, base_e1):
            for e2 in (3, 4, 5):
                for w2 in (1, 2):
                    for tma in (0, 1, 2, 3, 4):
                        for shfl in (0, 1, 3):
                            for tm in (0, t - 1):
                                yield (t, e1, e2, 8, w2, tma, shfl, tm)


@pytest.mark.parametrize("hv", [False, True])
@pytest.mark.parametrize("part", range(4))
def test_tuner_candidate_plans(hv, part):
    """Tunings the whole-array autotuner tries (and the shuffle-stage tile
    pass on and off, merges on the tile pass's tile or half of it) on an
    array of 2^16 elements: one candidate in 64 per case, the choice rotating
    through every block of 64 candidates so that over the four cases each
    tuning field takes all its values."""
    n = 1 << 16
    checked = 0
    for i, tn in enumerate(_tuner_candidates(hv)):
        if i % 64 != part * 16 + (i // 64) % 16:
            continue
        try:
            plan = darm.plan_dump(darm.U32, n, hv, "melded", tuning=tn)
        except darm.DarmError:
            continue  # no valid plan for this tuning: the tuner skips it too
        em.check_plan(plan, n, 4, hv, full=True)
        checked += 1
    assert checked >= 8


def test_plans_of_each_kernel_kind_are_covered():
    kinds = set()
    for dtype, kb, hv in KINDS:
        for m in (12, 16, 18, 24, 26):
            for L in darm.plan_dump(dtype, 1 << m, hv, "melded"):
                kinds.add(em.Kernel(L, kb, hv).kind)
    mshfl = False
    for tn in ((14, 5, 5, 8, 1, 0, 0), (13, 5, 4, 8, 2, 0, 0), (14, 5, 5, 8, 2, 2, 3)):
        for L in darm.plan_dump(darm.U32, 1 << 18, False, "melded", tuning=tn):
            kinds.add(em.Kernel(L, 4, False).kind)
            mshfl = mshfl or bool(L["mshfl"])
    assert {"tile_shfl", "tile_fixed", "tma_merge", "swz_merge", "window1", "window2"} <= kinds, kinds
    assert mshfl, "no plan with the two-round shuffle merge"


@pytest.mark.parametrize("mutation", ["cnt", "a", "w0", "grid", "p"])
def test_a_planted_off_by_one_is_caught(mutation):
    """An off-by-one planted in a plan (one field of one launch) fails the
    replay."""
    n = 1 << 16
    plan = darm.plan_dump(darm.U32, n, True, "melded")
    em.check_plan(plan, n, 4, True, full=True)
    bad = [dict(L, rounds=[dict(R) for R in L["rounds"]]) for L in plan]
    win = next(L for L in bad if L["kind"] == em.WINDOW)
    merge = next(L for L in bad if L["kind"] == em.MERGE)
    if mutation == "cnt":
        merge["rounds"][-1]["cnt"] -= 1
    elif mutation == "a":
        merge["rounds"][1]["a"] += 1
    elif mutation == "w0":
        win["w0"] += 1
    elif mutation == "grid":
        win["grid"] -= 1
    else:
        merge["rounds"][0]["p"] -= 1
    with pytest.raises(AssertionError):
        em.check_plan(bad, n, 4, True, full=True)


@pytest.mark.parametrize("t", [13, 14])
@pytest.mark.parametrize("mutation", ["none", "no_xor_round1", "row_bits_round2", "rounds"])
def test_swizzled_merge_replay(t, mutation, monkeypatch):
    """The swizzled in-place merge (keys only, tiles of 2^13 and 2^14): the
    replay checks that the kernel's word offsets are the 128-byte swizzle of
    the element each register holds in all three rounds; a planted mistake
    in those offsets or in the plan's rounds fails it."""
    n = 1 << 18
    plan = darm.plan_dump(darm.U32, n, False, "melded", tuning=(t, 5, 5, 8, 2, 3, 1))
    assert any(L["tma"] == 3 for L in plan), "no swizzled merge planned"
    if mutation == "none":
        em.check_plan(plan, n, 4, False, full=True)
        return
    if mutation == "rounds":
        plan = [dict(L, rounds=[dict(R) for R in L["rounds"]]) for L in plan]
        merge = next(L for L in plan if L["tma"] == 3)
        merge["rounds"][0]["cnt"] -= 1
        merge["rounds"][1]["cnt"] += 1
        merge["rounds"][1]["a"] += 1
    else:
        good = em.swz_kernel_word

        def bad(tid, r, rd, logt):
            w = good(tid, r, rd, logt)
            if mutation == "no_xor_round1" and rd == 1:
                return ((tid >> 5) << 10) + (r << 5) + (tid & 31)
            if mutation == "row_bits_round2" and rd == 2:
                return (tid << 5) + (((r >> 2) ^ ((tid >> 1) & 7)) << 2) + (r & 3)
            return w
        monkeypatch.setattr(em, "swz_kernel_word", bad)
    with pytest.raises(AssertionError):
        em.check_plan(plan, n, 4, False, full=True)


@pytest.mark.parametrize("hv", [False, True])
@pytest.mark.parametrize("mutation", ["none", "roles", "box_stride", "no_swap_in_kernel"])
def test_tma_two_window_replay(mutation, hv, monkeypatch):
    """The TMA two-window pass (keys alone, or pairs): the two-window launch
    of the 2^24-element plan with both windows full (the one that runs the
    pair-swapped lowest layer)
    replayed in full on eight of its blocks, the whole plan on single bits
    and samples.  The tensor box's geometry must give every
    element's global index, and the pair-swapped register order of round 1
    must keep the minimum on the register that holds the lower index;
    planted mistakes in either fail the replay."""
    n = 1 << 24
    plan = darm.plan_dump(darm.U32, n, hv, "melded")
    w2t = [L for L in plan if L["win2"] == 2 and L["rounds"][1]["cnt"] == L["loge"]]
    assert w2t, "no ten-layer TMA two-window pass"
    w2t = w2t[:1]
    if mutation == "roles":
        monkeypatch.setattr(em, "w2t_keeps_min_first", lambda tid: np.ones_like(tid, dtype=bool))
    elif mutation == "box_stride":
        good = em.tma_box_global

        def bad(L, blk, l):
            # top-window stride off by 2^w0
            return good(L, blk, l) + ((l >> (4 + L["loge"])) & 1) * (1 << L["w0"])
        monkeypatch.setattr(em, "tma_box_global", bad)
    elif mutation == "no_swap_in_kernel":
        # the kernel's register order without the swap, the roles unchanged
        orig = em.Kernel.local

        def local(self, tid, r, a, rd=None):
            return orig(self, tid, r, a, None)
        monkeypatch.setattr(em.Kernel, "local", local)

    def replay():
        for L in w2t:
            seq = []
            nb = L["nblocks"]
            some = sorted({0, 1, nb - 1} | set(np.random.default_rng(7).integers(0, nb, 5).tolist()))
            em.check_launch_full(em.Kernel(L, 4, hv), n, seq, blocks=some)
            p = L["rounds"][0]["p"]
            top = L["w0"] + 2 * L["loge"] - 1
            assert seq == [(p, q) for q in range(top, top - len(seq), -1)], seq

    if mutation == "none":
        replay()
        em.check_plan(plan, n, 4, hv, full=False, rng=np.random.default_rng(24))
        return
    with pytest.raises(AssertionError):
        replay()


@pytest.mark.parametrize("t", [12, 13])
@pytest.mark.parametrize("mutation", ["none", "roles", "bit4_no_swap", "bit0_chunks"])
def test_key_value_swizzled_merge_replay(t, mutation, monkeypatch):
    """The key-value in-place merge (16 pairs per thread, tiles of 2^12 and
    2^13 pairs): its word offsets are the 128-byte swizzle of the pair each
    register holds in every round, the window at bit 4 pair-swapped in
    lanes 16..31 with the roles of the lowest layer exchanged there; planted
    mistakes in the offsets or the roles fail the replay."""
    n = 1 << 17
    plan = darm.plan_dump(darm.U32, n, True, "melded", tuning=(t, 4, 4, 8, 2, 3, 1))
    assert any(L["tma"] == 3 for L in plan if L["kind"] == em.MERGE)
    if mutation == "roles":
        monkeypatch.setattr(em, "swz_kv_first_is_lower", lambda tid: np.ones_like(tid, dtype=bool))
    elif mutation in ("bit4_no_swap", "bit0_chunks"):
        good = em.swz_kv_kernel_word

        def bad(tid, r, a):
            if mutation == "bit4_no_swap" and a == 4:
                tl = (tid & 15) | ((tid >> 4) << 8)
                return ((tl | ((r & 1) << 4)) ^ (((r >> 1) & 7) << 2)) + ((r >> 1) << 5)
            if mutation == "bit0_chunks" and a == 0:
                return ((tid >> 1) << 5) + (((((tid & 1) << 2) | (r >> 2)) ^ (tid & 7)) << 2) + (r & 3)
            return good(tid, r, a)
        monkeypatch.setattr(em, "swz_kv_kernel_word", bad)
    if mutation == "none":
        em.check_plan(plan, n, 4, True, full=True)
        return
    with pytest.raises(AssertionError):
        em.check_plan(plan, n, 4, True, full=True)
