"""The melding analysis through the C ABI (host only, no GPU) against the
paper's statements and a plain oracle (oracle/meld_oracle.py)."""
import os

import numpy as np
import pytest

from oracle import meld_oracle as mo

HERE = os.path.dirname(os.path.abspath(__file__))
THRESHOLD = 0.2  # the paper's default melding profitability threshold


def _rand_block(rng, n, nop=4, ntype=2):
    lat = {op: int(rng.integers(1, 6)) for op in range(nop)}
    out = []
    for _ in range(n):
        op = int(rng.integers(0, nop))
        out.append((op, int(rng.integers(0, ntype)), lat[op]))
    return out


def _bit_model():
    sides = {}
    for line in open(os.path.join(HERE, "golden", "bit_sides_instruction_model.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        side, block, op, ty, latency = line[0], line[1], int(line[2]), int(line[3]), int(line[4])
        sides.setdefault(side, {}).setdefault(block, []).append((op, ty, latency))
    return sides


def test_identical_profiles_give_one_half():
    """Section IV-C: two blocks with identical opcode profiles have MP_B 0.5."""
    import paper_2107_05681_gb300 as darm
    rng = np.random.default_rng(1)
    for n in (1, 3, 8, 20):
        b = _rand_block(rng, n)
        perm = [b[i] for i in rng.permutation(len(b))]  # order does not matter
        assert darm.meld_mp_block(b, perm) == pytest.approx(0.5)
        assert mo.mp_block(b, perm) == pytest.approx(0.5)


def test_disjoint_profiles_give_zero_and_bounds_hold():
    import paper_2107_05681_gb300 as darm
    assert darm.meld_mp_block([(1, 0, 3), (2, 0, 1)], [(3, 0, 2)]) == 0.0
    rng = np.random.default_rng(2)
    for _ in range(200):
        b1, b2 = _rand_block(rng, int(rng.integers(0, 9))), _rand_block(rng, int(rng.integers(0, 9)))
        lat = {}
        b1 = [(o, t, lat.setdefault(o, l)) for o, t, l in b1]
        b2 = [(o, t, lat.setdefault(o, l)) for o, t, l in b2]
        got = darm.meld_mp_block(b1, b2)
        assert 0.0 <= got <= 0.5 + 1e-12
        assert got == pytest.approx(darm.meld_mp_block(b2, b1))


def test_mp_block_and_subgraph_match_the_oracle():
    import paper_2107_05681_gb300 as darm
    rng = np.random.default_rng(3)
    for _ in range(300):
        nb = int(rng.integers(1, 4))
        s1 = [_rand_block(rng, int(rng.integers(1, 7))) for _ in range(nb)]
        s2 = [_rand_block(rng, int(rng.integers(1, 7))) for _ in range(nb)]
        # one latency per opcode across both subgraphs
        lat = {}
        s1 = [[(o, t, lat.setdefault(o, l)) for o, t, l in b] for b in s1]
        s2 = [[(o, t, lat.setdefault(o, l)) for o, t, l in b] for b in s2]
        assert darm.meld_mp_block(s1[0], s2[0]) == pytest.approx(mo.mp_block(s1[0], s2[0]))
        assert darm.meld_mp_subgraph(s1, s2) == pytest.approx(mo.mp_subgraph(s1, s2))
        if nb == 1:
            assert darm.meld_mp_subgraph(s1, s2) == pytest.approx(darm.meld_mp_block(s1[0], s2[0]))


def test_inconsistent_latencies_are_rejected():
    import paper_2107_05681_gb300 as darm
    assert np.isnan(darm.meld_mp_block([(1, 0, 3)], [(1, 0, 4)]))


@pytest.mark.parametrize("gap", [0.0, 0.5, 1.0, 3.0])
def test_alignment_is_optimal_and_valid(gap):
    """Smith-Waterman score equals the brute-force optimum over every chain of
    compatible pairs; the returned alignment covers both sequences once, in
    order, aligns only compatible instructions and achieves the score."""
    import paper_2107_05681_gb300 as darm
    rng = np.random.default_rng(int(gap * 10) + 4)
    for _ in range(150):
        a = _rand_block(rng, int(rng.integers(0, 7)), nop=3)
        b = _rand_block(rng, int(rng.integers(0, 7)), nop=3)
        lat = {}
        a = [(o, t, lat.setdefault(o, l)) for o, t, l in a]
        b = [(o, t, lat.setdefault(o, l)) for o, t, l in b]
        pairs, score = darm.meld_align(a, b, gap)
        assert score == pytest.approx(mo.best_local_alignment_score(a, b, gap))
        assert [i for i, _ in pairs if i is not None] == list(range(len(a)))
        assert [j for _, j in pairs if j is not None] == list(range(len(b)))
        chain = [(i, j) for i, j in pairs if i is not None and j is not None]
        assert all(mo.compatible(a[i], b[j]) for i, j in chain)
        if chain:
            (i0, j0), (i1, j1) = chain[0], chain[-1]
            un = (i1 - i0 + 1 - len(chain)) + (j1 - j0 + 1 - len(chain))
            assert sum(a[i][2] for i, _ in chain) - gap * un == pytest.approx(score)


def test_bit_sides_align_except_the_compares():
    """Section IV-G: aligning the corresponding blocks of the two sides of
    Fig. 1 leaves only the compare instructions unaligned, and the pair is
    worth melding at the default threshold.  Gap penalty 0.25 per unaligned
    instruction (a quarter of the cheapest latency): with a penalty of half
    the branch's latency or more, the local alignment would rather stop
    before the compares and leave the branch after them unaligned too."""
    import paper_2107_05681_gb300 as darm
    m = _bit_model()
    asc, desc = m["asc"], m["desc"]
    unaligned = []
    for blk in ("C", "E", "X"):
        pairs, _ = darm.meld_align(asc[blk], desc[blk], gap=0.25)
        for i, j in pairs:
            if i is None or j is None:
                unaligned.append((blk, "asc" if j is None else "desc",
                                  (asc[blk][i] if j is None else desc[blk][j])[0]))
    icmp = 3
    assert sorted(unaligned) == [("C", "asc", icmp), ("C", "desc", icmp)]
    blocks = ("C", "E", "X")
    mps = darm.meld_mp_subgraph([asc[b] for b in blocks], [desc[b] for b in blocks])
    # every opcode is shared (both compares are icmp): identical profiles
    assert mps == pytest.approx(0.5)
    assert mps >= THRESHOLD


# ---- subgraph alignment (Def. 6, Def. 7) and the meld decision (Algorithm 1)

def _rand_subgraph(rng, lat, shapes=2):
    nb = int(rng.choice([1, 1, 2, 3]))
    blocks = []
    for _ in range(nb):
        b = _rand_block(rng, int(rng.integers(1, 5)), nop=4)
        blocks.append([(o, t, lat.setdefault(o, l)) for o, t, l in b])
    return (blocks, int(rng.integers(0, shapes)), bool(rng.integers(0, 2)))


def test_sese_profit_cases_by_hand():
    import paper_2107_05681_gb300 as darm
    a = [(1, 0, 2)]
    region = [[(1, 0, 2)], [(2, 0, 3)], [(1, 0, 2), (2, 0, 3)]]
    # case 2: A beside its best partner (block 0, MP_B 2/4 = 0.5) in a
    # replica of the 3-block region whose other blocks are empty:
    # 0.5 * (2 + 2) / (2 + 10)
    got = darm.meld_mp_sese((region, 7, True), ([a], 0, False))
    assert got == pytest.approx(0.5 * 4 / 12)
    assert mo.sese_profit(([a], 0, False), (region, 7, True)) == pytest.approx(0.5 * 4 / 12)
    # a block against a region that is not simple cannot be replicated
    assert darm.meld_mp_sese(([a], 0, True), (region, 7, False)) == -1.0
    # multi-block subgraphs must be isomorphic
    assert darm.meld_mp_sese((region, 7, True), (region, 8, True)) == -1.0
    assert darm.meld_mp_sese((region, 7, True), (region[:2], 7, True)) == -1.0
    assert darm.meld_mp_sese((region, 7, True), (region, 7, False)) == pytest.approx(0.5)
    # case 3: two single blocks is MP_B
    assert darm.meld_mp_sese(([a], 0, False), ([region[2]], 0, False)) == pytest.approx(2 / 7)


def test_sese_profit_matches_the_oracle():
    import paper_2107_05681_gb300 as darm
    rng = np.random.default_rng(11)
    for _ in range(400):
        lat = {}
        s1, s2 = _rand_subgraph(rng, lat), _rand_subgraph(rng, lat)
        want = mo.sese_profit(s1, s2)
        got = darm.meld_mp_sese(s1, s2)
        if want is None:
            assert got == -1.0
        else:
            assert got == pytest.approx(want)


@pytest.mark.parametrize("gap", [0.0, 0.05, 0.2, 1.0])
def test_subgraph_alignment_is_optimal_and_valid(gap):
    """Smith-Waterman over the two paths' subgraph sequences reaches the
    brute-force optimum over every chain of meldable pairs; the returned
    pairs are meldable, in order, achieve the score, and are melded exactly
    when their profitability reaches the threshold."""
    import paper_2107_05681_gb300 as darm
    rng = np.random.default_rng(int(gap * 100) + 12)
    for _ in range(120):
        lat = {}
        t = [_rand_subgraph(rng, lat) for _ in range(int(rng.integers(0, 5)))]
        f = [_rand_subgraph(rng, lat) for _ in range(int(rng.integers(0, 5)))]
        if not t and not f:
            continue
        thr = float(rng.choice([0.0, 0.1, THRESHOLD, 0.3]))
        pairs, score = darm.meld_subgraph_align(t, f, gap=gap, threshold=thr)
        assert score == pytest.approx(mo.best_subgraph_alignment_score(t, f, gap))
        prev = (-1, -1)
        for i, j, profit, meld in pairs:
            assert i > prev[0] and j > prev[1]
            prev = (i, j)
            want = mo.sese_profit(t[i], f[j])
            assert want is not None and profit == pytest.approx(want)
            assert meld == (profit >= thr)
        if pairs:
            (i0, j0, _, _), (i1, j1, _, _) = pairs[0], pairs[-1]
            un = (i1 - i0 + 1 - len(pairs)) + (j1 - j0 + 1 - len(pairs))
            assert sum(p[2] for p in pairs) - gap * un == pytest.approx(score)


def test_identical_paths_align_on_the_diagonal():
    """Two paths with the same subgraphs: every subgraph pairs with its
    counterpart at profitability 0.5 (identical profiles) and is melded."""
    import paper_2107_05681_gb300 as darm
    rng = np.random.default_rng(13)
    lat = {}
    path = [_rand_subgraph(rng, lat) for _ in range(5)]
    pairs, score = darm.meld_subgraph_align(path, path, gap=0.1)
    assert [(i, j) for i, j, _, _ in pairs] == [(k, k) for k in range(5)]
    assert all(p == pytest.approx(0.5) and m for _, _, p, m in pairs)
    assert score == pytest.approx(2.5)


def test_threshold_is_inclusive():
    """Algorithm 1 melds a pair whose profitability is at least the
    threshold: MP_B = 2 / (5 + 5) = 0.2 exactly."""
    import paper_2107_05681_gb300 as darm
    b1 = [(1, 0, 2), (2, 0, 3)]
    b2 = [(1, 0, 2), (3, 0, 3)]
    pairs, _ = darm.meld_subgraph_align([([b1], 0, False)], [([b2], 0, False)])
    assert len(pairs) == 1 and pairs[0][2] == pytest.approx(0.2) and pairs[0][3]
    pairs, _ = darm.meld_subgraph_align([([b1], 0, False)], [([b2], 0, False)],
                                        threshold=0.2000001)
    assert len(pairs) == 1 and not pairs[0][3]


def test_bit_region_is_aligned_and_melded():
    """Section IV-G: in Fig. 1's divergent region the two sides' subgraphs
    (condition block, swap block, exit; isomorphic simple regions) are
    profitable to meld: one aligned pair, melded at the default threshold."""
    import paper_2107_05681_gb300 as darm
    m = _bit_model()
    t = [([m["asc"][b] for b in ("C", "E", "X")], 1, True)]
    f = [([m["desc"][b] for b in ("C", "E", "X")], 1, True)]
    pairs, score = darm.meld_subgraph_align(t, f)
    assert len(pairs) == 1
    i, j, profit, meld = pairs[0]
    assert (i, j) == (0, 0) and profit == pytest.approx(0.5) and meld
    assert score == pytest.approx(0.5)
