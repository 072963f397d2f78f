"""Oracle for the melding analysis (Section IV-C): TEST INFRASTRUCTURE ONLY
(the tests use it; the library never does).  Plain Python restatements of
the paper's definitions, written independently of the C ABI tool:

* mp_block(b1, b2): MP_B = sum over opcodes of min(freq in b1, freq in b2)
  x latency, over lat(b1) + lat(b2);
* mp_subgraph(S1, S2): MP_S = latency-weighted mean of MP_B over the
  corresponding block pairs;
* best_local_alignment_score(a, b, gap): the optimal local alignment score
  by brute force over every chain of compatible pairs (i1 < i2 < ...,
  j1 < j2 < ...): sum of the aligned instructions' latencies minus `gap`
  for each unaligned instruction between the chain's first and last pair,
  or 0 for the empty alignment.  Exponential: small blocks only.

An instruction is (opcode, type, latency); two instructions are compatible
(can be aligned) when opcode and type are equal.

Subgraphs (Def. 3, Def. 6, Def. 7) are (blocks, shape, simple_region):
blocks in pre-order, `shape` naming the structure (two multi-block subgraphs
are isomorphic when their shapes and block counts agree):

* sese_profit(s1, s2): Def. 6's three cases - isomorphic multi-block
  subgraphs: MP_S of corresponding blocks; two single blocks: MP_B; a single
  block A and a simple region M: the region replicated around A, A beside
  its most profitable partner E and every other replicated block empty, so
  MP_S = MP_B(A, E) (lat(A) + lat(E)) / (lat(A) + lat(M)); anything else is
  not meldable (None);
* best_subgraph_alignment_score(t, f, gap): the optimal subgraph alignment
  by brute force over every chain of meldable pairs, scored like the
  instruction alignment with MP as the pair score.
"""
from __future__ import annotations

from collections import Counter


def lat(block) -> int:
    return sum(i[2] for i in block)


def mp_block(b1, b2) -> float:
    w = {}
    for op, _, latency in list(b1) + list(b2):
        w.setdefault(op, latency)
    f1 = Counter(i[0] for i in b1)
    f2 = Counter(i[0] for i in b2)
    total = lat(b1) + lat(b2)
    if total == 0:
        return 0.0
    return sum(min(f1[op], f2[op]) * w[op] for op in f1 if op in f2) / total


def mp_subgraph(s1, s2) -> float:
    num = sum(mp_block(b1, b2) * (lat(b1) + lat(b2)) for b1, b2 in zip(s1, s2))
    den = sum(lat(b1) + lat(b2) for b1, b2 in zip(s1, s2))
    return num / den if den else 0.0


def compatible(x, y) -> bool:
    return x[0] == y[0] and x[1] == y[1]


def best_local_alignment_score(a, b, gap: float) -> float:
    pairs = [(i, j) for i in range(len(a)) for j in range(len(b)) if compatible(a[i], b[j])]
    best = 0.0

    def extend(chain, start):
        nonlocal best
        if chain:
            (i0, j0), (i1, j1) = chain[0], chain[-1]
            matched = sum(a[i][2] for i, _ in chain)
            unaligned = (i1 - i0 + 1 - len(chain)) + (j1 - j0 + 1 - len(chain))
            best = max(best, matched - gap * unaligned)
        for k in range(start, len(pairs)):
            i, j = pairs[k]
            if not chain or (i > chain[-1][0] and j > chain[-1][1]):
                extend(chain + [(i, j)], k + 1)

    extend([], 0)
    return best


def sese_profit(s1, s2):
    b1, shape1, simple1 = s1
    b2, shape2, simple2 = s2
    if len(b1) == 1 and len(b2) == 1:
        return mp_block(b1[0], b2[0])
    if len(b1) > 1 and len(b2) > 1:
        if len(b1) != len(b2) or shape1 != shape2:
            return None
        return mp_subgraph(b1, b2)
    # a single block beside a region: replicate the region around it
    (single, _, _), (region, _, simple) = (s1, s2) if len(b1) == 1 else (s2, s1)
    if not simple:
        return None
    a = single[0]
    # the region's block with the highest MP_B; the first one on ties
    k_best = max(range(len(region)), key=lambda k: (mp_block(a, region[k]), -k))
    replica = [[] for _ in region]
    replica[k_best] = a
    return mp_subgraph(replica, region)


def best_subgraph_alignment_score(t, f, gap: float) -> float:
    cand = []
    for i in range(len(t)):
        for j in range(len(f)):
            mp = sese_profit(t[i], f[j])
            if mp is not None:
                cand.append((i, j, mp))
    best = 0.0

    def extend(chain, start):
        nonlocal best
        if chain:
            (i0, j0, _), (i1, j1, _) = chain[0], chain[-1]
            unaligned = (i1 - i0 + 1 - len(chain)) + (j1 - j0 + 1 - len(chain))
            best = max(best, sum(c[2] for c in chain) - gap * unaligned)
        for k in range(start, len(cand)):
            i, j, _ = cand[k]
            if not chain or (i > chain[-1][0] and j > chain[-1][1]):
                extend(chain + [cand[k]], k + 1)

    extend([], 0)
    return best
