"""Host replay of the index arithmetic every pass kernel applies to a plan.

The library's planner turns a sort into launches (darm_plan_dump); each
launch's kernel maps (block, thread, register) of every round to an element
of the array (its HBM address) and, between rounds, to a shared-memory slot.
This module restates those maps from the kernels' sources, in numpy, so that
a CPU test can check every plan without a GPU:

* every round touches each element of the array exactly once (the map is a
  bijection onto [0, n)), HBM addresses stay below n and shared-memory slots
  below the launch's allocation, distinct within a block;
* the layers a round runs pair register r with r | 2^q, and those registers
  hold elements whose indices differ in exactly one bit; the sequence of
  (stage, layer bit) over the whole plan is Fig. 1's: k = 2, 4, ..., n and
  j = k/2, ..., 1, each once, in order.

Small arrays are enumerated in full.  For large ones the maps are checked to
be bit-linear (an OR of disjoint shifted bit fields, which every map here is
by construction) on the images of single bits and on random samples, and the
single-bit images must be distinct bits covering [0, m): that is the same
bijection property without materialising 2^26 indices.
"""
from __future__ import annotations

import numpy as np

TILE, WINDOW, MERGE = 0, 1, 2
RK_PHASE_A, RK_WINDOW = 0, 1
LOC_GLOBAL, LOC_SMEM = 0, 1


def phys(l):
    """Four pad words after every 32 elements (pass_kernel.cuh phys)."""
    return l + ((l >> 5) << 2)


def phys8(l):
    """Two pad slots after every 16 key-value pairs."""
    return l + ((l >> 4) << 1)


def physp(l, pad):
    return l + (l >> 5) * pad


def swz128(l):
    """Word of element l in a tile buffer written by a TMA copy with the
    128-byte swizzle: 16-byte chunk c of 128-byte row w holds chunk c ^ (w & 7)."""
    return l ^ (((l >> 5) & 7) << 2)


def swz_kernel_word(tid, r, rd, logt):
    """The word offsets the swizzled in-place merge kernel computes
    (tma_merge_swz.cuh) for register r of thread tid in round rd."""
    if rd == 0:
        return (tid ^ (((tid >> 5) & 7) << 2)) + (r << (logt - 5))
    if rd == 1:
        return ((tid >> 5) << 10) + (r << 5) + ((tid & 31) ^ ((r & 7) << 2))
    return (tid << 5) + ((((r >> 2) ^ (tid & 7)) << 2) | (r & 3))


def tma_box_global(L, blk, l):
    """Global index of element l of block blk of a TMA two-window pass with
    windows of e bits: the tensor map's coordinates (16 consecutive
    elements, the w0 - 4 bits between them and the windows, bottom window,
    top window, the bits above) with the strides the host encodes (1, 16,
    2^w0, 2^(w0+e), 2^(w0+2e) elements)."""
    w0, e = L["w0"], L["loge"]
    nmid = w0 - 4
    mid = blk & ((1 << nmid) - 1)
    high = blk >> nmid
    d0, bw, tw = l & 15, (l >> 4) & ((1 << e) - 1), l >> (4 + e)
    return d0 + 16 * mid + (bw << w0) + (tw << (w0 + e)) + (high << (w0 + 2 * e))


def w2t_keeps_min_first(tid):
    """Round 1's lowest layer in the TMA two-window kernel: register r of a
    pair (r, r+1) takes the minimum (ascending) in lanes 0..15 and the
    maximum in lanes 16..31 (keep_lo_first = asc != tw0)."""
    return ((tid >> 4) & 1) == 0


def swz_kv_kernel_word(tid, r, a):
    """The word offsets the key-value in-place merge kernel computes
    (tma_merge_swz.cuh) for register r of thread tid in the round whose
    window sits at bit a (keys and payloads alike)."""
    if a >= 8:
        tl = (tid & ((1 << a) - 1)) | ((tid >> a) << (a + 4))
        return (tl ^ (((tl >> 5) & 7) << 2)) + (r << a)
    if a == 4:
        tl = (tid & 15) | ((tid >> 4) << 8)
        flip = (tid >> 4) & 1
        base = tl | (((r & 1) ^ flip) << 4)
        return (base ^ (((r >> 1) & 7) << 2)) + ((r >> 1) << 5)
    assert a == 0
    c = ((((tid & 1) << 2) | (r >> 2)) ^ ((tid >> 1) & 7)) << 2
    return ((tid >> 1) << 5) + c + (r & 3)


def swz_kv_first_is_lower(tid):
    """The key-value merge's lowest layer of the window at bit 4: register r
    of a pair (r, r+1) holds the lower index in lanes 0..15 (the kernel's
    `flip` is lane >> 4)."""
    return ((tid & 31) >> 4) == 0


def check_swz_kv_merge(K):
    L = K.L
    b = L["b"]
    assert K.loge == 4 and b in (12, 13) and K.hv and K.kb == 4, "key-value swizzled merge shape"
    assert L["threads"] == 1 << (b - 4)
    exp = []
    for i in range((b + 3) // 4 - 1, -1, -1):
        hi = min((i + 1) * 4, b) - 1
        exp.append((hi - 3, hi - i * 4 + 1))
    got = [(R["a"], R["cnt"]) for R in L["rounds"]]
    assert got == exp, ("key-value swizzled merge rounds", got, exp)
    tid = np.arange(L["threads"], dtype=np.int64)[:, None]
    r = np.arange(16, dtype=np.int64)[None, :]
    saved, K.pair_swap = K.pair_swap, True  # the kernel's own register order
    try:
        for rd, (a, _) in enumerate(got):
            l = K.local(tid, r, a, rd)
            w = swz_kv_kernel_word(tid, r, a)
            assert np.array_equal(w, swz128(l)), ("key-value swizzled word offsets", rd)
            assert w.min() >= 0 and w.max() < (1 << b) and np.unique(w).size == w.size
    finally:
        K.pair_swap = saved


def check_swz_merge(K):
    """The swizzled merge runs a fixed schedule: it must be the plan's, and
    the kernel's own word offsets must be the swizzled slot of the element
    the register holds, in every round (the rounds work in place)."""
    if K.hv:
        check_swz_kv_merge(K)
        return
    L = K.L
    b = L["b"]
    assert K.loge == 5 and b in (13, 14) and not K.hv and K.kb == 4, "swizzled merge shape"
    assert L["threads"] == 1 << (b - 5)
    got = [(R["a"], R["cnt"]) for R in L["rounds"]]
    assert got == [(b - 5, b - 10), (5, 5), (0, 5)], ("swizzled merge rounds", got)
    tid = np.arange(L["threads"], dtype=np.int64)[:, None]
    r = np.arange(32, dtype=np.int64)[None, :]
    for rd in range(3):
        l = K.local(tid, r, K.window_of(rd))
        w = swz_kernel_word(tid, r, rd, b)
        assert np.array_equal(w, swz128(l)), ("swizzled merge word offsets", rd)
        assert w.min() >= 0 and w.max() < (1 << b) and np.unique(w).size == w.size


def smem_words(elems):
    return elems + ((elems >> 5) << 2) + 4


class Kernel:
    """Index maps of one launch: global(blk, tid, r, rd) and smem(...)."""

    def __init__(self, L, key_bytes, has_vals):
        self.L = L
        self.E = 1 << L["loge"]
        self.loge = L["loge"]
        self.kb = key_bytes
        self.hv = has_vals
        self.interleave = has_vals and key_bytes == 4
        self.pair_swap = True  # round-1 / bit-4 register order in lanes 16..31 (TMA kernels)
        if L["win1"]:
            self.kind = "window1"
        elif L["win2"] == 2:
            self.kind = "window2_tma"
        elif L["win2"]:
            self.kind = "window2"
        elif L["tma"] in (3, 4):
            self.kind = "swz_merge"
        elif L["tma"]:
            self.kind = "tma_merge"
        elif L["shfl"]:
            self.kind = "tile_shfl"
        elif L["fixed"]:
            self.kind = "tile_fixed"
        else:
            self.kind = "generic"

    # -- shared-memory layout of the kernel that runs this launch
    def pad_words(self):
        if self.kind in ("tile_fixed", "tile_shfl", "window2"):
            if not self.hv and self.kb == 4 and self.loge == 5:
                return 1
        return 4

    def slot(self, l):
        if self.kind == "swz_merge":
            return swz128(l)
        if self.kind == "window2_tma":
            return l  # the tensor box, dense in local-index order
        if self.interleave:
            return phys8(l)
        if self.kind in ("tile_fixed", "tile_shfl", "window2"):
            return physp(l, self.pad_words())
        return phys(l)

    def slot_bound(self):
        b = self.L["b"]
        if self.kind == "swz_merge":
            return 1 << b
        if self.kind == "window2_tma":
            return 1 << b
        if self.kind == "window2":
            b = self.L["c"] + 2 * self.loge
        return smem_words(1 << b)

    # -- the element a register holds: its index in the block (local) and in
    # the array (global)
    def local(self, tid, r, a, rd=None):
        tl = (tid & ((1 << a) - 1)) | ((tid >> a) << (a + self.loge))
        if self.kind == "window2_tma" and rd == 1 and self.pair_swap:
            # lanes 16..31 of a warp hold bottom-window position r ^ 1
            r = r ^ ((tid >> 4) & 1)
        if self.kind == "swz_merge" and self.hv and a == 4 and self.pair_swap:
            # key-value merge, window at bit 4: the same swap
            r = r ^ ((tid >> 4) & 1)
        return tl | (r << a)

    def gblk(self, blk):
        L = self.L
        if self.kind in ("tile_fixed", "tile_shfl", "tma_merge", "swz_merge"):
            return blk << L["b"]
        c, w0 = L["c"], L["w0"]
        nmid = w0 - c
        span = L["s"] if self.kind == "generic" else (
            self.loge if self.kind == "window1" else 2 * self.loge)  # window2, window2_tma
        return ((blk & ((1 << nmid) - 1)) << c) | ((blk >> nmid) << (w0 + span))

    def gmap(self, l):
        L = self.L
        if self.kind in ("tile_fixed", "tile_shfl", "tma_merge", "swz_merge"):
            return l
        c, w0 = L["c"], L["w0"]
        return (l & ((1 << c) - 1)) | ((l >> c) << w0)

    def window_of(self, rd):
        """Window bit a of round rd as the kernel computes it."""
        L = self.L
        if self.kind == "window1":
            return L["c"]
        if self.kind in ("window2", "window2_tma"):
            return L["c"] + self.loge if rd == 0 else L["c"]
        return L["rounds"][rd]["a"]

    def hbm_address(self, blk, tid, r, rd):
        """The address arithmetic the kernel uses on HBM in round rd."""
        L, E = self.L, self.E
        a = self.window_of(rd)
        gb = self.gblk(blk)
        if self.kind == "window1":
            return (tid | gb) + (r << L["w0"])
        if self.kind == "window2_tma":
            return tma_box_global(L, blk, self.local(tid, r, a, rd))
        if self.kind == "window2":
            tl = (tid & ((1 << a) - 1)) | ((tid >> a) << (a + self.loge))
            c = L["c"]
            g_t = (tl & ((1 << c) - 1)) | ((tl >> c) << L["w0"]) | gb
            sh = L["w0"] + (self.loge if rd == 0 else 0)
            return g_t + (r << sh)
        tl = (tid & ((1 << a) - 1)) | ((tid >> a) << (a + self.loge))
        if self.kind == "generic":
            c, w0 = L["c"], L["w0"]
            g_t = self.gmap(tl) | gb
            vec = a == 0 and c >= self.loge
            if vec:
                return g_t + r
            gsh = (a - c + w0) if a >= c else a
            return g_t + (r << gsh)
        return (tl | gb) + (r << a)

    def touches_hbm(self, rd):
        L = self.L
        nr = len(L["rounds"]) if self.kind not in ("window1", "window2") else (
            1 if self.kind == "window1" else 2)
        if self.kind == "window1":
            return True
        if self.kind in ("window2", "window2_tma"):
            return True
        R = L["rounds"][rd]
        last = rd + 1 == nr
        return R["src"] == LOC_GLOBAL or R["dst"] == LOC_GLOBAL or last

    def nrounds(self):
        if self.kind == "window1":
            return 1
        if self.kind in ("window2", "window2_tma"):
            return 2
        return len(self.L["rounds"])

    def round_layers(self, rd):
        """(stage p, register bits q of the layers, high to low)."""
        L, E = self.L, self.E
        if self.kind == "tma_merge" and L.get("mshfl") and rd == 1:
            # lane layers by shuffles, then the register layers: checked by
            # _check_layers on the consecutive layout
            return L["rounds"][0]["p"], []
        R = L["rounds"][rd] if self.kind not in ("window1",) else L["rounds"][0]
        if self.kind in ("window2", "window2_tma"):
            R = L["rounds"][rd]
        if self.kind in ("tma_merge", "swz_merge") or (self.kind == "tile_fixed" and L["kind"] == MERGE):
            p = L["rounds"][0]["p"]
        else:
            p = R["p"]
        cnt = E.bit_length() - 1 if (self.kind in ("window2", "window2_tma") and rd == 0) else R["cnt"]
        return p, [self.loge - 1 - i for i in range(cnt)]


def _grid_arrays(K):
    L = K.L
    blocks = L["nblocks"] if K.kind in ("tma_merge", "swz_merge", "window2_tma") else L["grid"]
    blk = np.arange(blocks, dtype=np.int64)[:, None, None]
    tid = np.arange(L["threads"], dtype=np.int64)[None, :, None]
    r = np.arange(K.E, dtype=np.int64)[None, None, :]
    return blk, tid, r


def check_launch_full(K, n, seq, blocks=None):
    """Enumerate every (block, thread, register) of every round.  `blocks`:
    only these blocks (their elements distinct and in range; the bijection
    onto [0, n) is then left to check_launch_linear)."""
    blk, tid, r = _grid_arrays(K)
    if blocks is not None:
        blk = np.asarray(blocks, dtype=np.int64)[:, None, None]
    if K.kind == "swz_merge":
        check_swz_merge(K)
    for rd in range(K.nrounds()):
        a = K.window_of(rd)
        l = K.local(tid, r, a, rd) + 0 * blk
        g = K.gmap(l) | K.gblk(blk)
        flat = g.reshape(-1)
        assert flat.min() >= 0 and flat.max() < n, (K.kind, rd, "element index out of range")
        if blocks is None:
            assert np.unique(flat).size == flat.size == n, (K.kind, rd, "not a bijection onto [0, n)")
        else:
            assert np.unique(flat).size == flat.size, (K.kind, rd, "an element taken twice")
        if K.touches_hbm(rd):
            h = K.hbm_address(blk, tid, r, rd) + 0 * g
            assert np.array_equal(h, g), (K.kind, rd, "HBM address differs from the element")
        if K.kind in ("tile_fixed", "tile_shfl", "tma_merge", "swz_merge", "window2", "window2_tma",
                      "generic") and (
                K.kind != "generic" or K.L["smem"] > 0) and K.kind != "window1":
            s = K.slot(l)
            assert s.min() >= 0 and s.max() < K.slot_bound(), (K.kind, rd, "slot out of range")
            for b in range(min(g.shape[0], 4)):
                assert np.unique(s[b]).size == s[b].size, (K.kind, rd, "slot reused in a block")
        _check_layers(K, rd, g, seq)


def _check_layers(K, rd, g, seq):
    p, qs = K.round_layers(rd)
    R = K.L["rounds"][rd] if K.kind != "window1" else K.L["rounds"][0]
    if K.kind == "tma_merge" and K.L.get("mshfl") and rd == 1:
        # E consecutive elements per thread, lane b holding index bit E + b:
        # the layers below the first window, lanes first, then registers
        E = K.E
        assert np.array_equal(g[..., 1:] - g[..., :-1], np.ones_like(g[..., 1:])), \
            "two-round merge: registers are not consecutive"
        top = R["a"] + R["cnt"]  # = the first window's lowest bit
        lanes = 1 << (top - K.loge)
        t = g[:, :lanes, 0]
        assert np.all(t - t[:, :1] == np.arange(lanes)[None, :] * E), \
            "two-round merge: lanes are not consecutive runs"
        for q in range(top - 1, -1, -1):
            seq.append((p, q))
        return
    if R["kind"] == RK_PHASE_A and K.kind != "window2":
        # registers hold E consecutive elements (and lanes the next bits when
        # stages run across lanes): stages 1 .. p with every layer
        E = K.E
        assert np.array_equal(g[..., 1:] - g[..., :-1], np.ones_like(g[..., 1:])), \
            "Phase A registers are not consecutive"
        if p > K.loge:
            lanes = 1 << (p - K.loge)
            t = g[:, :lanes, 0]
            assert np.all(t - t[:, :1] == np.arange(lanes)[None, :] * E), \
                "lanes of a shuffle stage are not consecutive runs"
        for pp in range(1, p + 1):
            for q in range(pp - 1, -1, -1):
                seq.append((pp, q))
        return
    for q in qs:
        lo = g[..., [r for r in range(K.E) if not (r >> q) & 1]]
        hi = g[..., [r | (1 << q) for r in range(K.E) if not (r >> q) & 1]]
        d = hi - lo
        if K.kind == "swz_merge" and K.hv and K.window_of(rd) == 4 and q == 0 and K.pair_swap:
            tid = np.arange(K.L["threads"], dtype=np.int64)[None, :, None]
            assert np.all((d > 0) == swz_kv_first_is_lower(tid)), \
                (K.kind, rd, "pair-swapped layer keeps min and max on the wrong registers")
            d = np.abs(d)
        if K.kind == "window2_tma" and rd == 1 and q == 0 and K.pair_swap:
            # the pair-swapped lanes hold the higher index first; the kernel
            # must give the minimum to whichever register holds the lower one
            tid = np.arange(K.L["threads"], dtype=np.int64)[None, :, None]
            first_is_lower = (d > 0)
            assert np.all(first_is_lower == w2t_keeps_min_first(tid)), \
                (K.kind, rd, "pair-swapped layer keeps min and max on the wrong registers")
            d = np.abs(d)
        bit = int(d.reshape(-1)[0])
        assert bit > 0 and bit & (bit - 1) == 0 and np.all(d == bit), \
            (K.kind, rd, "layer pairs do not differ in one bit")
        seq.append((p, bit.bit_length() - 1))


def expected_sequence(m):
    return [(p, q) for p in range(1, m + 1) for q in range(p - 1, -1, -1)]


def check_plan(plan, n, key_bytes, has_vals, full=True, rng=None):
    """Check every launch of `plan`; returns the (stage, layer) sequence."""
    seq = []
    for L in plan:
        K = Kernel(L, key_bytes, has_vals)
        if full:
            check_launch_full(K, n, seq)
        else:
            check_launch_linear(K, n, seq, rng or np.random.default_rng(0))
    m = n.bit_length() - 1
    assert seq == expected_sequence(m), "layer order differs from Fig. 1"
    return seq


def check_launch_linear(K, n, seq, rng):
    """Large arrays: the maps are ORs of shifted bit fields; check them on
    single bits and random samples instead of enumerating.  (The TMA
    two-window pass's register order within a thread, a relabelling that
    keeps every bound and bijection, is checked by the full replay.)"""
    L = K.L
    K.pair_swap = False
    blocks = L["nblocks"] if K.kind in ("tma_merge", "swz_merge", "window2_tma") else L["grid"]
    if K.kind == "swz_merge":
        check_swz_merge(K)
    nbits = [blocks.bit_length() - 1, L["threads"].bit_length() - 1, K.loge]
    assert (1 << nbits[0]) == blocks and (1 << nbits[1]) == L["threads"]
    m = n.bit_length() - 1
    for rd in range(K.nrounds()):
        a = K.window_of(rd)

        def G(blk, tid, r):
            return K.gmap(K.local(tid, r, a)) | K.gblk(blk)

        images = []
        for which, nb in enumerate(nbits):
            for bit in range(nb):
                args = [np.int64(0)] * 3
                args[which] = np.int64(1 << bit)
                images.append(int(G(*args)))
        assert int(G(np.int64(0), np.int64(0), np.int64(0))) == 0
        assert sorted(images) == [1 << i for i in range(m)], (K.kind, rd, "bits not a permutation")
        blk = rng.integers(0, blocks, 4096, dtype=np.int64)
        tid = rng.integers(0, L["threads"], 4096, dtype=np.int64)
        r = rng.integers(0, K.E, 4096, dtype=np.int64)
        g = G(blk, tid, r)
        lin = np.zeros_like(g)
        for which, nb in enumerate(nbits):
            src = (blk, tid, r)[which]
            off = sum(nbits[:which])
            for bit in range(nb):
                lin |= np.where((src >> bit) & 1, images[off + bit], 0)
        assert np.array_equal(g, lin), (K.kind, rd, "map is not bit-linear")
        if K.touches_hbm(rd):
            assert np.array_equal(K.hbm_address(blk, tid, r, rd), g), (K.kind, rd, "HBM address")
        if K.kind != "window1" and (K.kind != "generic" or L["smem"] > 0):
            tblk = np.zeros(1, dtype=np.int64)[:, None, None]
            tt = np.arange(L["threads"], dtype=np.int64)[None, :, None]
            rr = np.arange(K.E, dtype=np.int64)[None, None, :]
            s = K.slot(K.local(tt, rr, a) + 0 * tblk)
            assert s.max() < K.slot_bound() and np.unique(s).size == s.size, (K.kind, rd, "slots")
        # layers: on single-bit images
        p, qs = K.round_layers(rd)
        R = L["rounds"][rd] if K.kind != "window1" else L["rounds"][0]
        if K.kind == "tma_merge" and L.get("mshfl") and rd == 1:
            off = nbits[0] + nbits[1]
            top = R["a"] + R["cnt"]
            assert images[off:off + K.loge] == [1 << i for i in range(K.loge)]
            lane = images[nbits[0]:nbits[0] + (top - K.loge)]
            assert lane == [1 << (K.loge + i) for i in range(top - K.loge)]
            for q in range(top - 1, -1, -1):
                seq.append((p, q))
            continue
        if R["kind"] == RK_PHASE_A and K.kind != "window2":
            off = nbits[0] + nbits[1]
            assert images[off:off + K.loge] == [1 << i for i in range(K.loge)]
            if p > K.loge:
                lane = images[nbits[0]:nbits[0] + (p - K.loge)]
                assert lane == [1 << (K.loge + i) for i in range(p - K.loge)]
            for pp in range(1, p + 1):
                for q in range(pp - 1, -1, -1):
                    seq.append((pp, q))
            continue
        off = nbits[0] + nbits[1]
        for q in qs:
            seq.append((p, images[off + q].bit_length() - 1))
