"""GPU parity of the batched segmented sort against the oracle's segmented
sort (same sentinel padding, bit-exact keys and payloads)."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_equal, to_dev

pytestmark = pytest.mark.gpu


def _run(darm, segs, vals=True, variant="melded", desc=False, per_seg=True, repeat=1):
    import torch
    k = to_dev(segs.keys)
    v = to_dev(segs.vals) if vals else None
    dd = segs.desc if per_seg else None
    for _ in range(repeat):
        k.copy_(to_dev(segs.keys))
        if v is not None:
            v.copy_(to_dev(segs.vals))
        darm.segmented_sort(k, v, segs.offsets, segs.lengths, descending=desc,
                            variant=variant, seg_desc=dd)
    torch.cuda.synchronize()
    return k.cpu().numpy(), (v.cpu().numpy() if v is not None else None)


def _expect(segs, vals=True, desc=False, per_seg=True):
    return oracle.segmented_sort(segs.keys, segs.vals if vals else None, segs.offsets,
                                 segs.lengths, desc=desc,
                                 desc_per_seg=segs.desc if per_seg else None)


@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("vals", [False, True])
def test_mixed_sizes_and_directions(darm, variant, vals):
    # lengths 1..40000 (capacities 1 .. 65536, tiny, packed and multi-tile
    # segments), mixed directions, ragged real lengths
    segs = synth.cfg4_segments(seed=21, num_segments=300, min_len=1, max_len=40000,
                               mixed_dirs=True, largest_first=True)
    ek, ev = _expect(segs, vals)
    gk, gv = _run(darm, segs, vals, variant)
    assert_equal("keys", gk, ek)
    if vals:
        assert_equal("payload", gv, ev)
    assert darm.device_status() == darm.OK


def test_uniform_direction_argument(darm):
    segs = synth.cfg4_segments(seed=22, num_segments=64, min_len=16, max_len=20000)
    for desc in (False, True):
        ek, ev = _expect(segs, True, desc=desc, per_seg=False)
        gk, gv = _run(darm, segs, True, "melded", desc=desc, per_seg=False)
        assert_equal("keys", gk, ek)
        assert_equal("payload", gv, ev)


def test_graph_replay_same_layout(darm):
    """The second call with the same layout replays the captured graph and
    reads the current contents of the buffers."""
    segs = synth.cfg4_segments(seed=23, num_segments=120, min_len=32, max_len=30000)
    ek, ev = _expect(segs, True, per_seg=False)
    before = darm.launch_count()
    gk, gv = _run(darm, segs, True, "melded", per_seg=False, repeat=3)
    assert_equal("keys", gk, ek)
    assert_equal("payload", gv, ev)
    assert darm.launch_count() > before


def test_edge_segments(darm):
    """Empty segments (capacity 0), capacity 1 and 2, zero real length, full
    length, a two-tile segment; offsets aligned to min(capacity, 4)."""
    caps = [0, 4, 2, 2, 8, 0, 16, 1, 1, 2, 32, 4096, 1, 1, 2, 32768]
    lens = [0, 4, 1, 0, 5, 0, 16, 0, 1, 2, 0, 4000, 1, 0, 1, 30000]
    offs = np.zeros(len(caps) + 1, np.uint64)
    offs[1:] = np.cumsum(caps)
    total = int(offs[-1])
    keys = synth.uniform_u32(31, total) % np.uint32(50)
    vals = np.arange(total, dtype=np.uint32)
    for desc in (False, True):
        s = synth.Segments(keys, vals, offs, np.array(lens, np.uint32),
                           np.full(len(caps), int(desc), np.uint8))
        ek, ev = _expect(s, True)
        for variant in ("divergent", "melded"):
            gk, gv = _run(darm, s, True, variant)
            assert_equal("keys", gk, ek)
            assert_equal("payload", gv, ev)


@pytest.mark.parametrize("entry", ["segmented_sort", "segmented_sort_noalloc"])
@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("vals", [False, True])
def test_tile_blocks_wholly_in_padding(darm, entry, variant, vals):
    """Segments longer than the tile whose real length ends just past half the
    capacity, on a tile boundary (keys- and key-value tiles are 2^14 and 2^13
    elements), one past it, or at zero: their tile blocks beyond the length
    hold only sentinels and go to a launch of their own that writes the
    sentinel result without running the network, and the blocks of later
    stages' window and merge passes that lie in a 2^p block of padding are
    left out (lengths at 2^14 and 3 x 2^14 end exactly on such a block).
    The padding starts as zeros (payload 0x5A5A5A5A), which would sort first
    and surface in the result if such a block were not written; mixed
    directions."""
    caps = [65536, 65536, 65536, 65536, 65536, 32768, 32768, 32768, 16384, 16384, 65536,
            65536, 32768]
    lens = [32769, 40960, 49153, 0, 65536, 16385, 24576, 1, 8193, 16384, 57344, 49152, 16384]
    offs = np.zeros(len(caps) + 1, np.uint64)
    offs[1:] = np.cumsum(caps)
    total = int(offs[-1])
    # real keys in 1 .. 2^20: neither sentinel (0 descending, 2^32 - 1 ascending)
    keys = synth.uniform_u32(0x9AD5, total) % np.uint32(1 << 20) + np.uint32(1)
    vv = np.arange(total, dtype=np.uint32)
    for o, c, n in zip(offs[:-1], caps, lens):
        keys[int(o) + n:int(o) + c] = 0
        vv[int(o) + n:int(o) + c] = 0x5A5A5A5A
    desc = np.array([i % 2 for i in range(len(caps))], np.uint8)
    s = synth.Segments(keys, vv, offs, np.array(lens, np.uint32), desc)
    ek, ev = _expect(s, vals)
    darm.device_status()  # clear a status latched by an earlier call
    k = to_dev(keys)
    v = to_dev(vv) if vals else None
    getattr(darm, entry)(k, v, offs, s.lengths, variant=variant, seg_desc=desc)
    gk = k.cpu().numpy()
    assert_equal("keys", gk, ek)
    if vals:
        assert_equal("payload", v.cpu().numpy(), ev)
    assert darm.device_status() == darm.OK


def test_sentinel_collision_is_reported(darm):
    segs = synth.cfg4_segments(seed=24, num_segments=20, min_len=100, max_len=3000)
    keys = segs.keys.copy()
    keys[int(segs.offsets[3]) + 5] = np.uint32(0xFFFFFFFF)  # a real key equal to the sentinel
    s = synth.Segments(keys, segs.vals, segs.offsets, segs.lengths, segs.desc)
    _run(darm, s, True, "melded", per_seg=False)
    assert darm.device_status() == darm.ERR_SENTINEL_COLLISION
    assert darm.device_status() == darm.OK  # reading clears it
    # keys only: no payload, so the result is still exact and nothing is latched
    ek, _ = _expect(s, False, per_seg=False)
    gk, _ = _run(darm, s, False, "melded", per_seg=False)
    assert_equal("keys", gk, ek)
    assert darm.device_status() == darm.OK


def test_invalid_layouts(darm):
    import torch
    k = to_dev(np.zeros(64, np.uint32))
    with pytest.raises(darm.DarmError) as e:  # capacity 12 is not a power of two
        darm.segmented_sort(k, None, np.array([0, 12], np.uint64), np.array([12], np.uint32))
    assert e.value.status == darm.ERR_NOT_POW2
    with pytest.raises(darm.DarmError) as e:  # length beyond capacity
        darm.segmented_sort(k, None, np.array([0, 16], np.uint64), np.array([17], np.uint32))
    assert e.value.status == darm.ERR_INVALID_ARG
    with pytest.raises(darm.DarmError) as e:  # offset not a multiple of min(capacity, 4)
        darm.segmented_sort(k, None, np.array([2, 18], np.uint64), np.array([16], np.uint32))
    assert e.value.status == darm.ERR_INVALID_ARG
    torch.cuda.synchronize()


@pytest.mark.parametrize("variant", ["divergent", "melded"])
def test_cfg4_full_10000_segments(darm, variant):
    """The full batched workload: 10,000 segments, real lengths log-uniform in
    32..65536, sentinel-padded to the next power of two; keys and payload
    (index within the segment) against the oracle, every element."""
    global _CFG4
    try:
        segs, ek, ev = _CFG4
    except NameError:
        segs = synth.cfg4_segments()
        ek, ev = _expect(segs, True, per_seg=False)
        _CFG4 = (segs, ek, ev)
    gk, gv = _run(darm, segs, True, variant, per_seg=False)
    assert_equal("keys", gk, ek)
    assert_equal("payload", gv, ev)
    assert darm.device_status() == darm.OK


def test_autotune_segmented_then_auto(darm, tmp_path):
    """The batch autotuner times whole batched sorts of the layout, leaves the
    segments sorted, persists its choice (a log2 n = 0 line) and later
    DARM_AUTO batched sorts with the tuned plan stay bit-exact."""
    segs = synth.cfg4_segments(seed=77, num_segments=300, largest_first=True)
    db = str(tmp_path / "seg.db")
    k, v = to_dev(segs.keys), to_dev(segs.vals)
    darm.autotune_segmented(k, v, segs.offsets, segs.lengths, db)
    ek, ev = _expect(segs)
    assert_equal("keys after tuning", k.cpu().numpy(), ek)
    lines = [ln.split() for ln in open(db).read().split("\n") if ln.strip()]
    assert len(lines) == 1 and lines[0][2] == "0"
    darm.load_tune_db(db)
    k, v = to_dev(segs.keys), to_dev(segs.vals)
    darm.segmented_sort(k, v, segs.offsets, segs.lengths, variant="auto")
    assert_equal("keys", k.cpu().numpy(), ek)
    assert_equal("payload", v.cpu().numpy(), ev)
