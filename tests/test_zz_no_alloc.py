"""The segmented sort entry point that allocates no device memory.

It serves callers that cannot let a library call cudaMalloc (their own
allocator owns the GPU, or they cannot take the synchronisation an allocation
brings).  Its results must equal those of the allocating entry point,
darm_segmented_sort, bit for bit (the tolerance every parity test here uses),
on two calls in a row - the shared scratch array keeps the first call's
contents, which must not leak into the second.  This file is collected last
so that a run stopping at the first failure has run every other test first;
it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests.gpu_util import assert_equal, to_dev

pytestmark = pytest.mark.gpu


def _call_noalloc(darm, k, v, segs, variant, seg_desc):
    """Through the C ABI directly."""
    import torch
    off = np.ascontiguousarray(segs.offsets, dtype=np.uint64)
    ln = np.ascontiguousarray(segs.lengths, dtype=np.uint32)
    dd = None if seg_desc is None else np.ascontiguousarray(seg_desc, dtype=np.uint8)
    rc = darm.lib.darm_segmented_sort_noalloc(
        ctypes.c_void_p(k.data_ptr()), None if v is None else ctypes.c_void_p(v.data_ptr()),
        off.ctypes.data_as(ctypes.c_void_p), ln.ctypes.data_as(ctypes.c_void_p), ln.size,
        darm.ASC, darm._variant(variant),
        None if dd is None else dd.ctypes.data_as(ctypes.c_void_p),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == darm.OK, darm.status_str(rc)


@pytest.mark.parametrize("variant", ["melded", "divergent"])
def test_noalloc_matches_allocating_entry_point_twice(darm, variant):
    import torch
    layouts = [
        # tiny, packed and multi-tile segments, mixed directions
        synth.cfg4_segments(seed=51, num_segments=400, min_len=1, max_len=40000,
                            mixed_dirs=True, largest_first=True),
        # a second, different layout: the scratch must not carry state over
        synth.cfg4_segments(seed=52, num_segments=1500, min_len=32, max_len=65536),
    ]
    for segs in layouts:
        seg_desc = segs.desc if segs.desc.any() else None
        ref_k, ref_v = to_dev(segs.keys), to_dev(segs.vals)
        darm.segmented_sort(ref_k, ref_v, segs.offsets, segs.lengths, variant=variant,
                            seg_desc=seg_desc)
        for _ in range(2):
            k, v = to_dev(segs.keys), to_dev(segs.vals)
            _call_noalloc(darm, k, v, segs, variant, seg_desc)
            torch.cuda.synchronize()
            assert_equal("keys", k.cpu().numpy(), ref_k.cpu().numpy())
            assert_equal("payload", v.cpu().numpy(), ref_v.cpu().numpy())
        # keys only
        ref_k2 = to_dev(segs.keys)
        darm.segmented_sort(ref_k2, None, segs.offsets, segs.lengths, variant=variant,
                            seg_desc=seg_desc)
        k2 = to_dev(segs.keys)
        _call_noalloc(darm, k2, None, segs, variant, seg_desc)
        torch.cuda.synchronize()
        assert_equal("keys only", k2.cpu().numpy(), ref_k2.cpu().numpy())
    assert darm.device_status() == darm.OK


def test_noalloc_rejects_layouts_beyond_its_scratch(darm):
    # 100,000 segments of capacity 32 in one tile pass: their slots alone
    # (16 bytes each) exceed the 1 MiB scratch
    n = 100_000
    offsets = np.arange(n + 1, dtype=np.uint64) * np.uint64(32)
    lengths = np.full(n, 32, np.uint32)
    k = to_dev(np.zeros(n * 32, np.uint32))
    segs = synth.Segments(None, None, offsets, lengths, np.zeros(n, np.uint8))
    off = np.ascontiguousarray(offsets)
    rc = darm.lib.darm_segmented_sort_noalloc(
        ctypes.c_void_p(k.data_ptr()), None, off.ctypes.data_as(ctypes.c_void_p),
        lengths.ctypes.data_as(ctypes.c_void_p), n, darm.ASC, darm.MELDED, None, None)
    assert rc == darm.ERR_INVALID_ARG
    del segs
