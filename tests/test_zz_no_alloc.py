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
import gc

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


def test_noalloc_allocates_no_device_memory(darm):
    """A warm call changes neither the device's free memory nor torch's
    allocator: the tables go through the library's fixed array."""
    import torch
    segs = synth.cfg4_segments(seed=53, num_segments=300, min_len=1, max_len=20000,
                               largest_first=True)
    src_k, src_v = to_dev(segs.keys), to_dev(segs.vals)
    k, v = src_k.clone(), src_v.clone()
    _call_noalloc(darm, k, v, segs, "melded", None)  # first call: one-time set-up
    torch.cuda.synchronize()
    gc.collect()  # tensors of earlier tests freed now, not during the loop
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        k.copy_(src_k)
        v.copy_(src_v)
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info()[0]
        _call_noalloc(darm, k, v, segs, "melded", None)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == before
    # torch's allocator served no new block (a late collection of an earlier
    # test's tensor may only lower the count)
    assert torch.cuda.memory_allocated() <= alloc0
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_refuses_a_capturing_stream(darm):
    """The call copies its tables from host memory it frees before returning,
    so it must never be recorded into a CUDA graph: on a capturing stream it
    returns DARM_ERR_INVALID_ARG and enqueues nothing."""
    import torch
    segs = synth.cfg4_segments(seed=54, num_segments=50, min_len=1, max_len=5000,
                               largest_first=True)
    k = to_dev(segs.keys)
    off = np.ascontiguousarray(segs.offsets, dtype=np.uint64)
    ln = np.ascontiguousarray(segs.lengths, dtype=np.uint32)
    side = torch.cuda.Stream()
    node = torch.zeros(16, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        g.capture_begin()
        rc = darm.lib.darm_segmented_sort_noalloc(
            ctypes.c_void_p(k.data_ptr()), None, off.ctypes.data_as(ctypes.c_void_p),
            ln.ctypes.data_as(ctypes.c_void_p), ln.size, darm.ASC, darm.MELDED, None,
            ctypes.c_void_p(side.cuda_stream))
        node.add_(1.0)  # the capture holds one node of torch's own
        g.capture_end()
    assert rc == darm.ERR_INVALID_ARG
    torch.cuda.synchronize()
    # nothing was enqueued: the keys are untouched
    assert np.array_equal(k.cpu().numpy(), segs.keys)
    # the same call outside the capture is valid and sorts
    _call_noalloc(darm, k, None, segs, "melded", None)
    torch.cuda.synchronize()
    assert not np.array_equal(k.cpu().numpy(), segs.keys)


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
