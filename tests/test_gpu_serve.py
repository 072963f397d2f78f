"""GPU tests of the continuous-batching sort service: every result equals the
oracle's and is the same alone and in the mix (tolerance 0); the budget is
enforced; waits time out; injected host faults fail only the jobs they hit."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_equal, to_dev

pytestmark = pytest.mark.gpu


def _requests(count, seed=5, min_log2=4.0, max_log2=15.0):
    reqs = synth.cfg5_requests(seed=seed, count=count, min_log2=min_log2, max_log2=max_log2,
                               materialize=True)
    return reqs


def _expected(r):
    cap = 1
    while cap < r.n:
        cap *= 2
    # the service pads to a power of two with the direction's extreme key;
    # the real elements come first
    sent = np.uint64(0) if r.desc else np.uint64(0xFFFFFFFFFFFFFFFF)
    k = np.concatenate([r.keys, np.full(cap - r.n, sent, np.uint64)])
    v = np.concatenate([r.vals, np.full(cap - r.n, 0xFFFFFFFF, np.uint32)])
    ek, ev = oracle.bitonic_sort(k, v, desc=r.desc)
    return ek[:r.n], ev[:r.n]


@pytest.fixture()
def server(darm):
    darm.serve_start(budget_bytes=24 << 20, max_inflight=16, variant="melded", num_streams=2)
    yield darm
    darm.serve_stop()


def test_mixed_equals_alone_and_oracle(server):
    darm = server
    import torch
    reqs = _requests(48)
    # alone: one request on the GPU at a time
    alone = []
    for r in reqs:
        k, v = to_dev(r.keys), to_dev(r.vals)
        rid = darm.serve_submit(k, v, descending=r.desc)
        darm.serve_wait(rid, 60000)
        alone.append((k.cpu().numpy(), v.cpu().numpy()))
    # mixed: all submitted at once, admitted as budget and slots free up
    bufs = [(to_dev(r.keys), to_dev(r.vals)) for r in reqs]
    ids = [darm.serve_submit(k, v, descending=r.desc) for (k, v), r in zip(bufs, reqs)]
    for rid in ids:
        darm.serve_wait(rid, 60000)
    torch.cuda.synchronize()
    for r, (ka, va), (k, v) in zip(reqs, alone, bufs):
        ek, ev = _expected(r)
        assert_equal("keys alone", ka, ek)
        assert_equal("payload alone", va, ev)
        assert_equal("keys mixed", k.cpu().numpy(), ek)
        assert_equal("payload mixed", v.cpu().numpy(), ev)
    p50, p99, kps, done = darm.serve_stats()
    assert done == 2 * len(reqs)
    assert 0 < p50 <= p99 and kps > 0


_FULL_RANGE = {}


def _full_range_requests():
    """Requests over the whole serving size range, 2^8 .. 2^20 keys (uint64
    keys, uint32 payload = index, mixed directions), both ends included, with
    the oracle's results computed once and shared by both kernel forms."""
    if not _FULL_RANGE:
        reqs = synth.cfg5_requests(seed=0xDA2C0005, count=30, materialize=True)
        for n, desc, seed in ((1 << 20, False, 61), (1 << 20, True, 62), (256, True, 63),
                              ((1 << 20) - 3, True, 64), (257, False, 65)):
            reqs.append(synth.Request(0.0, n, desc, synth.uniform_u64(seed, n),
                                      np.arange(n, dtype=np.uint32)))
        _FULL_RANGE["reqs"] = reqs
        _FULL_RANGE["expected"] = [_expected(r) for r in reqs]
    return _FULL_RANGE["reqs"], _FULL_RANGE["expected"]


@pytest.mark.parametrize("variant", ["melded", "divergent"])
def test_full_size_range_alone_and_mixed_equal_the_oracle(darm, variant):
    """Every request of 2^8 .. 2^20 keys equals the oracle's sort, alone on
    the GPU and admitted into a mix under a budget that holds only part of
    the batch at once (so later requests join while others run)."""
    import torch
    reqs, expected = _full_range_requests()
    assert min(r.n for r in reqs) == 256 and max(r.n for r in reqs) == 1 << 20
    darm.serve_start(budget_bytes=64 << 20, max_inflight=16, variant=variant, num_streams=2)
    try:
        for r, (ek, ev) in zip(reqs, expected):
            k, v = to_dev(r.keys), to_dev(r.vals)
            darm.serve_wait(darm.serve_submit(k, v, descending=r.desc), 120000)
            assert_equal(f"keys alone (n={r.n})", k.cpu().numpy(), ek)
            assert_equal(f"payload alone (n={r.n})", v.cpu().numpy(), ev)
        bufs = [(to_dev(r.keys), to_dev(r.vals)) for r in reqs]
        ids = [darm.serve_submit(k, v, descending=r.desc) for (k, v), r in zip(bufs, reqs)]
        for rid in ids:
            darm.serve_wait(rid, 120000)
        torch.cuda.synchronize()
        for r, (ek, ev), (k, v) in zip(reqs, expected, bufs):
            assert_equal(f"keys mixed (n={r.n})", k.cpu().numpy(), ek)
            assert_equal(f"payload mixed (n={r.n})", v.cpu().numpy(), ev)
        assert darm.device_status() == darm.OK
    finally:
        darm.serve_stop()


def _expected_narrow(words, vals, desc):
    """Service semantics for 32-bit keys: keys are ordered as 32-bit words
    (floats by their totalOrder word) and padding is strictly beyond every
    real key.  Computed with the oracle on 64-bit words w + 1, padded with 0
    or 2^64 - 1, which have exactly that order."""
    n = words.size
    cap = 1
    while cap < n:
        cap *= 2
    w = words.astype(np.uint64) + np.uint64(1)
    pad = np.uint64(0) if desc else np.uint64(0xFFFFFFFFFFFFFFFF)
    k = np.concatenate([w, np.full(cap - n, pad, np.uint64)])
    v = np.concatenate([vals, np.full(cap - n, 0xFFFFFFFF, np.uint32)])
    ek, ev = oracle.bitonic_sort(k, v, desc=desc)
    return (ek[:n] - np.uint64(1)).astype(np.uint32), ev[:n]


def test_u32_and_f32_keys(server):
    darm = server
    import torch
    from tests.gpu_util import total_order_u32
    n = 3000
    ku = synth.uniform_u32(41, n) % np.uint32(97)
    kf = synth.cfg3_f32(42, n, dup_frac=0.05, zeros_each=20)
    vals = np.arange(n, dtype=np.uint32)
    cases = [(ku, False), (ku, True), (kf, False), (kf, True)]
    outs = []
    for keys, desc in cases:
        k, v = to_dev(keys), to_dev(vals)
        outs.append((k, v, darm.serve_submit(k, v, descending=desc)))
    for (keys, desc), (k, v, rid) in zip(cases, outs):
        darm.serve_wait(rid, 60000)
        torch.cuda.synchronize()
        if keys.dtype == np.float32:
            words = total_order_u32(keys)
            ew, ev = _expected_narrow(words, vals, desc)
            got = total_order_u32(k.cpu().numpy())
        else:
            ew, ev = _expected_narrow(keys, vals, desc)
            got = k.cpu().numpy()
        assert_equal("keys", got, ew)
        assert_equal("payload", v.cpu().numpy(), ev)
    assert darm.device_status() == darm.OK


def test_budget_rejects_oversize_job(server):
    darm = server
    k = to_dev(np.zeros(1 << 22, np.uint64))  # 12 * 2^22 bytes > 24 MiB budget
    with pytest.raises(darm.DarmError) as e:
        darm.serve_submit(k)
    assert e.value.status == darm.ERR_BUDGET


def test_wait_times_out_then_completes(server):
    darm = server
    n = 1 << 20
    k = to_dev(synth.uniform_u64(7, n))
    # a job that needs the whole arena cannot start before the next one ends
    big = darm.DarmError
    rid = darm.serve_submit(to_dev(synth.uniform_u64(8, 1 << 20)))
    rid2 = darm.serve_submit(k)
    with pytest.raises(big) as e:
        darm.serve_wait(rid2, 0)
    assert e.value.status == darm.ERR_TIMEOUT
    darm.serve_wait(rid, 60000)
    darm.serve_wait(rid2, 60000)
    got = k.cpu().numpy()
    assert np.all(got[1:] >= got[:-1])


def test_injected_fault_fails_only_its_tick(server):
    darm = server
    k1 = to_dev(synth.uniform_u64(9, 5000))
    darm.serve_inject_fault(darm.ERR_CUDA)
    rid = darm.serve_submit(k1)
    with pytest.raises(darm.DarmError) as e:
        darm.serve_wait(rid, 60000)
    assert e.value.status == darm.ERR_CUDA
    # the service keeps running for later requests
    k2 = to_dev(synth.uniform_u64(10, 5000))
    rid2 = darm.serve_submit(k2)
    darm.serve_wait(rid2, 60000)
    got = k2.cpu().numpy()
    assert np.all(got[1:] >= got[:-1])
    assert darm.serve_poll(rid2)


def test_trivial_requests(server):
    darm = server
    for n in (0, 1):
        k = to_dev(np.full(n, 3, np.uint64))
        rid = darm.serve_submit(k)
        assert darm.serve_poll(rid)
        darm.serve_wait(rid, 1000)
