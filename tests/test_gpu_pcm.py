"""GPU parity of PCM (odd-even merge sort over sorted buckets with
merge-split comparators, both forms of the merge loop) against the oracle:
bit-exact keys and payload order under ties."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_equal, to_dev

pytestmark = pytest.mark.gpu


def _cases():
    out = []
    for m in (4, 10, 14, 18):
        for bucket in (1, 2, 64, 1024, 4096):
            if bucket <= (1 << m):
                out.append((m, bucket))
    return out


@pytest.mark.parametrize("variant", ["divergent", "melded"])
@pytest.mark.parametrize("m,bucket", _cases())
def test_pcm_matches_the_oracle(darm, m, bucket, variant):
    import torch
    n = 1 << m
    keys = synth.uniform_u32(1400 + m + bucket, n) % np.uint32(max(2, n // 8))
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.pcm_sort(keys, vals, bucket=bucket)
    k, v = to_dev(keys), to_dev(vals)
    darm.pcm_sort(k, v, bucket=bucket, variant=variant)
    torch.cuda.synchronize()
    assert_equal("keys", k.cpu().numpy(), ek)
    assert_equal("payload", v.cpu().numpy(), ev)
    # keys only
    k2 = to_dev(keys)
    darm.pcm_sort(k2, bucket=bucket, variant=variant)
    torch.cuda.synchronize()
    assert_equal("keys only", k2.cpu().numpy(), ek)


@pytest.mark.parametrize("variant", ["divergent", "melded"])
def test_pcm_key_value_2pow22_uniform(darm, variant):
    """Uniform keys, the paper's bucket size: 1024 buckets of 4096."""
    import torch
    n = 1 << 22
    keys = synth.uniform_u32(1450, n)
    vals = np.arange(n, dtype=np.uint32)
    ek, ev = oracle.pcm_sort(keys, vals, bucket=4096)
    k, v = to_dev(keys), to_dev(vals)
    darm.pcm_sort(k, v, bucket=4096, variant=variant)
    torch.cuda.synchronize()
    assert_equal("keys", k.cpu().numpy(), ek)
    assert_equal("payload", v.cpu().numpy(), ev)


@pytest.mark.parametrize("variant", ["divergent", "melded"])
def test_pcm_2pow26_keys(darm, variant):
    """2^26 uniform keys in 16,384 buckets of 4096: the sorted key sequence
    is unique, so numpy's sort is the exact expected result."""
    import torch
    keys = synth.uniform_u32(0xDA2C0008, 1 << 26)
    k = to_dev(keys)
    darm.pcm_sort(k, bucket=4096, variant=variant)
    torch.cuda.synchronize()
    assert_equal("keys", k.cpu().numpy(), np.sort(keys))


def test_pcm_arguments_are_checked(darm):
    import torch
    k = to_dev(np.zeros(1 << 12, np.uint32))
    for bucket in (3, 8192):
        with pytest.raises(darm.DarmError):
            darm.pcm_sort(k, bucket=bucket)
    with pytest.raises(darm.DarmError):  # 3 buckets: not a power of two
        darm.pcm_sort(to_dev(np.zeros(3 * 1024, np.uint32)), bucket=1024)
    with pytest.raises(darm.DarmError):  # payload without scratch for it
        rc = darm.lib.darm_pcm_sort(
            ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(k.data_ptr()),
            k.numel(), 64, ctypes.c_void_p(torch.empty_like(k).data_ptr()), None,
            darm.MELDED, None)
        darm._check(rc, "darm_pcm_sort")
    # one bucket: the bucket sort alone, no scratch needed
    keys = synth.uniform_u32(1460, 4096)
    k = to_dev(keys)
    rc = darm.lib.darm_pcm_sort(ctypes.c_void_p(k.data_ptr()), None, 4096, 4096,
                                None, None, darm.MELDED, None)
    assert rc == darm.OK
    torch.cuda.synchronize()
    assert_equal("one bucket", k.cpu().numpy(), oracle.pcm_sort(keys, bucket=4096)[0])
