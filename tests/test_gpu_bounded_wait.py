"""The bounded waits of the kernels that stream tiles with bulk copies: a
wait on an mbarrier that nothing completes gives up after about a second,
latches DARM_ERR_TIMEOUT in the device status word and returns, and the
context stays usable (a sort afterwards is exact)."""
import time

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_equal, gpu_sort

pytestmark = pytest.mark.gpu


def test_wait_gives_up_and_reports_timeout(darm):
    import torch
    assert darm.device_status() == 0
    t0 = time.monotonic()
    darm.check_bounded_wait()
    torch.cuda.synchronize()
    elapsed = time.monotonic() - t0
    assert darm.device_status() == darm.ERR_TIMEOUT
    assert 0.5 < elapsed < 30.0, elapsed
    assert darm.device_status() == 0  # read and cleared
    keys = synth.uniform_u32(0xB0E, 1 << 20)
    ek, _ = oracle.bitonic_sort(keys, None)
    gk, _ = gpu_sort(darm, keys, None)
    assert_equal("keys", gk, ek)
    assert darm.device_status() == 0
