"""Helpers for GPU parity tests: move numpy inputs to the device, run the
library through its C ABI, bring results back."""
from __future__ import annotations

import numpy as np


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_sort(darm, keys, vals=None, desc=False, variant="melded"):
    """Sort copies of numpy arrays on the GPU; return numpy results."""
    import torch
    k = to_dev(keys)
    v = None if vals is None else to_dev(vals)
    darm.sort(k, v, descending=desc, variant=variant)
    torch.cuda.synchronize()
    ko = k.cpu().numpy()
    vo = None if v is None else v.cpu().numpy()
    return ko, vo


def total_order_u32(x: np.ndarray) -> np.ndarray:
    """float32 -> uint32 whose unsigned order is IEEE totalOrder (test-side
    restatement used only to build expected key sequences for keys-only
    checks, where the sorted sequence is unique)."""
    u = x.view(np.uint32)
    neg = (u >> np.uint32(31)).astype(bool)
    return np.where(neg, ~u, u | np.uint32(0x80000000)).astype(np.uint32)


def assert_equal(name, got, exp):
    if not np.array_equal(got, exp):
        bad = np.flatnonzero(got != exp)
        i = int(bad[0])
        raise AssertionError(f"{name}: {bad.size} mismatches, first at {i}: "
                             f"got {got[i]!r} expected {exp[i]!r}")
