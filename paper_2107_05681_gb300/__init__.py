"""Python binding of the GB300 bitonic compare-exchange library (libdarm.so).

Argument marshalling only: every step of a sort runs in the CUDA library
behind the C ABI declared in include/darm.h.  PyTorch supplies device memory
and streams.  There is no fallback: if the library is missing or fails to
load, importing this package raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdarm.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_NOT_POW2 = 2
ERR_NOT_INIT = 3
ERR_OOM = 4
ERR_CUDA = 5
ERR_BUDGET = 6
ERR_TIMEOUT = 7
ERR_SENTINEL_COLLISION = 8
ERR_BUSY = 9
ERR_NOT_FOUND = 10

ASC, DESC = 0, 1
DIVERGENT, MELDED, AUTO = 0, 1, 2
U32, F32, U64 = 0, 1, 2

_VARIANTS = {"divergent": DIVERGENT, "melded": MELDED, "auto": AUTO,
             DIVERGENT: DIVERGENT, MELDED: MELDED, AUTO: AUTO}


class DarmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_str(status)}" if what else status_str(status))


if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(the library has no CPU fallback)")

lib = ctypes.CDLL(LIB_PATH)

_vp, _u64, _i32, _sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t
_sig = {
    "darm_sort_init": ([_i32, _sz], _i32),
    "darm_sort_finalize": ([], _i32),
    "darm_status_str": ([_i32], ctypes.c_char_p),
    "darm_device_status": ([ctypes.POINTER(_i32)], _i32),
    "darm_bitonic_sort": ([_vp, _vp, _sz, _i32, _i32, _vp], _i32),
    "darm_bitonic_sort_f32": ([_vp, _vp, _sz, _i32, _i32, _vp], _i32),
    "darm_bitonic_sort_u64": ([_vp, _vp, _sz, _i32, _i32, _vp], _i32),
    "darm_bitonic_sort_host": ([_vp, _vp, _sz, _i32, _i32, _i32], _i32),
    "darm_segmented_sort": ([_vp, _vp, _vp, _vp, ctypes.c_uint32, _i32, _i32, _vp, _vp], _i32),
    "darm_segmented_sort_noalloc": ([_vp, _vp, _vp, _vp, ctypes.c_uint32, _i32, _i32, _vp, _vp],
                                    _i32),
    "darm_oddeven_sort_block": ([_vp, _vp, _sz, _i32, _vp], _i32),
    "darm_oddeven_sort_buckets": ([_vp, _vp, _sz, _sz, _i32, _vp], _i32),
    "darm_sb_run": ([_i32, _vp, _sz, _i32, _i32, _i32, _vp], _i32),
    "darm_pcm_sort": ([_vp, _vp, _sz, _sz, _vp, _vp, _i32, _vp], _i32),
    "darm_bitonic_sort_shard": ([_vp, _vp, _sz, _i32, _sz, _sz, _i32, _i32, _vp], _i32),
    "darm_bitonic_exchange": ([_vp, _vp, _vp, _vp, _sz, _i32, _sz, _sz, _i32, _i32, _i32, _vp],
                              _i32),
    "darm_bitonic_merge_shard": ([_vp, _vp, _sz, _i32, _sz, _sz, _i32, _i32, _i32, _vp], _i32),
    "darm_meld_mp_block": ([_vp, _i32, _vp, _i32], ctypes.c_double),
    "darm_meld_mp_subgraph": ([_vp, _vp, _vp, _vp, _i32], ctypes.c_double),
    "darm_meld_align": ([_vp, _i32, _vp, _i32, ctypes.c_double, _vp, _vp], _i32),
    "darm_meld_mp_sese": ([_vp, _vp, _i32, _vp, _vp], ctypes.c_double),
    "darm_meld_subgraph_align": ([_vp, _vp, _i32, _vp, _i32, _vp, _i32, ctypes.c_double,
                                  ctypes.c_double, _vp, _vp, _vp, _vp], _i32),
    "darm_autotune": ([_i32, _sz, _i32, ctypes.c_char_p], _i32),
    "darm_autotune_segmented": ([_vp, _vp, _vp, _vp, ctypes.c_uint32, ctypes.c_char_p], _i32),
    "darm_load_tune_db": ([ctypes.c_char_p], _i32),
    "darm_reset_tunings": ([], _i32),
    "darm_plan_info": ([_i32, _sz, _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                        ctypes.POINTER(_i32)], _i32),
    "darm_launch_count": ([], _u64),
    "darm_plan_describe": ([_i32, _sz, _i32, _i32, ctypes.c_char_p, _sz], _i32),
    "darm_plan_dump": ([_i32, _sz, _i32, _i32, _vp, _sz, _vp, _i32, ctypes.POINTER(_i32)], _i32),
    "darm_sort_profile": ([_vp, _vp, _sz, _i32, _i32, _i32, _vp, ctypes.POINTER(ctypes.c_float),
                           ctypes.POINTER(_i32), _i32, ctypes.POINTER(_i32)], _i32),
    "darm_sort_serve_start": ([_vp], _i32),
    "darm_sort_serve_submit": ([_vp, _vp, _sz, _i32, _i32, ctypes.POINTER(_u64)], _i32),
    "darm_sort_serve_poll": ([_u64, ctypes.POINTER(_i32)], _i32),
    "darm_sort_serve_wait": ([_u64, _i32], _i32),
    "darm_sort_serve_stats": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_u64)], _i32),
    "darm_sort_serve_stop": ([], _i32),
    "darm_sort_serve_inject_fault": ([_i32], _i32),
    "darm_check_bounded_wait": ([_vp], _i32),
}
for _name, (_args, _res) in _sig.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res

EXPORTED = tuple(_sig)


class ServeCfg(ctypes.Structure):
    _fields_ = [("budget_bytes", _sz), ("max_inflight", _i32), ("variant", _i32),
                ("num_streams", _i32)]


def status_str(status: int) -> str:
    return lib.darm_status_str(int(status)).decode()


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise DarmError(rc, what)


def _variant(v) -> int:
    try:
        return _VARIANTS[v]
    except KeyError:
        raise ValueError(f"unknown variant {v!r}") from None


def init(device: int = 0, workspace_bytes: int = 0) -> None:
    _check(lib.darm_sort_init(int(device), int(workspace_bytes)), "darm_sort_init")


def finalize() -> None:
    _check(lib.darm_sort_finalize(), "darm_sort_finalize")


def device_status() -> int:
    st = ctypes.c_int(0)
    _check(lib.darm_device_status(ctypes.byref(st)), "darm_device_status")
    return st.value


def check_bounded_wait(stream=None) -> None:
    """Enqueue the bounded-wait diagnostic: a kernel waits on an mbarrier
    that nothing completes, gives up after about a second and latches
    ERR_TIMEOUT in the device status word (read it with device_status())."""
    _check(lib.darm_check_bounded_wait(_stream_handle(stream)), "darm_check_bounded_wait")


def launch_count() -> int:
    return int(lib.darm_launch_count())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def sort(keys, vals=None, descending: bool = False, variant="melded", stream=None) -> None:
    """Sort a contiguous CUDA tensor of uint32, float32 or uint64 keys in place
    (payload `vals`, a uint32 tensor, travels with its key)."""
    import torch
    if not keys.is_cuda or not keys.is_contiguous() or keys.dim() != 1:
        raise ValueError("keys must be a contiguous 1-D CUDA tensor")
    vp = None
    if vals is not None:
        if vals.dtype != torch.uint32 or vals.shape != keys.shape or not vals.is_contiguous():
            raise ValueError("vals must be a contiguous uint32 CUDA tensor shaped like keys")
        vp = ctypes.c_void_p(vals.data_ptr())
    kp = ctypes.c_void_p(keys.data_ptr())
    n = keys.numel()
    d = DESC if descending else ASC
    v = _variant(variant)
    s = _stream_handle(stream)
    if keys.dtype == torch.uint32:
        rc = lib.darm_bitonic_sort(kp, vp, n, d, v, s)
    elif keys.dtype == torch.float32:
        rc = lib.darm_bitonic_sort_f32(kp, vp, n, d, v, s)
    elif keys.dtype == torch.uint64:
        rc = lib.darm_bitonic_sort_u64(kp, vp, n, d, v, s)
    else:
        raise ValueError(f"unsupported key dtype {keys.dtype}")
    _check(rc, "darm_bitonic_sort")


def oddeven_sort_block(keys, vals=None, variant="melded", stream=None) -> None:
    """Sort a contiguous uint32 CUDA tensor of at most 4096 keys (power of two)
    ascending in place with Batcher's odd-even merge sort network on one
    thread block; `vals` (uint32) travels with its key."""
    import torch
    if keys.dtype != torch.uint32 or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous uint32 CUDA tensor")
    vp = None
    if vals is not None:
        if vals.dtype != torch.uint32 or vals.shape != keys.shape or not vals.is_contiguous():
            raise ValueError("vals must be a contiguous uint32 CUDA tensor shaped like keys")
        vp = ctypes.c_void_p(vals.data_ptr())
    rc = lib.darm_oddeven_sort_block(ctypes.c_void_p(keys.data_ptr()), vp, keys.numel(),
                                     _variant(variant), _stream_handle(stream))
    _check(rc, "darm_oddeven_sort_block")


# ---- synthetic divergent kernels -----------------------------------------------

SB_PATTERNS = {"SB1": 1, "SB2": 2, "SB3": 3, "SB4": 4,
               "SB1-R": 101, "SB2-R": 102, "SB3-R": 103, "SB4-R": 104}


def sb_run(pattern: str, data, iters: int, rounds: int, variant="melded", stream=None) -> None:
    """Run a synthetic divergent kernel (SB1-SB4, SB1-R-SB4-R) in place on a
    contiguous uint32 CUDA tensor of whole 1024-word blocks."""
    import torch
    if data.dtype != torch.uint32 or not data.is_cuda or not data.is_contiguous():
        raise ValueError("data must be a contiguous uint32 CUDA tensor")
    if data.numel() % 1024:
        raise ValueError("data must hold whole blocks of 1024 words")
    rc = lib.darm_sb_run(SB_PATTERNS[pattern], ctypes.c_void_p(data.data_ptr()),
                         data.numel() // 1024, int(iters), int(rounds), _variant(variant),
                         _stream_handle(stream))
    _check(rc, "darm_sb_run")


# ---- melding analysis (host only) ----------------------------------------------

def _insts(seq):
    """[(opcode, type, latency), ...] -> contiguous int32 array of darm_inst."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(seq, dtype=np.int32).reshape(-1, 3))
    return a, (a.ctypes.data_as(ctypes.c_void_p) if a.size else None)


def meld_mp_block(b1, b2) -> float:
    """MP_B of two basic blocks given as [(opcode, type, latency), ...]."""
    a1, p1 = _insts(b1)
    a2, p2 = _insts(b2)
    return float(lib.darm_meld_mp_block(p1, len(a1), p2, len(a2)))


def meld_mp_subgraph(blocks1, blocks2) -> float:
    """MP_S of two subgraphs given as lists of corresponding blocks."""
    import numpy as np
    if len(blocks1) != len(blocks2) or not blocks1:
        raise ValueError("subgraphs must have the same, non-zero number of blocks")
    off1 = np.cumsum([0] + [len(b) for b in blocks1]).astype(np.int32)
    off2 = np.cumsum([0] + [len(b) for b in blocks2]).astype(np.int32)
    a1, p1 = _insts([i for b in blocks1 for i in b])
    a2, p2 = _insts([i for b in blocks2 for i in b])
    return float(lib.darm_meld_mp_subgraph(p1, off1.ctypes.data_as(ctypes.c_void_p), p2,
                                           off2.ctypes.data_as(ctypes.c_void_p), len(blocks1)))


def meld_align(a, b, gap: float = 1.0):
    """Smith-Waterman instruction alignment of two blocks: returns
    ([(i or None, j or None), ...] in program order, score)."""
    import numpy as np
    aa, pa = _insts(a)
    ab, pb = _insts(b)
    pairs = np.zeros(2 * (len(aa) + len(ab)) + 2, dtype=np.int32)
    score = ctypes.c_double(0.0)
    n = lib.darm_meld_align(pa, len(aa), pb, len(ab), float(gap),
                            pairs.ctypes.data_as(ctypes.c_void_p), ctypes.byref(score))
    if n < 0:
        raise ValueError("bad alignment arguments")
    out = [(None if x < 0 else int(x), None if y < 0 else int(y))
           for x, y in pairs[: 2 * n].reshape(-1, 2)]
    return out, float(score.value)


MELD_THRESHOLD = 0.2  # the paper's default melding profitability threshold


def _subgraph_tables(*paths):
    """Subgraphs given as (blocks, shape, simple_region), blocks a list of
    [(opcode, type, latency), ...] in pre-order -> one instruction array, one
    block offset table and a darm_subgraph array (int32 x 4) per path."""
    import numpy as np
    insts, offs, out = [], [0], []
    for path in paths:
        rows = []
        for blocks, shape, simple in path:
            rows.append((len(offs) - 1, len(blocks), int(shape), int(bool(simple))))
            for b in blocks:
                insts.extend(b)
                offs.append(len(insts))
        out.append(np.ascontiguousarray(np.asarray(rows, dtype=np.int32).reshape(-1, 4)))
    ia, ip = _insts(insts)
    off = np.ascontiguousarray(np.asarray(offs, dtype=np.int32))
    return ia, ip, off, out


def meld_mp_sese(s1, s2) -> float:
    """Melding profitability of two SESE subgraphs (blocks, shape,
    simple_region) under Def. 6; -1 when they are not meldable."""
    ia, ip, off, (t1, t2) = _subgraph_tables([s1], [s2])
    return float(lib.darm_meld_mp_sese(ip, off.ctypes.data_as(ctypes.c_void_p), off.size - 1,
                                       t1.ctypes.data_as(ctypes.c_void_p),
                                       t2.ctypes.data_as(ctypes.c_void_p)))


def meld_subgraph_align(true_path, false_path, gap: float = 0.1,
                        threshold: float = MELD_THRESHOLD):
    """Subgraph alignment of two paths (lists of (blocks, shape,
    simple_region)) and Algorithm 1's meld decision: returns
    ([(i, j, profit, meld), ...], score)."""
    import numpy as np
    ia, ip, off, (ts, fs) = _subgraph_tables(true_path, false_path)
    cap = max(1, min(len(ts), len(fs)))
    pairs = np.zeros(2 * cap, dtype=np.int32)
    profit = np.zeros(cap, dtype=np.float64)
    meld = np.zeros(cap, dtype=np.int32)
    score = ctypes.c_double(0.0)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a.size else None  # noqa: E731
    k = lib.darm_meld_subgraph_align(ip, off.ctypes.data_as(ctypes.c_void_p), off.size - 1,
                                     vp(ts), len(ts), vp(fs), len(fs), float(gap),
                                     float(threshold), vp(pairs), vp(profit), vp(meld),
                                     ctypes.byref(score))
    if k < 0:
        raise ValueError("bad subgraph alignment arguments")
    return ([(int(pairs[2 * i]), int(pairs[2 * i + 1]), float(profit[i]), bool(meld[i]))
             for i in range(k)], float(score.value))


def oddeven_sort_buckets(keys, vals=None, bucket: int = 4096, variant="melded",
                         stream=None) -> None:
    """Sort every aligned bucket of `bucket` keys (power of two, <= 4096) of a
    contiguous uint32 CUDA tensor in place with the odd-even merge sort
    network, one thread block per bucket."""
    import torch
    if keys.dtype != torch.uint32 or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous uint32 CUDA tensor")
    vp = None
    if vals is not None:
        if vals.dtype != torch.uint32 or vals.shape != keys.shape or not vals.is_contiguous():
            raise ValueError("vals must be a contiguous uint32 CUDA tensor shaped like keys")
        vp = ctypes.c_void_p(vals.data_ptr())
    rc = lib.darm_oddeven_sort_buckets(ctypes.c_void_p(keys.data_ptr()), vp, keys.numel(),
                                       int(bucket), _variant(variant), _stream_handle(stream))
    _check(rc, "darm_oddeven_sort_buckets")


def pcm_sort(keys, vals=None, bucket: int = 4096, scratch_keys=None, scratch_vals=None,
             variant="melded", stream=None) -> None:
    """PCM: sort a contiguous uint32 CUDA tensor (and its payload) in place,
    buckets of `bucket` keys sorted by the odd-even network, then merged by
    the odd-even network over buckets with merge-splits.  The scratch
    tensors (same shape) are created here when not given."""
    import torch
    if keys.dtype != torch.uint32 or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous uint32 CUDA tensor")
    vp = svp = None
    if scratch_keys is None:
        scratch_keys = torch.empty_like(keys)
    if vals is not None:
        if vals.dtype != torch.uint32 or vals.shape != keys.shape or not vals.is_contiguous():
            raise ValueError("vals must be a contiguous uint32 CUDA tensor shaped like keys")
        vp = ctypes.c_void_p(vals.data_ptr())
        if scratch_vals is None:
            scratch_vals = torch.empty_like(vals)
        svp = ctypes.c_void_p(scratch_vals.data_ptr())
    rc = lib.darm_pcm_sort(ctypes.c_void_p(keys.data_ptr()), vp, keys.numel(), int(bucket),
                           ctypes.c_void_p(scratch_keys.data_ptr()), svp, _variant(variant),
                           _stream_handle(stream))
    _check(rc, "darm_pcm_sort")


def _key_dtype_code(keys):
    import torch
    codes = {torch.uint32: U32, torch.float32: F32, torch.uint64: U64}
    if keys.dtype not in codes or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous uint32, float32 or uint64 CUDA tensor")
    return codes[keys.dtype]


def _vals_ptr(keys, vals):
    import torch
    if vals is None:
        return None
    if vals.dtype != torch.uint32 or vals.shape != keys.shape or not vals.is_contiguous():
        raise ValueError("vals must be a contiguous uint32 CUDA tensor shaped like keys")
    return ctypes.c_void_p(vals.data_ptr())


def sort_shard(keys, vals, shard: int, nshards: int, descending=False, variant="melded",
               stream=None) -> None:
    """Stages 2 .. n of the network of an array of nshards shards, on shard
    `shard` (keys/vals: that shard, on this device)."""
    rc = lib.darm_bitonic_sort_shard(ctypes.c_void_p(keys.data_ptr()), _vals_ptr(keys, vals),
                                     keys.numel(), _key_dtype_code(keys), int(shard),
                                     int(nshards), DESC if descending else ASC,
                                     _variant(variant), _stream_handle(stream))
    _check(rc, "darm_bitonic_sort_shard")


def exchange_shard(keys, vals, peer_keys, peer_vals, shard: int, nshards: int, log2k: int,
                   log2j: int, descending=False, stream=None) -> None:
    """Layer 2^log2j of stage 2^log2k against the peer shard's copy."""
    rc = lib.darm_bitonic_exchange(
        ctypes.c_void_p(keys.data_ptr()), _vals_ptr(keys, vals),
        ctypes.c_void_p(peer_keys.data_ptr()),
        None if peer_vals is None else ctypes.c_void_p(peer_vals.data_ptr()), keys.numel(),
        _key_dtype_code(keys), int(shard), int(nshards), int(log2k), int(log2j),
        DESC if descending else ASC, _stream_handle(stream))
    _check(rc, "darm_bitonic_exchange")


def merge_shard(keys, vals, shard: int, nshards: int, log2k: int, descending=False,
                variant="melded", stream=None) -> None:
    """Layers n/2 .. 1 of stage 2^log2k on this shard."""
    rc = lib.darm_bitonic_merge_shard(ctypes.c_void_p(keys.data_ptr()), _vals_ptr(keys, vals),
                                      keys.numel(), _key_dtype_code(keys), int(shard),
                                      int(nshards), int(log2k), DESC if descending else ASC,
                                      _variant(variant), _stream_handle(stream))
    _check(rc, "darm_bitonic_merge_shard")


def sort_host(keys, vals=None, descending: bool = False, variant="melded") -> None:
    """Sort numpy arrays (host memory) in place through the library: the
    library copies them to the device, sorts and copies them back."""
    import numpy as np
    if not keys.flags.c_contiguous:
        raise ValueError("keys must be C-contiguous")
    dt = {np.dtype(np.uint32): U32, np.dtype(np.float32): F32,
          np.dtype(np.uint64): U64}.get(keys.dtype)
    if dt is None:
        raise ValueError(f"unsupported key dtype {keys.dtype}")
    vp = None
    if vals is not None:
        if vals.dtype != np.uint32 or vals.shape != keys.shape or not vals.flags.c_contiguous:
            raise ValueError("vals must be a C-contiguous uint32 array shaped like keys")
        vp = vals.ctypes.data_as(ctypes.c_void_p)
    rc = lib.darm_bitonic_sort_host(keys.ctypes.data_as(ctypes.c_void_p), vp, keys.size, dt,
                                    DESC if descending else ASC, _variant(variant))
    _check(rc, "darm_bitonic_sort_host")


def segmented_sort(keys, vals, offsets, lengths, descending: bool = False, variant="melded",
                   seg_desc=None, stream=None) -> None:
    """Sort independent power-of-two segments of a uint32 CUDA tensor in place.

    offsets (num_segments + 1, uint64) and lengths (uint32) are host numpy
    arrays; seg_desc (uint8 per segment) optionally overrides the direction.
    """
    import numpy as np
    import torch
    if keys.dtype != torch.uint32 or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous uint32 CUDA tensor")
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    ln = np.ascontiguousarray(lengths, dtype=np.uint32)
    if off.size != ln.size + 1:
        raise ValueError("offsets must have num_segments + 1 entries")
    dp = None
    if seg_desc is not None:
        dd = np.ascontiguousarray(seg_desc, dtype=np.uint8)
        dp = dd.ctypes.data_as(ctypes.c_void_p)
    vp = None if vals is None else ctypes.c_void_p(vals.data_ptr())
    rc = lib.darm_segmented_sort(ctypes.c_void_p(keys.data_ptr()), vp,
                                 off.ctypes.data_as(ctypes.c_void_p),
                                 ln.ctypes.data_as(ctypes.c_void_p), ln.size,
                                 DESC if descending else ASC, _variant(variant), dp,
                                 _stream_handle(stream))
    _check(rc, "darm_segmented_sort")


def segmented_sort_noalloc(keys, vals, offsets, lengths, descending: bool = False,
                           variant="melded", seg_desc=None, stream=None) -> None:
    """segmented_sort for callers that cannot let the library allocate device
    memory: the per-launch tables go through a fixed 1 MiB array inside the
    library (shared by all calls; calls overlapping on the GPU race)."""
    import numpy as np
    import torch
    if keys.dtype != torch.uint32 or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous uint32 CUDA tensor")
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    ln = np.ascontiguousarray(lengths, dtype=np.uint32)
    if off.size != ln.size + 1:
        raise ValueError("offsets must have num_segments + 1 entries")
    dp = None
    if seg_desc is not None:
        dd = np.ascontiguousarray(seg_desc, dtype=np.uint8)
        dp = dd.ctypes.data_as(ctypes.c_void_p)
    vp = None if vals is None else ctypes.c_void_p(vals.data_ptr())
    rc = lib.darm_segmented_sort_noalloc(ctypes.c_void_p(keys.data_ptr()), vp,
                                         off.ctypes.data_as(ctypes.c_void_p),
                                         ln.ctypes.data_as(ctypes.c_void_p), ln.size,
                                         DESC if descending else ASC, _variant(variant), dp,
                                         _stream_handle(stream))
    _check(rc, "darm_segmented_sort_noalloc")


def plan_info(dtype: int, n: int, has_vals: bool, variant="melded"):
    """(passes, launches, tile) of the whole-array plan for n elements."""
    p, l, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.darm_plan_info(int(dtype), int(n), int(bool(has_vals)), _variant(variant),
                              ctypes.byref(p), ctypes.byref(l), ctypes.byref(t)),
           "darm_plan_info")
    return p.value, l.value, t.value


PASS_NAMES = ("tile", "window", "merge")


def sort_profile(keys, vals=None, descending: bool = False, variant="melded", stream=None):
    """Sort in place like sort(), timing each kernel launch with CUDA events
    on the launching stream (the plan's launches in plan order on one stream,
    without the split schedule of large arrays).  Returns a list of (pass
    name, milliseconds)."""
    import torch
    dt = {torch.uint32: U32, torch.float32: F32, torch.uint64: U64}.get(keys.dtype)
    if dt is None or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous uint32/float32/uint64 CUDA tensor")
    cap = 256
    ms = (ctypes.c_float * cap)()
    kinds = (_i32 * cap)()
    cnt = _i32(0)
    vp = None if vals is None else ctypes.c_void_p(vals.data_ptr())
    _check(lib.darm_sort_profile(ctypes.c_void_p(keys.data_ptr()), vp, keys.numel(), dt,
                                 DESC if descending else ASC, _variant(variant),
                                 _stream_handle(stream), ms, kinds, cap, ctypes.byref(cnt)),
           "darm_sort_profile")
    return [(PASS_NAMES[kinds[i]], float(ms[i])) for i in range(min(cnt.value, cap))]


def autotune(dtype: int, n: int, has_vals: bool, db_path: str | None = None) -> None:
    _check(lib.darm_autotune(int(dtype), int(n), int(bool(has_vals)),
                             None if db_path is None else db_path.encode()), "darm_autotune")


def autotune_segmented(keys, vals, offsets, lengths, db_path: str | None = None) -> None:
    """Tune batched segmented sorts on this layout (see segmented_sort for the
    arguments); the segments are left sorted ascending.  Later
    segmented_sort(..., variant="auto") calls use the result."""
    import numpy as np
    import torch
    if keys.dtype != torch.uint32 or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous uint32 CUDA tensor")
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    ln = np.ascontiguousarray(lengths, dtype=np.uint32)
    if off.size != ln.size + 1:
        raise ValueError("offsets must have num_segments + 1 entries")
    vp = None if vals is None else ctypes.c_void_p(vals.data_ptr())
    rc = lib.darm_autotune_segmented(ctypes.c_void_p(keys.data_ptr()), vp,
                                     off.ctypes.data_as(ctypes.c_void_p),
                                     ln.ctypes.data_as(ctypes.c_void_p), ln.size,
                                     None if db_path is None else db_path.encode())
    _check(rc, "darm_autotune_segmented")


def load_tune_db(db_path: str) -> None:
    _check(lib.darm_load_tune_db(db_path.encode()), "darm_load_tune_db")


def plan_describe(dtype: int, n: int, has_vals: bool, variant="melded") -> list[str]:
    """The launch sequence of a whole-array sort, one line per launch."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib.darm_plan_describe(dtype, n, int(bool(has_vals)), _variant(variant), buf,
                                  len(buf)), "darm_plan_describe")
    return buf.value.decode().splitlines()


_LAUNCH_FIELDS = ("kind", "fixed", "tma", "win1", "win2", "shfl", "loge", "variant", "grid",
                  "threads", "smem", "b", "c", "w0", "s", "log2cap", "nrounds", "nblocks",
                  "map_in", "map_out", "mshfl")
_ROUND_FIELDS = ("kind", "p", "a", "cnt", "src", "dst", "lanediv")


def plan_dump(dtype: int, n: int, has_vals: bool, variant="melded", tuning=None,
              smem_limit: int = 0) -> list[dict]:
    """The launch sequence of a whole-array sort as dicts (host only: no
    device needed).  tuning: (t, e1, e2, c2, w2, tma, shfl[, tm]) or None
    (tm, the merge passes' log2 tile, 0 when absent: the tile pass's)."""
    import numpy as np
    tn = None
    if tuning is not None:
        t8 = list(tuning) + [0] * (8 - len(tuning))
        tn = np.ascontiguousarray(np.asarray(t8[:8], dtype=np.int32))
    cnt = ctypes.c_int(0)
    args = (dtype, n, int(bool(has_vals)), _variant(variant),
            None if tn is None else tn.ctypes.data_as(ctypes.c_void_p), smem_limit)
    rc = lib.darm_plan_dump(*args, None, 0, ctypes.byref(cnt))
    if rc not in (OK, ERR_INVALID_ARG) or cnt.value == 0:
        _check(rc if rc != OK else ERR_INVALID_ARG, "darm_plan_dump")
    buf = np.zeros(cnt.value, dtype=np.int32)
    _check(lib.darm_plan_dump(*args, buf.ctypes.data_as(ctypes.c_void_p), buf.size,
                              ctypes.byref(cnt)), "darm_plan_dump")
    out, i = [], 0
    while i < buf.size:
        L = dict(zip(_LAUNCH_FIELDS, (int(x) for x in buf[i:i + 21])))
        i += 21
        L["rounds"] = []
        for _ in range(L["nrounds"]):
            L["rounds"].append(dict(zip(_ROUND_FIELDS, (int(x) for x in buf[i:i + 7]))))
            i += 7
        out.append(L)
    return out


def reset_tunings() -> None:
    """Forget loaded or measured tunings: plans return to the defaults."""
    _check(lib.darm_reset_tunings(), "darm_reset_tunings")


# ---- serving -----------------------------------------------------------------

def serve_start(budget_bytes: int, max_inflight: int = 64, variant="melded",
                num_streams: int = 1) -> None:
    """Start the continuous-batching scheduler with a device arena of
    `budget_bytes` (a job of n keys costs 12 * next_pow2(n) bytes)."""
    cfg = ServeCfg(int(budget_bytes), int(max_inflight), _variant(variant), int(num_streams))
    _check(lib.darm_sort_serve_start(ctypes.byref(cfg)), "darm_sort_serve_start")


def serve_submit(keys, vals=None, descending: bool = False) -> int:
    """Queue an in-place sort of a CUDA tensor (uint64, uint32 or float32
    keys; optional uint32 payload).  The tensors must stay alive until done."""
    import torch
    dt = {torch.uint32: U32, torch.float32: F32, torch.uint64: U64}.get(keys.dtype)
    if dt is None or not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous uint64/uint32/float32 CUDA tensor")
    vp = None
    if vals is not None:
        if vals.dtype != torch.uint32 or vals.shape != keys.shape or not vals.is_contiguous():
            raise ValueError("vals must be a contiguous uint32 CUDA tensor shaped like keys")
        vp = ctypes.c_void_p(vals.data_ptr())
    rid = _u64(0)
    _check(lib.darm_sort_serve_submit(ctypes.c_void_p(keys.data_ptr()), vp, keys.numel(), dt,
                                      DESC if descending else ASC, ctypes.byref(rid)),
           "darm_sort_serve_submit")
    return int(rid.value)


def serve_poll(req_id: int) -> bool:
    done = _i32(0)
    _check(lib.darm_sort_serve_poll(int(req_id), ctypes.byref(done)), "darm_sort_serve_poll")
    return bool(done.value)


def serve_wait(req_id: int, timeout_ms: int = 60000) -> None:
    _check(lib.darm_sort_serve_wait(int(req_id), int(timeout_ms)), "darm_sort_serve_wait")


def serve_stats():
    """(p50 ms, p99 ms, keys/s, completed) over all completed requests."""
    p50, p99, kps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    done = _u64(0)
    _check(lib.darm_sort_serve_stats(ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(kps),
                                     ctypes.byref(done)), "darm_sort_serve_stats")
    return p50.value, p99.value, kps.value, int(done.value)


def serve_inject_fault(status: int) -> None:
    _check(lib.darm_sort_serve_inject_fault(int(status)), "darm_sort_serve_inject_fault")


def serve_stop() -> None:
    _check(lib.darm_sort_serve_stop(), "darm_sort_serve_stop")
