"""CPU oracle for the bitonic network of DARM's running example (Fig. 1).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may use this package;
the product library never does.  It shares no code with the CUDA library.

The arithmetic lives in ``darm_oracle.c`` (plain single-threaded C, see its
header for the readings of the paper it takes).  This module only compiles
that file with the host C compiler and marshals numpy arrays through ctypes.
Every function copies its inputs and returns new arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "darm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}

OK = 0
ERR_NOT_POW2 = 2


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (optionally with one planted mistake) and return the .so path."""
    out = lib_path(mutant)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = f"{out}.{os.getpid()}.tmp"
    cc = os.environ.get("CC", "gcc")
    cmd = [cc, "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC,
           f"-DDARM_ORACLE_MUTANT={mutant}"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib(mutant: int = 0) -> ctypes.CDLL:
    with _LOCK:
        if mutant not in _LIBS:
            lib = ctypes.CDLL(build(mutant))
            u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
            for name in ("oracle_bitonic_u32", "oracle_bitonic_u64",
                         "oracle_bitonic_rec_u32", "oracle_bitonic_rec_u64",
                         "oracle_bitonic_f32"):
                fn = getattr(lib, name)
                fn.argtypes = [vp, vp, u64, i32]
                fn.restype = i32
            for name in ("oracle_segmented_u32", "oracle_segmented_u64"):
                fn = getattr(lib, name)
                fn.argtypes = [vp, vp, vp, vp, u64, i32, vp]
                fn.restype = i32
            lib.oracle_oddeven_u32.argtypes = [vp, vp, u64, vp]
            lib.oracle_oddeven_u32.restype = i32
            lib.oracle_oddeven_rec_u32.argtypes = [vp, vp, u64]
            lib.oracle_oddeven_rec_u32.restype = i32
            for name in ("oracle_pcm_u32", "oracle_pcm_rec_u32"):
                fn = getattr(lib, name)
                fn.argtypes = [vp, vp, u64, u64]
                fn.restype = i32
            lib.oracle_sb.argtypes = [i32, vp, u64, i32, i32]
            lib.oracle_sb.restype = i32
            lib.oracle_compare_exchanges.argtypes = [u64]
            lib.oracle_compare_exchanges.restype = u64
            lib.oracle_mutant_id.restype = i32
            _LIBS[mutant] = lib
        return _LIBS[mutant]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


_KEY_FN = {
    np.dtype(np.uint32): "u32",
    np.dtype(np.uint64): "u64",
    np.dtype(np.float32): "f32",
}


def bitonic_sort(keys, vals=None, desc=False, recursive=False, mutant=0):
    """Sort copies of ``keys`` (and ``vals``) with the network of Fig. 1.

    keys: 1-D numpy array of uint32, uint64 or float32, power-of-two length.
    vals: optional uint32 payload of the same length.
    recursive: use the independent recursive formulation instead.
    Returns (keys_out, vals_out or None).  Raises ValueError on bad input.
    """
    k = np.ascontiguousarray(keys).copy()
    if k.ndim != 1:
        raise ValueError("keys must be 1-D")
    kind = _KEY_FN.get(k.dtype)
    if kind is None:
        raise ValueError(f"unsupported key dtype {k.dtype}")
    v = None
    if vals is not None:
        v = np.ascontiguousarray(vals, dtype=np.uint32).copy()
        if v.shape != k.shape:
            raise ValueError("vals must match keys")
    if recursive:
        if kind == "f32":
            raise ValueError("recursive formulation is integer-keyed")
        name = f"oracle_bitonic_rec_{kind}"
    else:
        name = f"oracle_bitonic_{kind}"
    rc = getattr(_lib(mutant), name)(_ptr(k), _ptr(v), k.size, int(bool(desc)))
    if rc == ERR_NOT_POW2:
        raise ValueError("length must be a power of two")
    if rc != OK:
        raise RuntimeError(f"oracle status {rc}")
    return k, v


def segmented_sort(keys, vals, offsets, lengths, desc=False, desc_per_seg=None,
                   mutant=0):
    """Sort every segment [offsets[s], offsets[s+1]) independently.

    Capacities must be powers of two; positions from lengths[s] to the
    capacity receive the sentinel before sorting.  Returns new arrays.
    """
    k = np.ascontiguousarray(keys).copy()
    kind = _KEY_FN.get(k.dtype)
    if kind not in ("u32", "u64"):
        raise ValueError(f"unsupported key dtype {k.dtype}")
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    ln = np.ascontiguousarray(lengths, dtype=np.uint32)
    nseg = ln.size
    if off.size != nseg + 1:
        raise ValueError("offsets must have num_segments + 1 entries")
    dps = None
    if desc_per_seg is not None:
        dps = np.ascontiguousarray(desc_per_seg, dtype=np.uint8)
    rc = getattr(_lib(mutant), f"oracle_segmented_{kind}")(
        _ptr(k), _ptr(v), _ptr(off), _ptr(ln), nseg, int(bool(desc)), _ptr(dps))
    if rc == ERR_NOT_POW2:
        raise ValueError("segment capacity must be a power of two")
    if rc != OK:
        raise RuntimeError(f"oracle status {rc}")
    return k, v


def oddeven_sort(keys, vals=None, recursive=False, mutant=0):
    """Sort copies of uint32 ``keys`` (and ``vals``) with Batcher's odd-even
    merge sort network (ascending).  Returns (keys_out, vals_out or None,
    comparators evaluated, or None for the recursive form)."""
    k = np.ascontiguousarray(keys, dtype=np.uint32).copy()
    if k.ndim != 1:
        raise ValueError("keys must be 1-D")
    v = None
    if vals is not None:
        v = np.ascontiguousarray(vals, dtype=np.uint32).copy()
        if v.shape != k.shape:
            raise ValueError("vals must match keys")
    if recursive:
        rc = _lib(mutant).oracle_oddeven_rec_u32(_ptr(k), _ptr(v), k.size)
        ncmp = None
    else:
        c = ctypes.c_uint64(0)
        rc = _lib(mutant).oracle_oddeven_u32(_ptr(k), _ptr(v), k.size, ctypes.byref(c))
        ncmp = int(c.value)
    if rc == ERR_NOT_POW2:
        raise ValueError("length must be a power of two")
    if rc != OK:
        raise RuntimeError(f"oracle status {rc}")
    return k, v, ncmp


def pcm_sort(keys, vals=None, bucket: int = 4096, recursive=False, mutant=0):
    """PCM (see oracle_pcm_u32 in darm_oracle.c) on copies of uint32 ``keys``
    (and ``vals``): buckets of ``bucket`` keys sorted by the odd-even merge
    sort network, then the network over buckets with merge-splits.
    Returns (keys_out, vals_out or None)."""
    k = np.ascontiguousarray(keys, dtype=np.uint32).copy()
    if k.ndim != 1:
        raise ValueError("keys must be 1-D")
    v = None
    if vals is not None:
        v = np.ascontiguousarray(vals, dtype=np.uint32).copy()
        if v.shape != k.shape:
            raise ValueError("vals must match keys")
    fn = _lib(mutant).oracle_pcm_rec_u32 if recursive else _lib(mutant).oracle_pcm_u32
    rc = fn(_ptr(k), _ptr(v), k.size, int(bucket))
    if rc == ERR_NOT_POW2:
        raise ValueError("bucket size and bucket count must be powers of two")
    if rc != OK:
        raise RuntimeError(f"oracle status {rc}")
    return k, v


SB_PATTERNS = {"SB1": 1, "SB2": 2, "SB3": 3, "SB4": 4,
               "SB1-R": 101, "SB2-R": 102, "SB3-R": 103, "SB4-R": 104}


def sb_run(pattern: str, data, iters: int, rounds: int):
    """The synthetic divergent kernels (see oracle_sb in darm_oracle.c) on a
    copy of ``data`` (uint32, a multiple of 1024 words: one block each)."""
    d = np.ascontiguousarray(data, dtype=np.uint32).copy()
    if d.size % 1024:
        raise ValueError("data must hold whole blocks of 1024 words")
    rc = _lib().oracle_sb(SB_PATTERNS[pattern], _ptr(d), d.size // 1024, int(iters), int(rounds))
    if rc != OK:
        raise ValueError(f"bad pattern {pattern}")
    return d


def compare_exchanges(n: int) -> int:
    """(n/2) * m(m+1)/2 comparators for n = 2^m."""
    return int(_lib().oracle_compare_exchanges(n))
