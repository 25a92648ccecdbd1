"""CPU oracle for the hash-join hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm
of ``bench.py`` may import this package.  The product path (the CUDA library
``libhj`` and its binding ``paper_1307_1955_gb300.hj``) never imports, links or
executes it, and this package imports nothing from the product.

The arithmetic lives in ``hj_oracle.c`` (plain single-threaded C, compiled with
gcc on first use); this module only marshals numpy arrays in and out.

Relations are numpy arrays of shape ``(n, 2)`` -- column 0 the key, column 1 the
rid -- of dtype uint32 (four-byte attributes, Sec. 5.1) or uint64.

Functions and what pins them (tests/test_oracle_pins.py):
  hash_join          equi-join by hash map (Sec. 3.1, Alg. 1)        brute force, closed forms, golden
  nested_loop_join   equi-join by definition                         closed forms, golden
  count_sortmerge    |J| = sum_k cR(k)*cS(k)                         closed forms, brute force
  checksum_pairs     order-free sums over the pairs                  SplitMix64 published outputs, golden
  join_aggregate     count and checksums by per-key grouping         equals the pair-level route
  radix_partition    Alg. 2 partitioning on low hash bits            permutation/stability/digit
                                                                     properties; MurmurHash2 pinned by
                                                                     SMHasher's published verification values
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hj_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

# MurmurHash2 seed that the partitioner uses (the library documents seed 0).
HASH_SEED = 0


def build(force: bool = False) -> str:
    """Compile hj_oracle.c into _build/liboracle.so (gcc, -O2, portable flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i64, vp, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            lib.oracle_mix_a.restype = u64
            lib.oracle_mix_a.argtypes = [u64]
            lib.oracle_mix_b.restype = u64
            lib.oracle_mix_b.argtypes = [u64]
            lib.oracle_murmur2_32.restype = ctypes.c_uint32
            lib.oracle_murmur2_32.argtypes = [vp, i32, ctypes.c_uint32]
            lib.oracle_murmur64a.restype = u64
            lib.oracle_murmur64a.argtypes = [vp, i32, u64]
            lib.oracle_key_hash.restype = u64
            lib.oracle_key_hash.argtypes = [u64, i32, u64]
            for name in ("oracle_hash_join", "oracle_nested_loop_join"):
                f = getattr(lib, name)
                f.restype = i64
                f.argtypes = [i32, vp, u64, vp, u64, vp, vp, u64]
            lib.oracle_count_sortmerge.restype = i64
            lib.oracle_count_sortmerge.argtypes = [i32, vp, u64, vp, u64, vp]
            lib.oracle_checksum_pairs.restype = None
            lib.oracle_checksum_pairs.argtypes = [u64, vp, vp, vp]
            lib.oracle_join_aggregate.restype = i64
            lib.oracle_join_aggregate.argtypes = [i32, vp, u64, vp, u64, vp, vp]
            lib.oracle_radix_partition.restype = i64
            lib.oracle_radix_partition.argtypes = [i32, vp, u64, i32, i32, u64, vp, vp]
            _lib = lib
    return _lib


def _rel(a: np.ndarray) -> tuple[np.ndarray, int]:
    a = np.ascontiguousarray(a)
    if a.ndim != 2 or a.shape[1] != 2 or a.dtype not in (np.uint32, np.uint64):
        raise ValueError("relation must be an (n, 2) uint32 or uint64 array")
    return a, a.dtype.itemsize


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def mix_a(x: int) -> int:
    return int(_load().oracle_mix_a(x))


def mix_b(x: int) -> int:
    return int(_load().oracle_mix_b(x))


def murmur2_32(data: bytes, seed: int) -> int:
    buf = ctypes.create_string_buffer(data, len(data) or 1)
    return int(_load().oracle_murmur2_32(buf, len(data), seed))


def murmur64a(data: bytes, seed: int) -> int:
    buf = ctypes.create_string_buffer(data, len(data) or 1)
    return int(_load().oracle_murmur64a(buf, len(data), seed))


def key_hash(key: int, width: int, seed: int = HASH_SEED) -> int:
    return int(_load().oracle_key_hash(key, width, seed))


def _join(fn_name: str, R: np.ndarray, S: np.ndarray, cap_hint: int | None = None):
    R, w = _rel(R)
    S, w2 = _rel(S)
    if w != w2:
        raise ValueError("R and S must have the same width")
    fn = getattr(_load(), fn_name)
    cap = 0 if cap_hint is None else int(cap_hint)
    rr = np.empty(cap, np.uint64)
    ss = np.empty(cap, np.uint64)
    n = fn(w, _ptr(R), len(R), _ptr(S), len(S), _ptr(rr), _ptr(ss), cap)
    if n < 0:
        raise MemoryError(fn_name)
    if n <= cap:
        return rr[:n], ss[:n]
    rr = np.empty(n, np.uint64)
    ss = np.empty(n, np.uint64)
    n2 = fn(w, _ptr(R), len(R), _ptr(S), len(S), _ptr(rr), _ptr(ss), n)
    assert n2 == n
    return rr, ss


def hash_join(R: np.ndarray, S: np.ndarray, cap_hint: int | None = None):
    """Pairs (rid_R, rid_S) of R join S on key, in probe order (two uint64 arrays).
    With cap_hint >= the pair count the join runs once; otherwise it counts first."""
    return _join("oracle_hash_join", R, S, cap_hint)


def nested_loop_join(R: np.ndarray, S: np.ndarray):
    """The same pairs by comparing every (r, s); tiny inputs only."""
    return _join("oracle_nested_loop_join", R, S)


def count_sortmerge(R: np.ndarray, S: np.ndarray) -> int:
    R, w = _rel(R)
    S, _ = _rel(S)
    out = np.zeros(1, np.uint64)
    if _load().oracle_count_sortmerge(w, _ptr(R), len(R), _ptr(S), len(S), _ptr(out)) < 0:
        raise MemoryError("count_sortmerge")
    return int(out[0])


def checksum_pairs(rid_r: np.ndarray, rid_s: np.ndarray) -> tuple[int, int]:
    rr = np.ascontiguousarray(rid_r, dtype=np.uint64)
    ss = np.ascontiguousarray(rid_s, dtype=np.uint64)
    out = np.zeros(2, np.uint64)
    _load().oracle_checksum_pairs(len(rr), _ptr(rr), _ptr(ss), _ptr(out))
    return int(out[0]), int(out[1])


def join_aggregate(R: np.ndarray, S: np.ndarray) -> tuple[int, int, int]:
    """(count, c0, c1) of R join S by per-key grouping, no pairs formed."""
    R, w = _rel(R)
    S, _ = _rel(S)
    cnt = np.zeros(1, np.uint64)
    c = np.zeros(2, np.uint64)
    if _load().oracle_join_aggregate(w, _ptr(R), len(R), _ptr(S), len(S), _ptr(cnt), _ptr(c)) < 0:
        raise MemoryError("join_aggregate")
    return int(cnt[0]), int(c[0]), int(c[1])


def radix_partition(rel: np.ndarray, b1: int, b2: int = 0, seed: int = HASH_SEED):
    """Stable radix partition on MurmurHash2 bits (Alg. 2); returns (tuples, offsets)."""
    rel, w = _rel(rel)
    out = np.empty_like(rel)
    offs = np.empty((1 << (b1 + b2)) + 1, np.uint64)
    if _load().oracle_radix_partition(w, _ptr(rel), len(rel), b1, b2, seed, _ptr(out), _ptr(offs)) < 0:
        raise ValueError("radix_partition")
    return out, offs


def sorted_pairs(rid_r: np.ndarray, rid_s: np.ndarray) -> np.ndarray:
    """Canonical form of a pair multiset: (n, 2) uint64 rows sorted by (rid_R, rid_S)."""
    rr = np.asarray(rid_r, np.uint64)
    ss = np.asarray(rid_s, np.uint64)
    order = np.lexsort((ss, rr))
    return np.stack([rr[order], ss[order]], axis=1)
