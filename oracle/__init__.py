"""HashGraph CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python front end (ctypes + numpy) of ``hg_oracle.cpp``: a plain,
single-threaded restatement of the method's results, used only by
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py``.  The product path (``paper_1907_02900_gb300``) never imports
this package.

Functions and the paper passage each follows:
  murmur3_x86_32      Section 2 "Hashing" (Eq. 1 names Murmur hashing)
  buckets             Eq. 1, hash(a) mod V; or the learned map (not in the paper)
  bucket_counts       the bucket histogram the build's prefix sum turns into offsets
  build               Alg. 1 / Alg. 2 / Section 3.1: CSR with V+1 offsets and
                      N (key, id) edges, grouped by bucket; canonical order
                      inside a bucket = ascending input position
  probe               Section 3.4, HashGraph-Probe-Standard (count all instances)
  multiplicity        table-free definition of the probe result (pin)
  join_count          Alg. 3, HashGraph-Probe-New, per-bucket intersection sizes
  join_size_by_keys   closed form sum_k m_A(k) m_B(k) (pin)
  join_materialize    Alg. 3 with the pairs written out in canonical order
The learned-map functions live in ``oracle.learned``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle_hg.so")
_SOURCES = ["hg_oracle.cpp", "hg_oracle_learned.cpp"]
_lib = None

KEY_U32 = 0
KEY_U64 = 1
MAP_MURMUR3 = 0
MAP_LEARNED = 1


def build_oracle(force: bool = False) -> str:
    """Compile the oracle into oracle/lib/liboracle_hg.so (g++, -O2, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(_LIBPATH):
        t = os.path.getmtime(_LIBPATH)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return _LIBPATH
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = ctypes.CDLL(_LIBPATH)
        vp, u64, i64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
        L.orc_murmur3_x86_32.restype = u32
        L.orc_murmur3_x86_32.argtypes = [vp, u64, u32]
        L.orc_hash_keys.restype = None
        L.orc_hash_keys.argtypes = [i32, vp, u64, u32, vp]
        L.orc_bucket_keys.restype = i32
        L.orc_bucket_keys.argtypes = [i32, vp, u64, i32, u32, u64, vp, vp]
        L.orc_bucket_counts.restype = i32
        L.orc_bucket_counts.argtypes = [i32, vp, u64, i32, u32, u64, vp, vp]
        L.orc_build.restype = i32
        L.orc_build.argtypes = [i32, vp, vp, u64, i32, u32, u64, vp, vp, vp, vp]
        L.orc_probe.restype = i32
        L.orc_probe.argtypes = [i32, vp, vp, u64, i32, u32, u64, vp, vp, u64, vp]
        L.orc_multiplicity.restype = None
        L.orc_multiplicity.argtypes = [i32, vp, u64, vp, u64, vp]
        L.orc_join_count.restype = i32
        L.orc_join_count.argtypes = [i32, vp, vp, vp, vp, u64, vp, vp]
        L.orc_join_size_by_keys.restype = i64
        L.orc_join_size_by_keys.argtypes = [i32, vp, u64, vp, u64]
        L.orc_join_materialize.restype = i64
        L.orc_join_materialize.argtypes = [i32, vp, vp, vp, vp, vp, vp, u64, vp, vp, i64]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _key_type(keys: np.ndarray) -> int:
    if keys.dtype == np.uint32:
        return KEY_U32
    if keys.dtype == np.uint64:
        return KEY_U64
    raise TypeError(f"keys must be uint32 or uint64, got {keys.dtype}")


def murmur3_x86_32(data: bytes, seed: int = 0) -> int:
    buf = np.frombuffer(bytes(data) + b"\0", dtype=np.uint8)
    return int(lib().orc_murmur3_x86_32(_ptr(buf), len(data), seed & 0xFFFFFFFF))


def hash_keys(keys: np.ndarray, seed: int = 0) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    out = np.empty(len(keys), dtype=np.uint32)
    lib().orc_hash_keys(_key_type(keys), _ptr(keys), len(keys), seed & 0xFFFFFFFF, _ptr(out))
    return out


def buckets(keys: np.ndarray, V: int, seed: int = 0, model: np.ndarray | None = None) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    out = np.empty(len(keys), dtype=np.uint64)
    kind = MAP_LEARNED if model is not None else MAP_MURMUR3
    rc = lib().orc_bucket_keys(_key_type(keys), _ptr(keys), len(keys), kind, seed & 0xFFFFFFFF, V,
                               _ptr(model), _ptr(out))
    if rc:
        raise ValueError("invalid bucket map")
    return out


def bucket_counts(keys: np.ndarray, V: int, seed: int = 0, model: np.ndarray | None = None) -> np.ndarray:
    """uint32[V]: number of keys in each bucket (the histogram under the CSR offsets)."""
    keys = np.ascontiguousarray(keys)
    out = np.empty(V, dtype=np.uint32)
    kind = MAP_LEARNED if model is not None else MAP_MURMUR3
    rc = lib().orc_bucket_counts(_key_type(keys), _ptr(keys), len(keys), kind, seed & 0xFFFFFFFF, V, _ptr(model),
                                 _ptr(out))
    if rc:
        raise ValueError("invalid bucket map")
    return out


def build(keys: np.ndarray, V: int, seed: int = 0, ids: np.ndarray | None = None,
          model: np.ndarray | None = None):
    """Returns (offsets uint32[V+1], csr_keys, csr_ids uint32[n])."""
    keys = np.ascontiguousarray(keys)
    n = len(keys)
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
    offsets = np.empty(V + 1, dtype=np.uint32)
    ck = np.empty(n, dtype=keys.dtype)
    ci = np.empty(n, dtype=np.uint32)
    kind = MAP_LEARNED if model is not None else MAP_MURMUR3
    rc = lib().orc_build(_key_type(keys), _ptr(keys), _ptr(ids), n, kind, seed & 0xFFFFFFFF, V,
                         _ptr(model), _ptr(offsets), _ptr(ck), _ptr(ci))
    if rc:
        raise ValueError("invalid bucket map")
    return offsets, ck, ci


def probe(offsets, csr_keys, queries, V: int, seed: int = 0, model=None) -> np.ndarray:
    queries = np.ascontiguousarray(queries, dtype=csr_keys.dtype)
    out = np.empty(len(queries), dtype=np.uint32)
    kind = MAP_LEARNED if model is not None else MAP_MURMUR3
    rc = lib().orc_probe(_key_type(csr_keys), _ptr(offsets), _ptr(csr_keys), len(csr_keys), kind,
                         seed & 0xFFFFFFFF, V, _ptr(model), _ptr(queries), len(queries), _ptr(out))
    if rc:
        raise ValueError("invalid bucket map")
    return out


def multiplicity(keys: np.ndarray, queries: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    queries = np.ascontiguousarray(queries, dtype=keys.dtype)
    out = np.empty(len(queries), dtype=np.uint32)
    lib().orc_multiplicity(_key_type(keys), _ptr(keys), len(keys), _ptr(queries), len(queries), _ptr(out))
    return out


def join_count(offA, keysA, offB, keysB, V: int):
    """Returns (total, per-bucket counts int64[V])."""
    bc = np.empty(V, dtype=np.int64)
    tot = np.zeros(1, dtype=np.int64)
    lib().orc_join_count(_key_type(keysA), _ptr(offA), _ptr(keysA), _ptr(offB), _ptr(keysB), V,
                         _ptr(bc), _ptr(tot))
    return int(tot[0]), bc


def join_size_by_keys(keysA, keysB) -> int:
    keysA = np.ascontiguousarray(keysA)
    keysB = np.ascontiguousarray(keysB, dtype=keysA.dtype)
    return int(lib().orc_join_size_by_keys(_key_type(keysA), _ptr(keysA), len(keysA), _ptr(keysB), len(keysB)))


def join_materialize(offA, keysA, idsA, offB, keysB, idsB, V: int, cap: int | None = None):
    """Returns (pairs_a int64[M], pairs_b int64[M]) in canonical order."""
    if cap is None:
        cap, _ = join_count(offA, keysA, offB, keysB, V)
    oa = np.empty(max(cap, 1), dtype=np.int64)
    ob = np.empty(max(cap, 1), dtype=np.int64)
    m = lib().orc_join_materialize(_key_type(keysA), _ptr(offA), _ptr(keysA), _ptr(idsA), _ptr(offB),
                                   _ptr(keysB), _ptr(idsB), V, _ptr(oa), _ptr(ob), cap)
    m = int(min(m, cap))
    return oa[:m], ob[:m]


def check_table(offsets, csr_keys, csr_ids, keys, V, seed=0, model=None, ids=None):
    """Structural invariants of a HashGraph table (Section 3.1-3.2): offsets
    monotone from 0 to n, every edge lies in the bucket its key maps to, the
    ids form the expected permutation and ascend inside each bucket.
    Returns a list of violated invariants (empty when the table is valid)."""
    errs = []
    n = len(keys)
    offsets = np.asarray(offsets, dtype=np.int64)
    if len(offsets) != V + 1:
        errs.append("offsets length")
        return errs
    if offsets[0] != 0 or offsets[-1] != n:
        errs.append("offsets endpoints")
    if np.any(np.diff(offsets) < 0):
        errs.append("offsets not monotone")
    if errs:
        return errs
    b = buckets(csr_keys, V, seed, model)
    owner = np.repeat(np.arange(V, dtype=np.uint64), np.diff(offsets))
    if not np.array_equal(b, owner):
        errs.append("edge outside its hashed bucket")
    pos = np.asarray(csr_ids, dtype=np.int64) if ids is None else None
    if ids is None:
        if not np.array_equal(np.sort(pos), np.arange(n)):
            errs.append("ids not a permutation")
        elif not np.array_equal(np.asarray(keys)[pos], csr_keys):
            errs.append("key/id mismatch")
        same = owner[1:] == owner[:-1]
        if np.any(pos[1:][same] <= pos[:-1][same]):
            errs.append("ids not ascending inside a bucket")
    return errs
