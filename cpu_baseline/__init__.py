"""Multithreaded CPU HashGraph (OpenMP), a CPU comparison point for the GPU
path: HashGraph-V2 build (Alg. 2) and HashGraph-Probe-Standard (Section 3.4)
over all host cores.  It produces the same canonical table as the GPU build
and the oracle, and shares no code with either; the GPU path never imports
it.  ``bench.py`` reports its rate beside the single-threaded oracle's.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "lib", "libhg_cpu_mt.so")
_SRC = os.path.join(_HERE, "hg_cpu_mt.cpp")
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile hg_cpu_mt.cpp into cpu_baseline/lib/libhg_cpu_mt.so (g++ -O3 -fopenmp)."""
    if not force and os.path.exists(_LIBPATH) and os.path.getmtime(_LIBPATH) >= os.path.getmtime(_SRC):
        return _LIBPATH
    os.makedirs(os.path.dirname(_LIBPATH), exist_ok=True)
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_lib())
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        L.hgcpu_build.argtypes = [i32, vp, vp, u64, u64, u32, vp, vp, vp, i32]
        L.hgcpu_build.restype = i32
        L.hgcpu_probe.argtypes = [i32, vp, vp, u64, u32, vp, u64, vp, i32]
        L.hgcpu_probe.restype = i32
        L.hgcpu_max_threads.argtypes = []
        L.hgcpu_max_threads.restype = i32
        _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().hgcpu_max_threads())


def _key_type(a: np.ndarray) -> int:
    if a.dtype == np.uint32:
        return 0
    if a.dtype == np.uint64:
        return 1
    raise TypeError(f"keys must be uint32 or uint64, got {a.dtype}")


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def build(keys: np.ndarray, V: int, seed: int = 0, ids: np.ndarray | None = None, threads: int = 0):
    """(offsets[V+1] uint32, csr_keys[n], csr_ids[n] uint32) of the canonical table."""
    keys = np.ascontiguousarray(keys)
    kt = _key_type(keys)
    n = len(keys)
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        if len(ids) != n:
            raise ValueError("ids must have one entry per key")
    off = np.empty(int(V) + 1, dtype=np.uint32)
    ck = np.empty(n, dtype=keys.dtype)
    ci = np.empty(n, dtype=np.uint32)
    rc = lib().hgcpu_build(kt, _p(keys), _p(ids), n, int(V), seed & 0xFFFFFFFF, _p(off), _p(ck), _p(ci), threads)
    if rc != 0:
        raise ValueError(f"hgcpu_build: invalid argument (n={n}, V={V})")
    return off, ck, ci


def probe(offsets: np.ndarray, csr_keys: np.ndarray, V: int, queries: np.ndarray, seed: int = 0,
          threads: int = 0) -> np.ndarray:
    """uint32 count of equal keys in each query's bucket."""
    queries = np.ascontiguousarray(queries, dtype=csr_keys.dtype)
    counts = np.empty(len(queries), dtype=np.uint32)
    rc = lib().hgcpu_probe(_key_type(csr_keys), _p(offsets), _p(csr_keys), int(V), seed & 0xFFFFFFFF,
                           _p(queries), len(queries), _p(counts), threads)
    if rc != 0:
        raise ValueError(f"hgcpu_probe: invalid argument (V={V})")
    return counts
