"""GPU copy of the batched input recipes of ``datagen`` (libhg_datagen.so).

Draws the same numbers as ``datagen.batched_keys_u32`` and
``datagen.batched_queries_u32`` directly into the padded batched layout on
the device, for batches too large to draw on the host quickly.  Inputs only:
nothing here belongs to the hash-table method.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def load():
    global _lib
    if _lib is None:
        path = os.path.join(_HERE, "lib", "libhg_datagen.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1907_02900_gb300._build.build()")
        L = ctypes.CDLL(path)
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        L.hgd_batched_keys_u32.restype = i32
        L.hgd_batched_keys_u32.argtypes = [u64, u32, vp, vp, vp, u64, vp, vp]
        L.hgd_batched_queries_u32.restype = i32
        L.hgd_batched_queries_u32.argtypes = [u64, ctypes.c_double, u32, vp, vp, vp, vp, vp, vp, u64, vp, vp]
        _lib = L
    return _lib


def fill_batch(plan, bufs: dict, key_seed: int, query_seed: int, hit_rate: float = 0.5, stream=None):
    """Write the keys and queries of every table of ``plan`` into ``bufs``."""
    import torch
    dev = bufs["keys"].device
    T = plan.T
    ub = np.concatenate([[0], np.cumsum(plan.sizes.astype(np.uint64))]).astype(np.uint64)
    qub = np.concatenate([[0], np.cumsum(plan.qsizes.astype(np.uint64))]).astype(np.uint64)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a).astype(dt)).to(dev)
    kp, ku, kl = t(plan.key_begin, np.uint64), t(ub, np.uint64), t(plan.sizes, np.uint32)
    qp, qu, ql = t(plan.query_begin, np.uint64), t(qub, np.uint64), t(plan.qsizes, np.uint32)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    L = load()
    rc = L.hgd_batched_keys_u32(key_seed, T, kp.data_ptr(), ku.data_ptr(), kl.data_ptr(), plan.total_keys,
                                bufs["keys"].data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"hgd_batched_keys_u32: CUDA error {rc}")
    rc = L.hgd_batched_queries_u32(query_seed, hit_rate, T, qp.data_ptr(), qu.data_ptr(), ql.data_ptr(),
                                   kp.data_ptr(), kl.data_ptr(), bufs["keys"].data_ptr(), plan.total_queries,
                                   bufs["queries"].data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"hgd_batched_queries_u32: CUDA error {rc}")
    torch.cuda.current_stream().synchronize()
