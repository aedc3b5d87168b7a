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


def _one_table(n: int, dev):
    """Layout arrays of a batch of one table of n entries: first positions
    (uint64[2], padded = unpadded) and its length (uint32[1])."""
    import torch
    beg = torch.from_numpy(np.array([0, n], dtype=np.uint64).view(np.int64)).to(dev)
    ln = torch.from_numpy(np.array([n], dtype=np.uint32).view(np.int32)).to(dev)
    return beg, ln


def uniform_keys_u32(n: int, seed: int, device="cuda", stream=None):
    """datagen.uniform_keys_u32(n, seed) drawn on the device (CUDA uint32 tensor)."""
    import torch
    assert 0 <= n < (1 << 32)
    out = torch.empty(n + 4, dtype=torch.uint32, device=device)[:n]
    beg, ln = _one_table(n, out.device)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    rc = load().hgd_batched_keys_u32(seed, 1, beg.data_ptr(), beg.data_ptr(), ln.data_ptr(), n, out.data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"hgd_batched_keys_u32: CUDA error {rc}")
    torch.cuda.current_stream().synchronize()
    return out


def queries_u32(q: int, keys, hit_rate: float, seed: int, stream=None):
    """datagen.queries_u32(q, keys, hit_rate, seed) drawn on the device from
    the device key tensor (CUDA uint32 tensor)."""
    import torch
    n = keys.numel()
    assert 0 <= q < (1 << 32) and n < (1 << 32)
    out = torch.empty(q + 4, dtype=torch.uint32, device=keys.device)[:q]
    qbeg, qln = _one_table(q, keys.device)
    kbeg, kln = _one_table(n, keys.device)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    rc = load().hgd_batched_queries_u32(seed, hit_rate, 1, qbeg.data_ptr(), qbeg.data_ptr(), qln.data_ptr(),
                                        kbeg.data_ptr(), kln.data_ptr(), keys.data_ptr(), q, out.data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"hgd_batched_queries_u32: CUDA error {rc}")
    torch.cuda.current_stream().synchronize()
    return out
