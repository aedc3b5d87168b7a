"""Learned bucket map, CPU oracle side -- TEST INFRASTRUCTURE ONLY.

ctypes front end of ``hg_oracle_learned.cpp`` plus the model-blob writer.
The learned map is not in the paper (Section 2 hashes with Murmur); see the
C++ file for the model: a linear root over a monotone feature picks one of L
leaves, and leaf j maps its key range linearly between knot values Y_j and
Y_{j+1} (a continuous piecewise-linear CDF in bucket units).

Blob layout (little-endian), shared by both sides as a file format:
  header 32 B: u32 magic 'HGLM', u32 L, u64 V, f32 a, f32 b, u32 key_type, u32 flags
  leaf   24 B: u64 xmin, f32 slope, f32 icpt, u32 base, u32 width
"""
from __future__ import annotations

import ctypes
import math
import struct

import numpy as np

from . import _ptr, lib as _baselib

MAGIC = 0x4D4C4748
SAMPLE_STREAM = 0x4C4541524E

_sig_done = False


def lib():
    global _sig_done
    L = _baselib()
    if not _sig_done:
        vp, u64, u32, i32, f32, f64 = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                       ctypes.c_float, ctypes.c_double)
        L.orc_rmi_sample_indices.restype = None
        L.orc_rmi_sample_indices.argtypes = [u64, u64, u64, vp]
        L.orc_rmi_sorted_sample.restype = None
        L.orc_rmi_sorted_sample.argtypes = [i32, vp, u64, u64, u64, vp]
        L.orc_rmi_root_leaf.restype = u32
        L.orc_rmi_root_leaf.argtypes = [f32, f32, u32, i32, u64]
        L.orc_rmi_knots.restype = u32
        L.orc_rmi_knots.argtypes = [f32, f32, u32, i32, vp]
        L.orc_rmi_leaf_loss_grad.restype = f64
        L.orc_rmi_leaf_loss_grad.argtypes = [i32, vp, u64, u64, f32, f32, u32, vp, u32, vp, vp, f64, vp, vp]
        L.orc_rmi_leaf_lsq.restype = None
        L.orc_rmi_leaf_lsq.argtypes = [i32, vp, u64, u64, f32, f32, u32, vp, u32, vp, f64, vp]
        L.orc_rmi_leaf_train.restype = None
        L.orc_rmi_leaf_train.argtypes = [i32, vp, u64, u64, f32, f32, u32, vp, u32, vp, f64, f64, u32, f64, vp]
        L.orc_rmi_leaf_init.restype = None
        L.orc_rmi_leaf_init.argtypes = [i32, vp, u64, u64, u32, vp, u32, vp]
        L.orc_rmi_leaf_project.restype = None
        L.orc_rmi_leaf_project.argtypes = [u64, u32, u32, vp, f64, vp]
        L.orc_rmi_root_lsq.restype = None
        L.orc_rmi_root_lsq.argtypes = [i32, vp, u64, u32, vp]
        L.orc_rmi_root_loss_grad.restype = f64
        L.orc_rmi_root_loss_grad.argtypes = [i32, vp, u64, u32, f64, f64, vp]
        _sig_done = True
    return L


def _kt(dtype) -> int:
    return 0 if np.dtype(dtype) == np.uint32 else 1


def sample_indices(n: int, S: int, seed: int) -> np.ndarray:
    out = np.empty(S, dtype=np.uint64)
    lib().orc_rmi_sample_indices(n, S, seed, _ptr(out))
    return out


def sorted_sample(keys: np.ndarray, S: int, seed: int) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    out = np.empty(S, dtype=np.uint64)
    lib().orc_rmi_sorted_sample(_kt(keys.dtype), _ptr(keys), len(keys), S, seed, _ptr(out))
    return out


def root_leaf(a: float, b: float, L: int, key_type: int, key: int) -> int:
    return int(lib().orc_rmi_root_leaf(a, b, L, key_type, key))


def knots(a: float, b: float, L: int, key_type: int):
    """(kb uint64[L+1], J) for the fp32 root (a, b)."""
    kb = np.empty(L + 1, dtype=np.uint64)
    J = lib().orc_rmi_knots(a, b, L, key_type, _ptr(kb))
    return kb, int(J)


RIDGE = 1.0        # rho: knot-value ridge, in units of one sample's squared error
MIN_WIDTH = 0.5    # gamma: a leaf keeps at least this share of its prior width
ETA = 0.9          # Jacobi step size
ITERS = 40         # default number of training rounds


def leaf_init(x: np.ndarray, V: int, L: int, kb: np.ndarray, J: int, key_type: int = 1) -> np.ndarray:
    """Prior knot values: the sample's rank-target interpolant at the knots."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    kb = np.ascontiguousarray(kb, dtype=np.uint64)
    Y = np.empty(L + 1, dtype=np.float64)
    lib().orc_rmi_leaf_init(key_type, _ptr(x), len(x), V, L, _ptr(kb), J, _ptr(Y))
    return Y


def leaf_project(V: int, L: int, J: int, Y0: np.ndarray, Y: np.ndarray, gamma: float = MIN_WIDTH) -> np.ndarray:
    Y0 = np.ascontiguousarray(Y0, dtype=np.float64)
    out = np.array(Y, dtype=np.float64, copy=True)
    lib().orc_rmi_leaf_project(V, L, J, _ptr(Y0), gamma, _ptr(out))
    return out


def leaf_loss_grad(key_type: int, x: np.ndarray, V: int, a: float, b: float, L: int, kb: np.ndarray, J: int,
                   Y: np.ndarray, Y0: np.ndarray | None = None, rho: float = RIDGE):
    """(loss, grad[L+1], hessian diagonal[L+1]) in double; Y0 defaults to the
    initial knot values of the sample."""
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    if Y0 is None:
        Y0 = leaf_init(x, V, L, kb, J, key_type)
    Y0 = np.ascontiguousarray(Y0, dtype=np.float64)
    g = np.empty(L + 1)
    d = np.empty(L + 1)
    loss = lib().orc_rmi_leaf_loss_grad(key_type, _ptr(x), len(x), V, a, b, L, _ptr(kb), J, _ptr(Y), _ptr(Y0), rho,
                                        _ptr(g), _ptr(d))
    return float(loss), g, d


def leaf_lsq(key_type: int, x: np.ndarray, V: int, a: float, b: float, L: int, kb: np.ndarray, J: int,
             Y_init: np.ndarray, rho: float = RIDGE) -> np.ndarray:
    Y_init = np.ascontiguousarray(Y_init, dtype=np.float64)
    out = np.empty(L + 1)
    lib().orc_rmi_leaf_lsq(key_type, _ptr(x), len(x), V, a, b, L, _ptr(kb), J, _ptr(Y_init), rho, _ptr(out))
    return out


def leaf_train(key_type: int, x: np.ndarray, V: int, a: float, b: float, L: int, kb: np.ndarray, J: int,
               Y0: np.ndarray, iters: int = ITERS, eta: float = ETA, rho: float = RIDGE,
               gamma: float = MIN_WIDTH) -> np.ndarray:
    """Knot values after `iters` rounds of (Jacobi step, projection) from Y0."""
    Y0 = np.ascontiguousarray(Y0, dtype=np.float64)
    out = np.empty(L + 1)
    lib().orc_rmi_leaf_train(key_type, _ptr(x), len(x), V, a, b, L, _ptr(kb), J, _ptr(Y0), rho, gamma, iters, eta,
                             _ptr(out))
    return out


def root_lsq(key_type: int, x: np.ndarray, L: int):
    ab = np.empty(2)
    lib().orc_rmi_root_lsq(key_type, _ptr(x), len(x), L, _ptr(ab))
    return float(ab[0]), float(ab[1])


def root_loss_grad(key_type: int, x: np.ndarray, L: int, a: float, b: float):
    g = np.empty(2)
    loss = lib().orc_rmi_root_loss_grad(key_type, _ptr(x), len(x), L, a, b, _ptr(g))
    return float(loss), g


def make_blob(a: float, b: float, key_type: int, V: int, kb: np.ndarray, J: int, Y: np.ndarray) -> np.ndarray:
    """Model blob from the root and the knot values: leaf j (j <= J) has
    base = floor(Y_j), icpt = Y_j - base, slope = (Y_{j+1} - Y_j) / width_keys,
    width = base_{j+1} - base_j, xmin = kb_j; leaves above J are empty."""
    L = len(kb) - 1
    kmax = 0xFFFFFFFF if key_type == 0 else (1 << 64) - 1
    Yc = np.minimum(np.maximum.accumulate(np.clip(np.asarray(Y, dtype=np.float64), 0.0, float(V))), float(V))
    base = np.floor(Yc).astype(np.uint64)
    buf = bytearray(32 + 24 * L)
    struct.pack_into("<IIQffII", buf, 0, MAGIC, L, V, np.float32(a), np.float32(b), key_type, 0)
    for j in range(L):
        if j <= J:
            wkeys = float(int(kb[j + 1]) - int(kb[j])) if j < J else float(kmax - int(kb[j])) + 1.0
            nb = int(base[j + 1]) if j < J else V
            slope = (Yc[j + 1] - Yc[j]) / wkeys if wkeys > 0 and j < J else ((V - Yc[j]) / wkeys if wkeys > 0 else 0.0)
            icpt = Yc[j] - float(base[j])
            width = nb - int(base[j])
            struct.pack_into("<QffII", buf, 32 + 24 * j, int(kb[j]), np.float32(slope), np.float32(icpt),
                             int(base[j]), width)
        else:
            struct.pack_into("<QffII", buf, 32 + 24 * j, kmax, 0.0, 0.0, V, 0)
    return np.frombuffer(bytes(buf), dtype=np.uint8).copy()
