"""Helpers shared by the GPU tests: host<->device copies that keep unsigned
dtypes intact, and sampled oracle checks for tables too large for the full
oracle."""
import numpy as np

_SIGNED = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}


def to_dev(a: np.ndarray):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype in _SIGNED:
        t = torch.from_numpy(a.view(_SIGNED[a.dtype])).cuda()
        return t.view(torch.uint32 if a.dtype == np.uint32 else torch.uint64)
    return torch.from_numpy(a).cuda()


def to_np(t) -> np.ndarray:
    import torch
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    if t.dtype == torch.uint64:
        return t.view(torch.int64).cpu().numpy().view(np.uint64)
    return t.cpu().numpy()


def table_np(t):
    return to_np(t.offsets), to_np(t.keys), to_np(t.ids)


def sampled_reference(orc, keys: np.ndarray, V: int, seed: int, sample_buckets: np.ndarray, model=None):
    """Oracle facts of a large table without building it:
    the full offsets array (exclusive prefix of the bucket histogram, i.e.
    offsets[v] = #{i : bucket(key_i) < v}) and, for each sampled bucket, its
    keys and ids in canonical order (ascending input position)."""
    b = orc.buckets(keys, V, seed, model)
    counts = np.bincount(b.astype(np.int64), minlength=V)
    offsets = np.zeros(V + 1, dtype=np.uint64)
    np.cumsum(counts, out=offsets[1:])
    mark = np.zeros(V, dtype=bool)
    mark[sample_buckets.astype(np.int64)] = True
    pos = np.nonzero(mark[b.astype(np.int64)])[0]
    bsel = b[pos]
    order = np.argsort(bsel, kind="stable")
    pos, bsel = pos[order], bsel[order]
    segs = {}
    starts = np.searchsorted(bsel, sample_buckets.astype(np.uint64), side="left")
    ends = np.searchsorted(bsel, sample_buckets.astype(np.uint64), side="right")
    for v, s, e in zip(sample_buckets.tolist(), starts, ends):
        p = pos[s:e]
        segs[int(v)] = (keys[p], p.astype(np.uint32))
    return offsets.astype(np.uint32), segs, b
