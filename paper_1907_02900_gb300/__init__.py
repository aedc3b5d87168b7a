"""GB300-native HashGraph (Green, arXiv 1907.02900): Python binding of libhg.so.

This module only marshals arguments: it allocates outputs and workspaces
with PyTorch (device memory and streams are PyTorch's plumbing) and calls the
C ABI declared in include/hg.h, where every step of the method runs as
hand-written sm_103a CUDA.  There is no CPU fallback: if the CUDA library is
missing or no GPU is present, calls raise.

    import paper_1907_02900_gb300 as hg
    t = hg.build(keys, num_buckets=1 << 20)          # keys: CUDA uint32/uint64 tensor
    counts = hg.probe(t, queries)                    # per-query match counts
    total, per_bucket = hg.join_count(tA, tB)        # Alg. 3 (same V and map)
    a_ids, b_ids = hg.join_materialize(tA, tB)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBDIR = os.path.join(_HERE, "lib")
LIBPATH = os.path.join(LIBDIR, "libhg.so")

HG_OK = 0
STATUS_NAMES = {0: "HG_OK", 1: "HG_ERR_INVALID_ARG", 2: "HG_ERR_WORKSPACE_TOO_SMALL", 3: "HG_ERR_OVERFLOW",
                4: "HG_ERR_CUDA", 5: "HG_ERR_TIMEOUT", 6: "HG_ERR_MODEL", 7: "HG_ERR_UNSUPPORTED"}
KEY_U32, KEY_U64 = 0, 1
MAP_MURMUR3, MAP_LEARNED = 0, 1
ALGOS = {"auto": 0, "v1": 1, "v2": 2}


class HGError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}")
        self.code = code


class hg_config(ctypes.Structure):
    _fields_ = [("key_type", ctypes.c_int32), ("map", ctypes.c_int32), ("num_buckets", ctypes.c_uint64),
                ("seed", ctypes.c_uint32), ("algo", ctypes.c_int32), ("d_model", ctypes.c_void_p),
                ("bin_shift", ctypes.c_uint32), ("threads_per_bin", ctypes.c_uint32)]


class hg_table(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("d_offsets", ctypes.c_void_p), ("d_keys", ctypes.c_void_p),
                ("d_ids", ctypes.c_void_p)]


_lib = None

# Entry points and their ctypes signatures; every name here is declared in include/hg.h.
_VP, _SZ, _U64, _U32, _I32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
_CFGP, _TABP = ctypes.POINTER(hg_config), ctypes.POINTER(hg_table)
SIGNATURES = {
    "hg_version": (ctypes.c_char_p, []),
    "hg_status_string": (ctypes.c_char_p, [_I32]),
    "hg_build_workspace_size": (_SZ, [_CFGP, _U64]),
    "hg_build": (_I32, [_CFGP, _VP, _VP, _U64, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "hg_probe": (_I32, [_CFGP, _TABP, _VP, _U64, _VP, _VP]),
    "hg_probe_workspace_size": (_SZ, [_CFGP, _U64, _U64]),
    "hg_probe_binned": (_I32, [_CFGP, _TABP, _VP, _U64, _VP, _VP, _SZ, _VP]),
    "hg_learned_model_bytes": (_SZ, [_U32]),
    "hg_learned_workspace_size": (_SZ, [_I32, _U64, _U64, _U32]),
    "hg_learned_train": (_I32, [_I32, _VP, _U64, _U64, _U32, _U64, _U64, _U32, _VP, _VP, _VP, _SZ, _VP]),
    "hg_learned_sorted_sample": (_I32, [_I32, _VP, _U64, _U64, _U64, _VP, _VP, _SZ, _VP]),
    "hg_learned_root_grad": (_I32, [_I32, _VP, _U64, _U32, ctypes.c_double, ctypes.c_double, _VP, _VP, _SZ, _VP]),
    "hg_learned_leaf_grad": (_I32, [_I32, _VP, _U64, _U64, ctypes.c_float, ctypes.c_float, _U32, _VP, _VP, _VP,
                                    _VP, _VP, _SZ, _VP]),
    "hg_bucket_stats": (_I32, [_CFGP, _VP, _U64, _VP, _VP, _VP, _SZ, _VP]),
    "hg_learned_judge_workspace_size": (_SZ, []),
    "hg_learned_judge": (_I32, [_CFGP, _VP, _U64, ctypes.c_double, ctypes.c_double, _VP, _VP, _SZ, _VP, _VP, _VP]),
    "hg_batch_plan_create": (_I32, [_I32, _U32, _U32, _VP, _VP, _VP, ctypes.POINTER(_VP)]),
    "hg_batch_plan_destroy": (None, [_VP]),
    "hg_batch_layout": (_I32, [_VP, _VP, _VP, _VP, _VP]),
    "hg_batch_workspace_size": (_SZ, [_VP]),
    "hg_batch_set_config": (_I32, [_VP, _U32, _U32]),
    "hg_batch_get_config": (_I32, [_VP, _VP, _VP, _VP]),
    "hg_batch_run": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "hg_batch_autotune": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP, _U32, _VP]),
    "hg_batch_run_plain": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "hg_batch_run_eager": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "hg_static_scratch_bytes": (_SZ, []),
    "hg_build_static_scratch": (_I32, [_CFGP, _VP, _VP, _U64, _VP, _VP, _VP, _VP]),
    "hg_static_scratch_status": (_I32, [_VP]),
    "hg_build_probe_host": (_I32, [_CFGP, _VP, _U64, _VP, _U64, _VP, _VP, _VP, _VP, _TABP, _VP, _SZ, _VP, _SZ, _VP]),
    "hg_join_workspace_size": (_SZ, [_CFGP, _U64, _U64]),
    "hg_join_count": (_I32, [_CFGP, _TABP, _TABP, _VP, _VP, _VP, _SZ, _VP]),
    "hg_join_materialize": (_I32, [_CFGP, _TABP, _TABP, _VP, _VP, _U64, _VP, _VP, _SZ, _VP]),
    "hg_join_materialize_after_count": (_I32, [_CFGP, _TABP, _TABP, _VP, _VP, _U64, _VP, _VP, _SZ, _VP]),
    "hg_selftest_wait_timeout": (_I32, [_VP, _U32, _VP]),
    "hg_workspace_status": (_I32, [_VP, _VP]),
    "hg_workspace_clear": (_I32, [_VP, _VP]),
    "hg_profile_enable": (None, [ctypes.c_int]),
    "hg_profile_reset": (None, []),
    "hg_profile_read": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]),
}


def profile_enable(on: bool = True):
    load().hg_profile_enable(1 if on else 0)


def profile_reset():
    load().hg_profile_reset()


def profile_read() -> dict:
    """{kernel name: (total ms, launches)} of the launches recorded while tracing was on."""
    lib = load()
    n = lib.hg_profile_read(0, None, None, None)
    if n < 0:
        raise HGError(4, "hg_profile_read")
    names = (ctypes.c_char_p * max(n, 1))()
    ms = (ctypes.c_double * max(n, 1))()
    cnt = (ctypes.c_uint64 * max(n, 1))()
    n = lib.hg_profile_read(n, names, ms, cnt)
    return {names[i].decode(): (ms[i], int(cnt[i])) for i in range(n)}


def build_library(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)["libhg.so"]


def load(path: str | None = None):
    """Load libhg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("HG_LIBHG") or LIBPATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1907_02900_gb300._build.build() "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != HG_OK:
        raise HGError(code, where)


def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _key_type_of(t) -> int:
    torch = _torch()
    if t.dtype in (torch.uint32, torch.int32):
        return KEY_U32
    if t.dtype in (torch.uint64, torch.int64):
        return KEY_U64
    raise TypeError(f"keys must be 32- or 64-bit integers, got {t.dtype}")


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _require_cuda(t, name):
    if t is not None and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t is not None and not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def make_config(key_type: int, num_buckets: int, seed: int = 0, algo: str = "auto", model=None,
                bin_shift: int = 0) -> hg_config:
    c = hg_config()
    c.key_type = key_type
    c.map = MAP_LEARNED if model is not None else MAP_MURMUR3
    c.num_buckets = int(num_buckets)
    c.seed = seed & 0xFFFFFFFF
    c.algo = ALGOS[algo]
    c.d_model = _ptr(model)
    c.bin_shift = bin_shift
    c.threads_per_bin = 0
    return c


@dataclass
class Table:
    """A built HashGraph: offsets[V+1], keys[n], ids[n] (CUDA tensors) and its config."""
    offsets: object
    keys: object
    ids: object
    cfg: hg_config
    model: object = None

    @property
    def num_buckets(self) -> int:
        return int(self.cfg.num_buckets)

    def view(self) -> hg_table:
        t = hg_table()
        t.n = self.keys.numel()
        t.d_offsets = self.offsets.data_ptr()
        t.d_keys = self.keys.data_ptr()
        t.d_ids = self.ids.data_ptr()
        return t


def build_workspace_size(cfg: hg_config, n: int) -> int:
    return int(load().hg_build_workspace_size(ctypes.byref(cfg), n))


def build_into(cfg: hg_config, keys, ids, offsets, csr_keys, csr_ids, ws, stream=None):
    """hg_build on caller-provided tensors (no allocation)."""
    lib = load()
    rc = lib.hg_build(ctypes.byref(cfg), _ptr(keys), _ptr(ids), keys.numel(), _ptr(offsets), _ptr(csr_keys),
                      _ptr(csr_ids), _ptr(ws), ws.numel(), _stream_handle(stream))
    _check(rc, "hg_build")


def build(keys, num_buckets: int, ids=None, seed: int = 0, algo: str = "auto", model=None,
          bin_shift: int = 0, stream=None, ws=None) -> Table:
    """HashGraph build (Alg. 1 V1 / Alg. 2 V2) of a CUDA key tensor."""
    torch = _torch()
    _require_cuda(keys, "keys")
    _require_cuda(ids, "ids")
    if ids is not None and (ids.dtype not in (torch.uint32, torch.int32) or ids.numel() != keys.numel()):
        raise ValueError("ids must be a 32-bit integer tensor with one entry per key")
    kt = _key_type_of(keys)
    cfg = make_config(kt, num_buckets, seed, algo, model, bin_shift)
    n = keys.numel()
    dev = keys.device
    need = build_workspace_size(cfg, n)
    if need == 0:
        raise HGError(1, "hg_build_workspace_size")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    offsets = torch.empty(num_buckets + 1, dtype=torch.uint32, device=dev)
    csr_keys = torch.empty(n, dtype=keys.dtype, device=dev)
    csr_ids = torch.empty(n, dtype=torch.uint32, device=dev)
    build_into(cfg, keys, ids, offsets, csr_keys, csr_ids, ws, stream)
    return Table(offsets, csr_keys, csr_ids, cfg, model)


def probe_into(table: Table, queries, counts, stream=None):
    lib = load()
    tv = table.view()
    rc = lib.hg_probe(ctypes.byref(table.cfg), ctypes.byref(tv), _ptr(queries), queries.numel(), _ptr(counts),
                      _stream_handle(stream))
    _check(rc, "hg_probe")


BINNED_PROBE_MIN_QUERIES = 1 << 20


def probe_workspace_size(table: Table, q: int) -> int:
    return int(load().hg_probe_workspace_size(ctypes.byref(table.cfg), table.keys.numel(), q))


def probe_binned_into(table: Table, queries, counts, ws, stream=None):
    """hg_probe_binned on caller-provided tensors (no allocation)."""
    tv = table.view()
    rc = load().hg_probe_binned(ctypes.byref(table.cfg), ctypes.byref(tv), _ptr(queries), queries.numel(),
                                _ptr(counts), _ptr(ws), ws.numel(), _stream_handle(stream))
    _check(rc, "hg_probe_binned")


def probe(table: Table, queries, stream=None, binned: bool | None = None, ws=None):
    """uint32 count of build keys equal to each query (HashGraph-Probe-Standard
    semantics).  binned=None picks the binned probe for large batches."""
    torch = _torch()
    _require_cuda(queries, "queries")
    if _key_type_of(queries) != table.cfg.key_type:
        raise TypeError("query key type differs from the table's")
    counts = torch.empty(queries.numel(), dtype=torch.uint32, device=queries.device)
    if binned is None:
        binned = queries.numel() >= BINNED_PROBE_MIN_QUERIES
    if binned:
        need = probe_workspace_size(table, queries.numel())
        if need == 0:
            raise HGError(7, "hg_probe_workspace_size")
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=queries.device)
        probe_binned_into(table, queries, counts, ws, stream)
    else:
        probe_into(table, queries, counts, stream)
    return counts


def build_probe_host(cfg: hg_config, h_keys, h_queries, h_counts, d_keys, d_queries, d_counts, table: Table,
                     ws, probe_ws=None, stream=None):
    """hg_build_probe_host: host keys/queries in, host counts out (pinned CPU
    tensors), device staging and table buffers given; asynchronous."""
    for name, t in (("h_keys", h_keys), ("h_queries", h_queries), ("h_counts", h_counts)):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor")
    tv = table.view()
    _check(load().hg_build_probe_host(ctypes.byref(cfg), _ptr(h_keys), h_keys.numel(), _ptr(h_queries),
                                      h_queries.numel(), _ptr(h_counts), _ptr(d_keys), _ptr(d_queries),
                                      _ptr(d_counts), ctypes.byref(tv), _ptr(ws), ws.numel(), _ptr(probe_ws),
                                      0 if probe_ws is None else probe_ws.numel(), _stream_handle(stream)),
           "hg_build_probe_host")


def join_workspace_size(cfg: hg_config, nA: int, nB: int) -> int:
    return int(load().hg_join_workspace_size(ctypes.byref(cfg), nA, nB))


def _same_space(A: Table, B: Table):
    if A.cfg.num_buckets != B.cfg.num_buckets or A.cfg.key_type != B.cfg.key_type or A.cfg.map != B.cfg.map \
            or A.cfg.seed != B.cfg.seed or A.model is not B.model:
        raise ValueError("Alg. 3 needs both tables built with the same V and bucket map")


def join_count(A: Table, B: Table, per_bucket: bool = True, stream=None, ws=None):
    """Alg. 3 (HashGraph-Probe-New): inner-join size; optional int64 pairs per bucket."""
    torch = _torch()
    _same_space(A, B)
    dev = A.keys.device
    need = join_workspace_size(A.cfg, A.keys.numel(), B.keys.numel())
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    total = torch.empty(1, dtype=torch.int64, device=dev)
    bc = torch.empty(A.num_buckets, dtype=torch.int64, device=dev) if per_bucket else None
    ta, tb = A.view(), B.view()
    rc = load().hg_join_count(ctypes.byref(A.cfg), ctypes.byref(ta), ctypes.byref(tb), _ptr(total), _ptr(bc),
                              _ptr(ws), ws.numel(), _stream_handle(stream))
    _check(rc, "hg_join_count")
    return total, bc


def join_materialize(A: Table, B: Table, capacity: int | None = None, stream=None, ws=None,
                     after_count: bool = False):
    """Alg. 3 with the pairs written out: (A ids, B ids) int64 in canonical order.
    Without a capacity the join is counted first (hg_join_count) in the same
    workspace and the pairs are written from that count's per-edge match counts
    (hg_join_materialize_after_count), so the buckets are intersected once.
    after_count=True says that ws already holds hg_join_count's result for A and B."""
    torch = _torch()
    _same_space(A, B)
    dev = A.keys.device
    need = join_workspace_size(A.cfg, A.keys.numel(), B.keys.numel())
    if ws is None or ws.numel() < need:
        if after_count:
            raise ValueError("after_count needs the workspace of the preceding join_count")
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    if capacity is None:
        capacity = int(join_count(A, B, per_bucket=False, stream=stream, ws=ws)[0].item())
        after_count = True
    oa = torch.empty(max(capacity, 1), dtype=torch.int64, device=dev)
    ob = torch.empty(max(capacity, 1), dtype=torch.int64, device=dev)
    total = torch.empty(1, dtype=torch.int64, device=dev)
    join_materialize_into(A, B, oa, ob, total, ws, stream, after_count=after_count, capacity=capacity)
    m = min(int(total.item()), capacity)
    return oa[:m], ob[:m]


def join_count_into(A: Table, B: Table, total, bucket_counts, ws, stream=None):
    """hg_join_count on caller-provided tensors (bucket_counts may be None)."""
    _same_space(A, B)
    ta, tb = A.view(), B.view()
    _check(load().hg_join_count(ctypes.byref(A.cfg), ctypes.byref(ta), ctypes.byref(tb), _ptr(total),
                                _ptr(bucket_counts), _ptr(ws), ws.numel(), _stream_handle(stream)), "hg_join_count")


def join_materialize_into(A: Table, B: Table, out_a, out_b, total, ws, stream=None, after_count: bool = False,
                          capacity: int | None = None):
    """hg_join_materialize (or, after_count=True, hg_join_materialize_after_count,
    which reuses the per-edge counts hg_join_count left in ws) on caller-provided
    tensors; capacity defaults to out_a.numel()."""
    _same_space(A, B)
    ta, tb = A.view(), B.view()
    lib = load()
    fn, name = ((lib.hg_join_materialize_after_count, "hg_join_materialize_after_count") if after_count
                else (lib.hg_join_materialize, "hg_join_materialize"))
    cap = out_a.numel() if capacity is None else capacity
    _check(fn(ctypes.byref(A.cfg), ctypes.byref(ta), ctypes.byref(tb), _ptr(out_a), _ptr(out_b), cap, _ptr(total),
              _ptr(ws), ws.numel(), _stream_handle(stream)), name)


def selftest_wait_timeout(ws, limit_ms: int = 50, stream=None):
    """Run the bounded-wait self-test (hg_selftest_wait_timeout) on ws."""
    _check(load().hg_selftest_wait_timeout(_ptr(ws), limit_ms, _stream_handle(stream)), "hg_selftest_wait_timeout")


def workspace_status(ws, stream=None) -> int:
    return int(load().hg_workspace_status(_ptr(ws), _stream_handle(stream)))


# --------------------------------------------------------------------------
# learned bucket map
# --------------------------------------------------------------------------
def learned_train(keys, num_buckets: int, num_leaves: int = 1024, sample_size: int | None = None,
                  seed: int = 0x4C524E, iters: int = 40, stream=None):
    """Train the learned bucket map on the GPU (hg_learned_train).  Returns
    (model uint8 tensor, diag dict with the loss before/after, the root loss
    and the knot values)."""
    torch = _torch()
    _require_cuda(keys, "keys")
    kt = _key_type_of(keys)
    n = keys.numel()
    S = sample_size or max(1, n // 100)
    lib = load()
    model = torch.empty(int(lib.hg_learned_model_bytes(num_leaves)), dtype=torch.uint8, device=keys.device)
    wsz = int(lib.hg_learned_workspace_size(kt, n, S, num_leaves))
    ws = torch.empty(wsz, dtype=torch.uint8, device=keys.device)
    diag = torch.zeros(num_leaves + 5, dtype=torch.float64, device=keys.device)
    rc = lib.hg_learned_train(kt, _ptr(keys), n, num_buckets, num_leaves, S, seed, iters, _ptr(model), _ptr(diag),
                              _ptr(ws), ws.numel(), _stream_handle(stream))
    _check(rc, "hg_learned_train")
    d = diag.cpu().numpy()
    return model, {"loss_before": float(d[0]), "loss_after": float(d[1]), "root_loss": float(d[2]),
                   "Y": d[4:4 + num_leaves + 1].copy(), "sample_size": S}


def learned_sorted_sample(keys, sample_size: int, seed: int, stream=None):
    torch = _torch()
    kt = _key_type_of(keys)
    lib = load()
    out = torch.empty(sample_size + 2, dtype=torch.uint64, device=keys.device)[:sample_size]
    ws = torch.empty(int(lib.hg_learned_workspace_size(kt, keys.numel(), sample_size, 1)), dtype=torch.uint8,
                     device=keys.device)
    rc = lib.hg_learned_sorted_sample(kt, _ptr(keys), keys.numel(), sample_size, seed, _ptr(out), _ptr(ws),
                                      ws.numel(), _stream_handle(stream))
    _check(rc, "hg_learned_sorted_sample")
    return out


def learned_root_grad(key_type: int, sorted_sample, num_leaves: int, a: float, b: float, stream=None):
    torch = _torch()
    out = torch.empty(4, dtype=torch.float64, device=sorted_sample.device)
    ws = torch.empty(1 << 16, dtype=torch.uint8, device=sorted_sample.device)
    rc = load().hg_learned_root_grad(key_type, _ptr(sorted_sample), sorted_sample.numel(), num_leaves, a, b,
                                     _ptr(out), _ptr(ws), ws.numel(), _stream_handle(stream))
    _check(rc, "hg_learned_root_grad")
    o = out.cpu().numpy()
    return float(o[0]), float(o[1]), float(o[2])


def learned_leaf_grad(key_type: int, sorted_sample, num_buckets: int, a: float, b: float, num_leaves: int, Y,
                      stream=None):
    """(loss, dL/dY float32[L+1], Hessian diagonal float32[L+1]) at knot values Y (float64[L+1])."""
    torch = _torch()
    dev = sorted_sample.device
    lib = load()
    S = sorted_sample.numel()
    Yd = torch.as_tensor(Y, dtype=torch.float64).to(dev)
    g = torch.empty(num_leaves + 1, dtype=torch.float32, device=dev)
    h = torch.empty(num_leaves + 1, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    ws = torch.empty(int(lib.hg_learned_workspace_size(key_type, S, S, num_leaves)), dtype=torch.uint8, device=dev)
    rc = lib.hg_learned_leaf_grad(key_type, _ptr(sorted_sample), S, num_buckets, a, b, num_leaves, _ptr(Yd), _ptr(g),
                                  _ptr(h), _ptr(loss), _ptr(ws), ws.numel(), _stream_handle(stream))
    _check(rc, "hg_learned_leaf_grad")
    return float(loss.item()), g.cpu().numpy(), h.cpu().numpy()


def bucket_stats(keys, num_buckets: int, model=None, seed: int = 0, stream=None) -> dict:
    """Bucket-length max / mean / variance / non-empty count of a map over keys."""
    torch = _torch()
    kt = _key_type_of(keys)
    cfg = make_config(kt, num_buckets, seed, "auto", model)
    counts = torch.empty(num_buckets, dtype=torch.uint32, device=keys.device)
    out = torch.empty(4, dtype=torch.float64, device=keys.device)
    ws = torch.empty(1 << 16, dtype=torch.uint8, device=keys.device)
    rc = load().hg_bucket_stats(ctypes.byref(cfg), _ptr(keys), keys.numel(), _ptr(counts), _ptr(out), _ptr(ws),
                                ws.numel(), _stream_handle(stream))
    _check(rc, "hg_bucket_stats")
    o = out.cpu().numpy()
    return {"max": float(o[0]), "mean": float(o[1]), "var": float(o[2]), "nonempty": float(o[3])}


def choose_map(keys, num_buckets: int, model, seed: int = 0, var_tolerance: float = 0.0,
               max_factor: float = 0.0, stream=None):
    """(model or None, report): Murmur judges the learned map on `keys`
    (hg_learned_judge): the model is returned while the library keeps it,
    else None (build with Murmur).  Tolerances <= 0 take the library's
    defaults.  report: both maps' bucket-length statistics and the verdict."""
    torch = _torch()
    _require_cuda(keys, "keys")
    lib = load()
    cfg = make_config(_key_type_of(keys), num_buckets, seed, "auto", model)
    counts = torch.empty(num_buckets, dtype=torch.uint32, device=keys.device)
    ws = torch.empty(int(lib.hg_learned_judge_workspace_size()), dtype=torch.uint8, device=keys.device)
    st = (ctypes.c_double * 8)()
    keep = ctypes.c_int32(0)
    _check(lib.hg_learned_judge(ctypes.byref(cfg), _ptr(keys), keys.numel(), var_tolerance, max_factor, _ptr(counts),
                                _ptr(ws), ws.numel(), st, ctypes.byref(keep), _stream_handle(stream)),
           "hg_learned_judge")
    names = ("max", "mean", "var", "nonempty")
    rep = {"learned": {k: float(st[i]) for i, k in enumerate(names)},
           "murmur": {k: float(st[4 + i]) for i, k in enumerate(names)}, "kept": bool(keep.value)}
    return (model if keep.value else None), rep


class BatchPlan:
    """Many independent uint32 tables built and probed together
    (hg_batch_*).  Table t has sizes[t] keys, qsizes[t] queries and
    num_buckets[t] buckets (default max(1, sizes[t])).  Buffers live in one
    padded concatenated layout (see ``alloc``); ``run`` replays one CUDA
    graph for the whole batch."""

    def __init__(self, sizes, qsizes, num_buckets=None, seed: int = 0):
        import numpy as np
        lib = load()
        self._lib = lib
        self.T = len(sizes)
        self.seed = seed & 0xFFFFFFFF
        self.sizes = np.ascontiguousarray(sizes, dtype=np.uint64)
        self.qsizes = np.ascontiguousarray(qsizes, dtype=np.uint64)
        self.V = None if num_buckets is None else np.ascontiguousarray(num_buckets, dtype=np.uint64)
        h = _VP()
        rc = lib.hg_batch_plan_create(KEY_U32, seed & 0xFFFFFFFF, self.T, self.sizes.ctypes.data,
                                      self.qsizes.ctypes.data, None if self.V is None else self.V.ctypes.data,
                                      ctypes.byref(h))
        _check(rc, "hg_batch_plan_create")
        self._h = h
        tot = np.zeros(4, dtype=np.uint64)
        self.key_begin = np.zeros(self.T + 1, dtype=np.uint64)
        self.query_begin = np.zeros(self.T + 1, dtype=np.uint64)
        self.offset_begin = np.zeros(self.T + 1, dtype=np.uint64)
        _check(lib.hg_batch_layout(h, tot.ctypes.data, self.key_begin.ctypes.data, self.query_begin.ctypes.data,
                                   self.offset_begin.ctypes.data), "hg_batch_layout")
        self.total_keys, self.total_queries, self.total_offsets = int(tot[0]), int(tot[1]), int(tot[2])
        self.ws_bytes = int(lib.hg_batch_workspace_size(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.hg_batch_plan_destroy(h)
            self._h = None

    def num_buckets(self, t: int) -> int:
        return int(self.offset_begin[t + 1] - self.offset_begin[t]) - 1

    def alloc(self, device="cuda") -> dict:
        """Device buffers of the batch: keys, queries, offsets, csr_keys, csr_ids, counts, ws."""
        torch = _torch()
        u32 = torch.uint32
        return {"keys": torch.zeros(self.total_keys + 4, dtype=u32, device=device)[:self.total_keys],
                "queries": torch.zeros(self.total_queries + 4, dtype=u32, device=device)[:self.total_queries],
                "offsets": torch.empty(self.total_offsets, dtype=u32, device=device),
                "csr_keys": torch.empty(self.total_keys + 4, dtype=u32, device=device)[:self.total_keys],
                "csr_ids": torch.empty(self.total_keys + 4, dtype=u32, device=device)[:self.total_keys],
                "counts": torch.empty(self.total_queries + 4, dtype=u32, device=device)[:self.total_queries],
                "ws": torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)}

    def pad_keys(self, flat):
        """Host array of all tables' keys back to back (unpadded) -> padded layout."""
        import numpy as np
        out = np.zeros(self.total_keys, dtype=np.uint32)
        ub = np.concatenate([[0], np.cumsum(self.sizes.astype(np.int64))])
        out[np.repeat(self.key_begin[:-1].astype(np.int64) - ub[:-1], self.sizes.astype(np.int64))
            + np.arange(int(ub[-1]))] = flat
        return out

    def pad_queries(self, flat):
        import numpy as np
        out = np.zeros(self.total_queries, dtype=np.uint32)
        ub = np.concatenate([[0], np.cumsum(self.qsizes.astype(np.int64))])
        out[np.repeat(self.query_begin[:-1].astype(np.int64) - ub[:-1], self.qsizes.astype(np.int64))
            + np.arange(int(ub[-1]))] = flat
        return out

    def _args(self, b):
        for k in ("keys", "queries", "offsets", "csr_keys", "csr_ids", "counts", "ws"):
            _require_cuda(b[k], k)
        return (_ptr(b["keys"]), _ptr(b["queries"]), _ptr(b["offsets"]), _ptr(b["csr_keys"]), _ptr(b["csr_ids"]),
                _ptr(b["counts"]), _ptr(b["ws"]), b["ws"].numel())

    def run(self, b: dict, stream=None):
        _check(self._lib.hg_batch_run(self._h, *self._args(b), _stream_handle(stream)), "hg_batch_run")

    def run_eager(self, b: dict, stream=None):
        _check(self._lib.hg_batch_run_eager(self._h, *self._args(b), _stream_handle(stream)), "hg_batch_run_eager")

    def run_plain(self, b: dict, stream=None):
        _check(self._lib.hg_batch_run_plain(self._h, *self._args(b), _stream_handle(stream)), "hg_batch_run_plain")

    def autotune(self, b: dict, reps: int = 2, stream=None) -> dict:
        ms = ctypes.c_float(0.0)
        _check(self._lib.hg_batch_autotune(self._h, *self._args(b), _stream_handle(stream), reps, ctypes.byref(ms)),
               "hg_batch_autotune")
        return dict(self.config(), ms=ms.value)

    def set_config(self, bin_shift: int = 0, threads_per_bin: int = 0):
        _check(self._lib.hg_batch_set_config(self._h, bin_shift, threads_per_bin), "hg_batch_set_config")

    def config(self) -> dict:
        s, t, w = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(self._lib.hg_batch_get_config(self._h, ctypes.byref(s), ctypes.byref(t), ctypes.byref(w)),
               "hg_batch_get_config")
        return {"bin_shift": s.value, "threads_per_bin": t.value, "waves": w.value}

    def table(self, b: dict, t: int):
        """Views of table t: (offsets[V_t+1] as positions in the batch, csr keys, csr ids, counts)."""
        k0, k1 = int(self.key_begin[t]), int(self.key_begin[t]) + int(self.sizes[t])
        q0, q1 = int(self.query_begin[t]), int(self.query_begin[t]) + int(self.qsizes[t])
        o0, o1 = int(self.offset_begin[t]), int(self.offset_begin[t + 1])
        return b["offsets"][o0:o1], b["csr_keys"][k0:k1], b["csr_ids"][k0:k1], b["counts"][q0:q1]
