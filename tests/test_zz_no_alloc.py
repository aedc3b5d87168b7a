"""hg_build_static_scratch: the build for callers that cannot allocate device
memory -- a plug-in running inside a runtime that owns all device memory
and offers it no allocator, or a serving loop that may not call cudaMalloc
or cudaFree because they can synchronise the device.  Its scratch is a
fixed array inside the library.

Called through the C ABI, twice in a row, its table must equal the
oracle's and hg_build's byte for byte, and the array's status word (read by
hg_static_scratch_status, which needs no workspace pointer) must be HG_OK
after every build; the second call also shows that leftovers of the first
call in the shared array do not leak into the result.  The documented size
bound is exercised at its edge: 2^18 keys into 2^29 buckets (uint32 keys)
and 2^28 buckets (uint64 keys).  Runs alone or after the other tests."""
import ctypes

import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def _static_entry(lib):
    f = lib.hg_build_static_scratch
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_uint64] + [ctypes.c_void_p] * 4
    lib.hg_static_scratch_bytes.restype = ctypes.c_size_t
    lib.hg_static_scratch_status.restype = ctypes.c_int32
    lib.hg_static_scratch_status.argtypes = [ctypes.c_void_p]
    return f


def _static_build(hg, lib, f, cfg, keys_d, n, V):
    import torch
    off = torch.full((V + 1,), 0xFFFFFFFF, dtype=torch.uint32, device="cuda")
    ck = torch.empty(n, dtype=keys_d.dtype, device="cuda")
    ci = torch.empty(n, dtype=torch.uint32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = f(ctypes.byref(cfg), keys_d.data_ptr(), None, n, off.data_ptr(), ck.data_ptr(), ci.data_ptr(), stream)
    assert rc == 0, hg.STATUS_NAMES.get(rc, rc)
    st = lib.hg_static_scratch_status(stream)
    assert st == 0, hg.STATUS_NAMES.get(st, st)
    return to_np(off), to_np(ck), to_np(ci)


def _same(got, want):
    for g, w, name in zip(got, want, ("offsets", "csr keys", "csr ids")):
        assert np.array_equal(g, w), name


@pytest.mark.parametrize("kt,n,V", [("u32", 200_003, 1 << 18), ("u64", 150_001, 1 << 16)])
def test_static_scratch_build_matches_oracle_and_hg_build_twice(hg, orc, kt, n, V):
    lib = hg.load()
    f = _static_entry(lib)
    assert lib.hg_static_scratch_bytes() == 8 << 20
    keys = dg.uniform_keys_u32(n, 21) if kt == "u32" else dg.uniform_keys_u64(n, 21)
    keys_d = to_dev(keys)
    want = orc.build(keys, V)
    ref = hg.build(keys_d, V)
    _same((to_np(ref.offsets), to_np(ref.keys), to_np(ref.ids)), want)
    cfg = hg.make_config(ref.cfg.key_type, V)
    for _ in range(2):
        _same(_static_build(hg, lib, f, cfg, keys_d, n, V), want)
    # a different input on the same array right after: still exact
    keys2 = dg.dup_keys_u32(n, 7, 22) if kt == "u32" else dg.zipf_keys_u64(n, 5000, 22)
    _same(_static_build(hg, lib, f, cfg, to_dev(keys2), n, V), orc.build(keys2, V))


@pytest.mark.parametrize("kt,log2v", [("u32", 29), ("u64", 28)])
def test_static_scratch_documented_bound(hg, orc, kt, log2v):
    """2^18 keys with the automatic bin size into the most buckets the header
    promises to fit: 2^29 for uint32 keys, 2^28 for uint64 keys; one more
    doubling of V for uint64 keys is refused before anything is launched."""
    import torch
    lib = hg.load()
    f = _static_entry(lib)
    n, V = 1 << 18, 1 << log2v
    keys = dg.uniform_keys_u32(n, 23) if kt == "u32" else dg.uniform_keys_u64(n, 23)
    kt_id = hg.KEY_U32 if kt == "u32" else hg.KEY_U64
    cfg = hg.make_config(kt_id, V)
    assert hg.build_workspace_size(cfg, n) <= lib.hg_static_scratch_bytes()
    keys_d = to_dev(keys)
    want = orc.build(keys, V)
    for _ in range(2):
        _same(_static_build(hg, lib, f, cfg, keys_d, n, V), want)
    if kt == "u64":
        V2 = 2 * V
        cfg2 = hg.make_config(kt_id, V2)
        assert hg.build_workspace_size(cfg2, n) > lib.hg_static_scratch_bytes()
        off = torch.empty(V2 + 1, dtype=torch.uint32, device="cuda")
        ck = torch.empty(n, dtype=keys_d.dtype, device="cuda")
        ci = torch.empty(n, dtype=torch.uint32, device="cuda")
        rc = f(ctypes.byref(cfg2), keys_d.data_ptr(), None, n, off.data_ptr(), ck.data_ptr(), ci.data_ptr(),
               torch.cuda.current_stream().cuda_stream)
        assert rc == 2                            # HG_ERR_WORKSPACE_TOO_SMALL
    torch.cuda.empty_cache()


def test_static_scratch_refuses_oversized_plans(hg):
    import torch
    lib = hg.load()
    f = _static_entry(lib)
    n = 1 << 22                                  # plan needs far more than 8 MiB
    cfg = hg.make_config(hg.KEY_U32, 1 << 22)
    assert hg.build_workspace_size(cfg, n) > lib.hg_static_scratch_bytes()
    k = torch.zeros(n, dtype=torch.uint32, device="cuda")
    off = torch.empty((1 << 22) + 1, dtype=torch.uint32, device="cuda")
    ck = torch.empty(n, dtype=torch.uint32, device="cuda")
    ci = torch.empty(n, dtype=torch.uint32, device="cuda")
    rc = f(ctypes.byref(cfg), k.data_ptr(), None, n, off.data_ptr(), ck.data_ptr(), ci.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert rc == 2                                # HG_ERR_WORKSPACE_TOO_SMALL, nothing launched
