"""hg_build_static_scratch: the build for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Called through the
C ABI, twice in a row, its table must equal hg_build's byte for byte; the
second call also shows that leftovers of the first call in the shared array
do not leak into the result.  Runs alone or after the other tests."""
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
    return f


def _static_build(hg, f, cfg, keys_d, n, V):
    import torch
    off = torch.full((V + 1,), 0xFFFFFFFF, dtype=torch.uint32, device="cuda")
    ck = torch.empty(n, dtype=keys_d.dtype, device="cuda")
    ci = torch.empty(n, dtype=torch.uint32, device="cuda")
    rc = f(ctypes.byref(cfg), keys_d.data_ptr(), None, n, off.data_ptr(), ck.data_ptr(), ci.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert rc == 0, hg.STATUS_NAMES.get(rc, rc)
    torch.cuda.synchronize()
    return to_np(off), to_np(ck), to_np(ci)


@pytest.mark.parametrize("kt,n,V", [("u32", 200_003, 1 << 18), ("u64", 150_001, 1 << 16)])
def test_static_scratch_build_matches_hg_build_twice(hg, kt, n, V):
    lib = hg.load()
    f = _static_entry(lib)
    assert lib.hg_static_scratch_bytes() == 8 << 20
    keys = dg.uniform_keys_u32(n, 21) if kt == "u32" else dg.uniform_keys_u64(n, 21)
    keys_d = to_dev(keys)
    ref = hg.build(keys_d, V)
    want = (to_np(ref.offsets), to_np(ref.keys), to_np(ref.ids))
    cfg = hg.make_config(ref.cfg.key_type, V)
    for _ in range(2):
        got = _static_build(hg, f, cfg, keys_d, n, V)
        for g, w in zip(got, want):
            assert np.array_equal(g, w)
    # a different input on the same array right after: still exact
    keys2 = dg.dup_keys_u32(n, 7, 22) if kt == "u32" else dg.zipf_keys_u64(n, 5000, 22)
    k2 = to_dev(keys2)
    ref2 = hg.build(k2, V)
    got2 = _static_build(hg, f, cfg, k2, n, V)
    for g, w in zip(got2, (to_np(ref2.offsets), to_np(ref2.keys), to_np(ref2.ids))):
        assert np.array_equal(g, w)


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
