"""The bounded waits: a wait that nobody completes gives up after its limit,
the workspace status reads HG_ERR_TIMEOUT, and the CUDA context stays usable
(a build right after is still exact)."""
import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg
from gpu_util import table_np, to_dev

pytestmark = pytest.mark.gpu


def test_wait_gives_up_and_context_survives(hg, orc):
    import time
    import torch
    ws = torch.empty(1 << 12, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    hg.selftest_wait_timeout(ws, limit_ms=50)
    st = hg.workspace_status(ws)
    dt = time.perf_counter() - t0
    assert st == 5, hg.STATUS_NAMES.get(st, st)          # HG_ERR_TIMEOUT
    assert 0.05 <= dt < 5.0
    hg.load().hg_workspace_clear(hg._ptr(ws), None)
    assert hg.workspace_status(ws) == 0
    keys = dg.uniform_keys_u32(100_000, 3)
    t = hg.build(to_dev(keys), 1 << 17)
    off, ck, ci = table_np(t)
    roff, rk, ri = orc.build(keys, 1 << 17)
    assert np.array_equal(off, roff) and np.array_equal(ck, rk) and np.array_equal(ci, ri)


def test_selftest_argument_checks(hg):
    assert hg.load().hg_selftest_wait_timeout(None, 50, None) == 1
