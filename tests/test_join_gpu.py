"""Parity of Alg. 3 (bucket-wise intersection) with the CPU oracle."""
import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def _tables(hg, orc, a, b, V, seed=0):
    tA = hg.build(to_dev(a), V, seed=seed)
    tB = hg.build(to_dev(b), V, seed=seed)
    rA = orc.build(a, V, seed)
    rB = orc.build(b, V, seed)
    return tA, tB, rA, rB


@pytest.mark.parametrize("V", [1, 64, 4096, 1 << 17, 1 << 22])
def test_join_count_u32(hg, orc, V):
    a = dg.dup_keys_u32(120_000, 3, 1)
    b = dg.dup_keys_u32(90_000, 2, 2)
    tA, tB, rA, rB = _tables(hg, orc, a, b, V, seed=4)
    total, per = hg.join_count(tA, tB)
    rt, rper = orc.join_count(rA[0], rA[1], rB[0], rB[1], V)
    assert int(total.item()) == rt == orc.join_size_by_keys(a, b)
    assert np.array_equal(to_np(per), rper)


@pytest.mark.parametrize("kt", ["u32", "u64"])
@pytest.mark.parametrize("V", [1, 7, 4096])
def test_join_with_zero_and_largest_keys(hg, orc, kt, V):
    """Key 0 and the largest key of the width join like any other key: both
    sides hold several copies of each, next to random keys of a small domain."""
    rng = np.random.default_rng(101)
    dt = np.uint32 if kt == "u32" else np.uint64
    top = np.iinfo(dt).max
    dom = rng.integers(1, 1 << 30, 300).astype(dt)
    a = dom[rng.integers(0, 300, 4000)]
    b = dom[rng.integers(0, 300, 3000)]
    a[rng.integers(0, 4000, 30)] = 0
    a[rng.integers(0, 4000, 20)] = top
    b[rng.integers(0, 3000, 10)] = 0
    b[rng.integers(0, 3000, 15)] = top
    tA, tB, rA, rB = _tables(hg, orc, a, b, V, seed=6)
    total, per = hg.join_count(tA, tB)
    rt, rper = orc.join_count(rA[0], rA[1], rB[0], rB[1], V)
    assert int(total.item()) == rt == orc.join_size_by_keys(a, b)
    assert np.array_equal(to_np(per), rper)
    pa, pb = hg.join_materialize(tA, tB)
    ra, rb = orc.join_materialize(rA[0], rA[1], rA[2], rB[0], rB[1], rB[2], V)
    assert np.array_equal(to_np(pa), ra) and np.array_equal(to_np(pb), rb)


def test_join_count_zipf_u64(hg, orc):
    # Section 5 join workload shape: Zipf(1) build side vs uniform probe side.
    a = dg.zipf_keys_u64(1 << 20, 1 << 17, 3)
    b = dg.uniform_domain_keys_u64(1 << 20, 1 << 17, 4)
    V = 1 << 20
    tA, tB, rA, rB = _tables(hg, orc, a, b, V)
    total, per = hg.join_count(tA, tB)
    rt, rper = orc.join_count(rA[0], rA[1], rB[0], rB[1], V)
    assert int(total.item()) == rt
    assert np.array_equal(to_np(per), rper)


@pytest.mark.parametrize("V", [1, 512, 1 << 16])
def test_join_materialize_canonical_order(hg, orc, V):
    a = dg.zipf_keys_u64(60_000, 4000, 5)
    b = dg.uniform_domain_keys_u64(50_000, 4000, 6)
    tA, tB, rA, rB = _tables(hg, orc, a, b, V, seed=2)
    pa, pb = hg.join_materialize(tA, tB)
    ra, rb = orc.join_materialize(rA[0], rA[1], rA[2], rB[0], rB[1], rB[2], V)
    assert np.array_equal(to_np(pa), ra) and np.array_equal(to_np(pb), rb)


def test_join_materialize_capacity_overflow(hg, orc):
    a = dg.dup_keys_u32(20_000, 10, 7)
    b = dg.dup_keys_u32(20_000, 10, 8)
    V = 1 << 12
    tA, tB, rA, rB = _tables(hg, orc, a, b, V)
    total = int(hg.join_count(tA, tB)[0].item())
    cap = total // 3
    pa, pb = hg.join_materialize(tA, tB, capacity=cap)
    ra, rb = orc.join_materialize(rA[0], rA[1], rA[2], rB[0], rB[1], rB[2], V, cap=cap)
    assert len(pa) == cap
    assert np.array_equal(to_np(pa), ra) and np.array_equal(to_np(pb), rb)


def test_join_empty_sides(hg):
    import torch
    e = torch.empty(0, dtype=torch.uint32, device="cuda")
    tA = hg.build(e, 32)
    tB = hg.build(to_dev(dg.uniform_keys_u32(1000, 1)), 32)
    assert int(hg.join_count(tA, tB)[0].item()) == 0
    assert int(hg.join_count(tB, tA)[0].item()) == 0
    pa, pb = hg.join_materialize(tB, tA)
    assert pa.numel() == 0


@pytest.mark.parametrize("V", [1, 1 << 10])
def test_join_materialize_long_pair_lists(hg, orc, V):
    # 3000 copies of one key against 1500 copies of it: every such A edge
    # writes 1500 pairs, spanning many output windows; the other keys share
    # the bucket with it when V = 1; a capacity cut inside a window
    u = dg.uniform_keys_u32(8000, 41)
    a = np.concatenate([np.full(3000, u[0], dtype=np.uint32), u[1:5001]])
    b = np.concatenate([np.full(1500, u[0], dtype=np.uint32), u[2000:5000]])
    pa_ = dg.splitmix64(3, 7, np.arange(len(a), dtype=np.uint64)).argsort(kind="stable")
    pb_ = dg.splitmix64(3, 8, np.arange(len(b), dtype=np.uint64)).argsort(kind="stable")
    a, b = a[pa_], b[pb_]
    tA, tB, rA, rB = _tables(hg, orc, a, b, V, seed=6)
    pa, pb = hg.join_materialize(tA, tB)
    ra, rb = orc.join_materialize(rA[0], rA[1], rA[2], rB[0], rB[1], rB[2], V)
    assert len(ra) == 3000 * 1500 + 3000
    assert np.array_equal(to_np(pa), ra) and np.array_equal(to_np(pb), rb)
    cap = 1_234_567
    pa, pb = hg.join_materialize(tA, tB, capacity=cap)
    ra, rb = orc.join_materialize(rA[0], rA[1], rA[2], rB[0], rB[1], rB[2], V, cap=cap)
    assert np.array_equal(to_np(pa), ra) and np.array_equal(to_np(pb), rb)


def test_join_materialize_after_count_reuses_the_count(hg, orc):
    """hg_join_materialize_after_count writes the same pairs as the
    self-contained call from the per-edge counts hg_join_count left in the
    workspace; the device refuses a workspace counted for other tables, and
    a second call without a new count (the counts are consumed)."""
    import torch
    a = dg.zipf_keys_u64(80_000, 3000, 31)
    b = dg.uniform_domain_keys_u64(70_000, 3000, 32)
    V = 1 << 15
    tA, tB, rA, rB = _tables(hg, orc, a, b, V, seed=1)
    ra, rb = orc.join_materialize(rA[0], rA[1], rA[2], rB[0], rB[1], rB[2], V)
    M = len(ra)
    ws = torch.empty(hg.join_workspace_size(tA.cfg, len(a), len(b)), dtype=torch.uint8, device="cuda")
    out_a = torch.full((M,), -7, dtype=torch.int64, device="cuda")
    out_b = torch.full((M,), -7, dtype=torch.int64, device="cuda")
    total = torch.empty(1, dtype=torch.int64, device="cuda")
    hg.join_count_into(tA, tB, total, None, ws)
    assert int(total.item()) == M
    hg.join_materialize_into(tA, tB, out_a, out_b, total, ws, after_count=True)
    assert hg.workspace_status(ws) == 0 and int(total.item()) == M
    assert np.array_equal(to_np(out_a), ra) and np.array_equal(to_np(out_b), rb)
    # consumed: a second call without a count is refused on the device
    out_a.fill_(-7)
    hg.join_materialize_into(tA, tB, out_a, out_b, total, ws, after_count=True)
    assert hg.workspace_status(ws) == 1 and int(total.item()) == 0   # HG_ERR_INVALID_ARG
    assert bool((out_a == -7).all())
    # counted for (A, B), materialised for (B, A): refused
    hg.join_count_into(tA, tB, total, None, ws)
    hg.join_materialize_into(tB, tA, out_a, out_b, total, ws, after_count=True)
    assert hg.workspace_status(ws) == 1
    # the convenience call counts and then materialises from that count
    pa, pb = hg.join_materialize(tA, tB)
    assert np.array_equal(to_np(pa), ra) and np.array_equal(to_np(pb), rb)
