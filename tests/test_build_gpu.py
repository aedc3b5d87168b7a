"""Parity of the CUDA build and probe with the CPU oracle, bit for bit."""
import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg
from gpu_util import sampled_reference, table_np, to_dev, to_np

pytestmark = pytest.mark.gpu


def _check_build(hg, orc, keys, V, seed=0, algo="auto", bin_shift=0, ids=None):
    t = hg.build(to_dev(keys), V, ids=None if ids is None else to_dev(ids), seed=seed, algo=algo,
                 bin_shift=bin_shift)
    off, ck, ci = table_np(t)
    roff, rk, ri = orc.build(keys, V, seed, ids=ids)
    assert np.array_equal(off, roff), "offsets differ"
    assert np.array_equal(ck, rk), "csr keys differ"
    assert np.array_equal(ci, ri), "csr ids differ"
    return t


@pytest.mark.parametrize("algo", ["v2", "v1"])
@pytest.mark.parametrize("n,V", [(1, 1), (33, 7), (1000, 1), (4096, 4096), (100_000, 100_003),
                                 ((1 << 20) + 37, 1 << 20), ((1 << 20) + 5, 1 << 16), (300_000, 1 << 22)])
def test_build_u32_uniform(hg, orc, algo, n, V):
    _check_build(hg, orc, dg.uniform_keys_u32(n, 1), V, seed=3, algo=algo)


@pytest.mark.parametrize("bin_shift", [1, 4, 8, 12, 15])
def test_build_v2_any_bin_size_same_table(hg, orc, bin_shift):
    # Section 5.1: V1 and V2 produce the same table; with the canonical order
    # the bytes are identical for every bin size.
    _check_build(hg, orc, dg.uniform_keys_u32(200_000, 2), 1 << 18, algo="v2", bin_shift=bin_shift)


def test_build_explicit_ids(hg, orc):
    keys = dg.uniform_keys_u32(50_000, 4)
    ids = (np.arange(50_000, dtype=np.uint64) * np.uint64(2654435761) % np.uint64(1 << 32)).astype(np.uint32)
    for algo in ("v1", "v2"):
        _check_build(hg, orc, keys, 1 << 15, algo=algo, ids=ids)


@pytest.mark.parametrize("algo", ["v2", "v1"])
def test_build_u64(hg, orc, algo):
    _check_build(hg, orc, dg.uniform_keys_u64(300_001, 5), 1 << 18, seed=11, algo=algo)


@pytest.mark.parametrize("algo", ["v2", "v1"])
@pytest.mark.parametrize("mult", [4, 32, 1000, 100_000])
def test_build_duplicates(hg, orc, algo, mult):
    # Fig. "dup-keys": keys drawn from [1 .. N/d]; heavy buckets and bins
    # larger than shared memory.
    _check_build(hg, orc, dg.dup_keys_u32(400_000, mult, 6), 1 << 19, algo=algo)


@pytest.mark.parametrize("kt", ["u32", "u64"])
@pytest.mark.parametrize("explicit", [False, True])
def test_build_long_buckets_every_sort_tier(hg, orc, kt, explicit):
    """Buckets of 33 .. 300 edges in bins that fit shared memory: the bin
    build sorts them by position in registers (up to 64, 128 and 256 edges)
    or with bitmaps (longer).  Explicit ids keep the stable partitions; with
    implicit ids the partitions may rank in any order and every bucket is
    ranked by id."""
    lens = np.array([33, 47, 64, 65, 100, 128, 129, 200, 255, 256, 257, 300], dtype=np.int64)
    distinct = dg.uniform_keys_u32(6000, 12) if kt == "u32" else dg.uniform_keys_u64(6000, 12)
    counts = np.ones(len(distinct), dtype=np.int64)
    counts[:20 * len(lens)] = np.tile(lens, 20)
    keys = np.repeat(distinct, counts)
    keys = keys[np.random.default_rng(13).permutation(len(keys))]
    ids = np.arange(len(keys), dtype=np.uint32) if explicit else None
    _check_build(hg, orc, keys, 1 << 14, algo="v2", bin_shift=10, ids=ids)


def test_build_all_keys_equal_and_single_bucket(hg, orc):
    keys = np.full(70_000, 123456789, dtype=np.uint32)
    for algo in ("v1", "v2"):
        _check_build(hg, orc, keys, 1 << 16, algo=algo)
        _check_build(hg, orc, dg.uniform_keys_u32(70_000, 8), 1, algo=algo)


@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_build_huge_bins_split_across_ctas(hg, orc, kt):
    # Two keys hold 40% and 20% of 2^22 keys: their bins exceed 2^17 edges and
    # are built by several CTAs, one per 2^17-edge segment; the rest of the
    # table stays on the shared-memory path.
    n = 1 << 22
    base = dg.uniform_keys_u32(n, 21) if kt == "u32" else dg.uniform_keys_u64(n, 21)
    sel = dg.splitmix64(21, 99, np.arange(n, dtype=np.uint64)) >> np.uint64(11)
    u = sel.astype(np.float64) / float(1 << 53)
    keys = base.copy()
    keys[u < 0.4] = base[0]
    keys[(u >= 0.4) & (u < 0.6)] = base[1]
    for algo in ("v2", "v1"):
        _check_build(hg, orc, keys, 1 << 20, algo=algo)


@pytest.mark.parametrize("n", [1 << 22, (1 << 22) + 1, (1 << 22) + (5 << 17) - 3])
def test_build_single_bucket_segment_edges(hg, orc, n):
    # one bin, one bucket: exactly 32 segments, 32 segments plus one edge, a
    # ragged last segment; and the same number of equal keys
    keys = dg.uniform_keys_u32(n, 5)
    _check_build(hg, orc, keys, 1, algo="v2")
    _check_build(hg, orc, np.full(n, 77, dtype=np.uint32), 1 << 12, algo="v2")


def test_build_zipf_u64(hg, orc):
    keys = dg.zipf_keys_u64(1 << 20, 1 << 16, 7)
    for algo in ("v2", "v1"):
        _check_build(hg, orc, keys, 1 << 20, algo=algo)


@pytest.mark.parametrize("kt", ["u32", "u64"])
@pytest.mark.parametrize("algo", ["v2", "v1"])
@pytest.mark.parametrize("V", [1, 7, 4096])
def test_zero_and_largest_key_are_ordinary_keys(hg, orc, kt, algo, V):
    """No key value is reserved (the table is a CSR, not open addressing):
    key 0 and the largest key of the width are built, probed and counted like
    any other, next to random keys."""
    rng = np.random.default_rng(91)
    dt = np.uint32 if kt == "u32" else np.uint64
    top = np.iinfo(dt).max
    n = 5003
    keys = (dg.uniform_keys_u32(n, 92) if kt == "u32" else dg.uniform_keys_u64(n, 92)).copy()
    keys[rng.integers(0, n, 40)] = 0
    keys[rng.integers(0, n, 25)] = top
    keys[:3] = [0, top, 0]
    _check_build(hg, orc, keys, V, seed=4, algo=algo)
    q = np.concatenate([np.array([0, top, 1, top - 1], dtype=dt), keys[rng.integers(0, n, 3000)],
                        (dg.uniform_keys_u32(3000, 93) if kt == "u32" else dg.uniform_keys_u64(3000, 93))])
    t = hg.build(to_dev(keys), V, seed=4, algo=algo)
    want = orc.multiplicity(keys, q)
    assert want[0] == int((keys == 0).sum()) and want[1] == int((keys == top).sum())
    assert np.array_equal(to_np(hg.probe(t, to_dev(q), binned=False)), want)
    assert np.array_equal(to_np(hg.probe(t, to_dev(q), binned=True)), want)


def test_build_sequence_input(hg, orc):
    _check_build(hg, orc, dg.sequence_keys_u32(1 << 21), 1 << 20)


def test_build_empty(hg):
    import torch
    t = hg.build(torch.empty(0, dtype=torch.uint32, device="cuda"), 17)
    assert np.all(to_np(t.offsets) == 0)


@pytest.mark.parametrize("hit", [0.0, 0.5, 1.0])
def test_probe_u32(hg, orc, hit):
    keys = dg.dup_keys_u32(300_000, 2, 9)
    q = dg.queries_u32(200_000, keys, hit, 10)
    V = 1 << 18
    t = hg.build(to_dev(keys), V, seed=5)
    got = to_np(hg.probe(t, to_dev(q)))
    off, ck, _ = orc.build(keys, V, 5)
    assert np.array_equal(got, orc.probe(off, ck, q, V, 5))
    assert np.array_equal(got, orc.multiplicity(keys, q))


def test_probe_u64_long_buckets(hg, orc):
    keys = dg.zipf_keys_u64(200_000, 5000, 12)
    q = dg.queries_u64(100_000, keys, 0.5, 13)
    t = hg.build(to_dev(keys), 1 << 10)
    assert np.array_equal(to_np(hg.probe(t, to_dev(q))), orc.multiplicity(keys, q))


@pytest.mark.parametrize("kt,nq,V,hit", [("u32", 300_001, 1 << 18, 0.5), ("u32", 1 << 20, 1 << 20, 1.0),
                                          ("u32", 50_000, 1000, 0.3), ("u64", 400_000, 1 << 19, 0.5),
                                          ("u32", 2_000_000, 3_000_017, 0.5), ("u32", 7, 1, 1.0)])
def test_probe_binned_matches_oracle(hg, orc, kt, nq, V, hit):
    # The binned probe returns exactly HashGraph-Probe-Standard's counts.
    if kt == "u32":
        keys = dg.dup_keys_u32(max(nq // 2, 1), 2, 31)
        q = dg.queries_u32(nq, keys, hit, 32)
    else:
        keys = dg.zipf_keys_u64(nq // 2, 20_000, 31)
        q = dg.queries_u64(nq, keys, hit, 32)
    t = hg.build(to_dev(keys), V, seed=9)
    got = to_np(hg.probe(t, to_dev(q), binned=True))
    std = to_np(hg.probe(t, to_dev(q), binned=False))
    assert np.array_equal(got, std)
    assert np.array_equal(got, orc.multiplicity(keys, q))


def test_probe_binned_empty_table(hg):
    import torch
    e = hg.build(torch.empty(0, dtype=torch.uint32, device="cuda"), 1 << 12)
    q = to_dev(dg.uniform_keys_u32(100_000, 2))
    assert np.all(to_np(hg.probe(e, q, binned=True)) == 0)


def test_probe_empty_queries_and_table(hg):
    import torch
    t = hg.build(to_dev(dg.uniform_keys_u32(1000, 1)), 64)
    assert hg.probe(t, torch.empty(0, dtype=torch.uint32, device="cuda")).numel() == 0
    e = hg.build(torch.empty(0, dtype=torch.uint32, device="cuda"), 64)
    assert np.all(to_np(hg.probe(e, to_dev(dg.uniform_keys_u32(100, 2)))) == 0)


def test_full_size_build_and_probe_sampled(hg, orc):
    # 2^28 uint32 keys, V = 2^28 (load factor 1), the benchmark's launch
    # configuration.  The whole offsets array and 2000 sampled buckets are
    # checked against the oracle's definitions; probe counts of 20000 sampled
    # queries against their multiplicity.
    import torch
    n = V = 1 << 28
    keys = dg.uniform_keys_u32(n, dg.SEED_SCALE)
    dk = to_dev(keys)
    t = hg.build(dk, V)
    rng = np.random.default_rng(0)
    sample = np.unique(rng.integers(0, V, 2000))
    roff, segs, b = sampled_reference(orc, keys, V, 0, sample)
    off = to_np(t.offsets)
    assert np.array_equal(off, roff)
    ck, ci = t.keys, t.ids
    for v, (rk, ri) in segs.items():
        s, e = int(off[v]), int(off[v + 1])
        assert np.array_equal(to_np(ck[s:e]), rk) and np.array_equal(to_np(ci[s:e]), ri)
    q = dg.queries_u32(1 << 28, keys, 0.5, dg.SEED_SCALE + 1)
    dq = to_dev(q)
    counts = to_np(hg.probe(t, dq, binned=True))
    assert np.array_equal(counts, to_np(hg.probe(t, dq, binned=False)))
    del dq
    qi = rng.integers(0, len(q), 20000)
    qs = q[qi]
    qb = orc.buckets(qs, V)
    # multiplicity of each sampled query: count equal keys inside its bucket
    _, segq, _ = sampled_reference(orc, keys, V, 0, np.unique(qb))
    want = np.array([int((segq[int(bb)][0] == x).sum()) for x, bb in zip(qs, qb)], dtype=np.uint32)
    assert np.array_equal(counts[qi], want)
    del t, dk
    torch.cuda.empty_cache()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("binned", [True, False])
def test_build_probe_host_buffers(hg, orc, pinned, binned):
    import torch
    n, V = (1 << 18) + 3, 1 << 18
    keys = dg.uniform_keys_u32(n, 61)
    q = dg.queries_u32(n + 11, keys, 0.5, 62)
    hk = torch.from_numpy(keys.view(np.int32).copy())
    hq = torch.from_numpy(q.view(np.int32).copy())
    hc = torch.zeros(len(q), dtype=torch.int32)
    if pinned:
        hk, hq, hc = hk.pin_memory(), hq.pin_memory(), hc.pin_memory()
    cfg = hg.make_config(hg.KEY_U32, V, 0, "v2")
    dev = "cuda"
    t = hg.Table(torch.empty(V + 1, dtype=torch.uint32, device=dev), torch.empty(n, dtype=torch.uint32, device=dev),
                 torch.empty(n, dtype=torch.uint32, device=dev), cfg)
    ws = torch.empty(hg.build_workspace_size(cfg, n), dtype=torch.uint8, device=dev)
    pws = torch.empty(hg.probe_workspace_size(t, len(q)), dtype=torch.uint8, device=dev) if binned else None
    dk = torch.empty(n, dtype=torch.uint32, device=dev)
    dq = torch.empty(len(q), dtype=torch.uint32, device=dev)
    dc = torch.empty(len(q), dtype=torch.uint32, device=dev)
    hg.build_probe_host(cfg, hk, hq, hc, dk, dq, dc, t, ws, pws)
    torch.cuda.synchronize()
    assert np.array_equal(hc.numpy().view(np.uint32), orc.multiplicity(keys, q))
    off, ck, ci = table_np(t)
    roff, rk, ri = orc.build(keys, V)
    assert np.array_equal(off, roff) and np.array_equal(ck, rk) and np.array_equal(ci, ri)


def test_build_probe_host_refuses_before_copying(hg):
    """The host-buffer call finds argument errors before it enqueues the first
    copy: a probe workspace one byte short, a staging buffer for the queries
    that is missing, or a build workspace one byte short each raise, and the
    device staging buffer for the keys keeps the contents it had."""
    import torch
    n, V = (1 << 12) + 5, 1 << 12
    keys = dg.uniform_keys_u32(n, 71)
    q = dg.queries_u32(n, keys, 0.5, 72)
    hk = torch.from_numpy(keys.view(np.int32).copy()).pin_memory()
    hq = torch.from_numpy(q.view(np.int32).copy()).pin_memory()
    hc = torch.zeros(len(q), dtype=torch.int32).pin_memory()
    cfg = hg.make_config(hg.KEY_U32, V, 0, "v2")
    dev = "cuda"
    t = hg.Table(torch.empty(V + 1, dtype=torch.uint32, device=dev), torch.empty(n, dtype=torch.uint32, device=dev),
                 torch.empty(n, dtype=torch.uint32, device=dev), cfg)
    ws = torch.empty(hg.build_workspace_size(cfg, n), dtype=torch.uint8, device=dev)
    pws = torch.empty(hg.probe_workspace_size(t, len(q)), dtype=torch.uint8, device=dev)
    dk = torch.full((n,), 0x5A5A5A5A, dtype=torch.int32, device=dev).view(torch.uint32)
    dq = torch.empty(len(q), dtype=torch.uint32, device=dev)
    dc = torch.empty(len(q), dtype=torch.uint32, device=dev)
    for bad in ("probe_ws", "d_queries", "build_ws"):
        args = dict(d_queries=dq, ws=ws, probe_ws=pws)
        if bad == "probe_ws":
            args["probe_ws"] = pws[:-1]
        elif bad == "build_ws":
            args["ws"] = ws[:-1]
        else:
            args["d_queries"] = torch.empty(0, dtype=torch.uint32, device=dev)  # a null staging pointer
        with pytest.raises(hg.HGError):
            hg.build_probe_host(cfg, hk, hq, hc, dk, args["d_queries"], dc, t, args["ws"], args["probe_ws"])
        torch.cuda.synchronize()
        assert bool((dk.view(torch.int32) == 0x5A5A5A5A).all()), bad
    hg.build_probe_host(cfg, hk, hq, hc, dk, dq, dc, t, ws, pws)  # the same call with valid arguments
    torch.cuda.synchronize()
    assert np.array_equal(to_np(dk), keys)


def test_build_probe_host_batches_in_flight(hg, orc):
    """Several host-buffer calls on two streams that reuse two sets of device
    staging buffers: every call's counts and last table equal the oracle's
    (the uploads, which queue on the library's copy stream, must wait for the
    earlier call that used the same buffers)."""
    import torch
    n, V, calls = (1 << 17) + 5, 1 << 17, 6
    cfg = hg.make_config(hg.KEY_U32, V, 0, "v2")
    dev = "cuda"
    hosts = []
    for i in range(calls):
        keys = dg.uniform_keys_u32(n, 300 + i)
        q = dg.queries_u32(n, keys, 0.5, 400 + i)
        hosts.append((keys, q, torch.from_numpy(keys.view(np.int32).copy()).pin_memory(),
                      torch.from_numpy(q.view(np.int32).copy()).pin_memory(),
                      torch.zeros(n, dtype=torch.int32).pin_memory()))
    slots = []
    for _ in range(2):
        t = hg.Table(torch.empty(V + 1, dtype=torch.uint32, device=dev), torch.empty(n, dtype=torch.uint32, device=dev),
                     torch.empty(n, dtype=torch.uint32, device=dev), cfg)
        slots.append({"stream": torch.cuda.Stream(), "t": t,
                      "ws": torch.empty(hg.build_workspace_size(cfg, n), dtype=torch.uint8, device=dev),
                      "pws": torch.empty(hg.probe_workspace_size(t, n), dtype=torch.uint8, device=dev),
                      "dk": torch.empty(n, dtype=torch.uint32, device=dev),
                      "dq": torch.empty(n, dtype=torch.uint32, device=dev),
                      "dc": torch.empty(n, dtype=torch.uint32, device=dev)})
    for i in range(calls):
        sl = slots[i % 2]
        _, _, hk, hq, hc = hosts[i]
        hg.build_probe_host(cfg, hk, hq, hc, sl["dk"], sl["dq"], sl["dc"], sl["t"], sl["ws"], sl["pws"],
                            stream=sl["stream"])
    torch.cuda.synchronize()
    for i in range(calls):
        keys, q, _, _, hc = hosts[i]
        assert np.array_equal(hc.numpy().view(np.uint32), orc.multiplicity(keys, q)), i
    for i in (calls - 2, calls - 1):
        off, ck, ci = table_np(slots[i % 2]["t"])
        roff, rk, ri = orc.build(hosts[i][0], V)
        assert np.array_equal(off, roff) and np.array_equal(ck, rk) and np.array_equal(ci, ri), i


@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_any_order_tiles_equal_stable_build(hg, orc, kt):
    """Implicit ids let the partitions rank tiles in any order (the bin build
    restores input order from the ids); explicit ids equal to the positions
    force the stable partitions.  Both must give the canonical table, byte
    for byte, with buckets of many edges (ranked by id) included."""
    n, V = (1 << 21) + 77, 1 << 20
    keys = dg.uniform_keys_u32(n, 41) if kt == "u32" else dg.uniform_keys_u64(n, 41)
    keys[:1500] = keys[1500]  # one bucket of 1501+ edges in a bin that still fits shared memory
    t_any = hg.build(to_dev(keys), V)
    t_stable = hg.build(to_dev(keys), V, ids=to_dev(np.arange(n, dtype=np.uint32)))
    a, b = table_np(t_any), table_np(t_stable)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    roff, rk, ri = orc.build(keys, V)
    assert np.array_equal(a[0], roff) and np.array_equal(a[1], rk) and np.array_equal(a[2], ri)


@pytest.mark.parametrize("mult", [8, 32])
def test_build_duplicates_bins_above_the_double_buffered_size(hg, orc, mult):
    """Keys drawn from [1 .. N/D] at load factor 1: bins of 8192 buckets hold
    8192 edges on average, with a spread that grows with D, so some exceed
    the double-buffered bin build (9216 edges) and take the single-buffered
    second launch; the partitions still rank tiles in any order and every
    bucket (about D edges) is ranked by id.  Canonical table, byte for byte."""
    n = (1 << 22) + 7
    _check_build(hg, orc, dg.dup_keys_u32(n, mult, 15 + mult), 1 << 22)
