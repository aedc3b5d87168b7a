"""Seeded input generators: determinism and the structure each workload promises."""
import numpy as np

from paper_1907_02900_gb300 import datagen as dg


def test_splitmix64_counter_based_and_deterministic():
    a = dg.splitmix64_range(1, 2, 0, 1000)
    b = dg.splitmix64(1, 2, np.arange(500, 1000, dtype=np.uint64))
    assert np.array_equal(a[500:], b)
    assert len(np.unique(a)) == 1000
    assert not np.array_equal(a, dg.splitmix64_range(1, 3, 0, 1000))


def test_splitmix64_published_sequence():
    # SplitMix64 with state 0: first output is mix64(gamma) = 0xE220A8397B1DCDAF
    # (the published reference sequence of the generator, seeded with 0).
    z = dg._mix64(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))[0]
    assert int(z) == 0xE220A8397B1DCDAF


def test_scramblers_are_bijective_on_samples():
    x = np.arange(1 << 20, dtype=np.uint64)
    assert len(np.unique(dg.scramble32(x))) == 1 << 20
    assert len(np.unique(dg.scramble64(x * np.uint64(0x100000001)))) == 1 << 20


def test_queries_hit_rate_and_misses():
    keys = dg.uniform_keys_u32(1 << 16, 1)
    for rate in (0.0, 0.5, 1.0):
        q = dg.queries_u32(1 << 16, keys, rate, 2)
        hits = np.isin(q, keys).mean()
        assert abs(hits - rate) < 0.01


def test_dup_keys_average_multiplicity():
    k = dg.dup_keys_u32(1 << 16, 8, 3)
    assert k.min() >= 1 and k.max() <= (1 << 16) // 8
    assert abs(len(k) / len(np.unique(k)) - 8) < 0.1


def test_zipf_top_rank_share():
    r = dg.zipf_ranks(1 << 18, 1 << 12, 4)
    h = sum(1.0 / k for k in range(1, (1 << 12) + 1))
    assert abs((r == 1).mean() - 1.0 / h) < 0.005
    assert r.min() >= 1 and r.max() <= 1 << 12


def test_lognormal_mixture_shape():
    k = dg.lognormal_mixture_u64(1 << 16, 5)
    assert k.dtype == np.uint64
    frac_dup = 1 - len(np.unique(k)) / len(k)
    assert frac_dup < 0.01
    # roughly 10% uniform words: most of them exceed 2^56
    assert 0.08 < (k > np.uint64(1 << 56)).mean() < 0.14


def test_batched_sizes_log_uniform():
    s = dg.batched_table_sizes(10000, 7)
    assert s.min() >= 1024 and s.max() < 1 << 22
    lg = np.log2(s)
    assert abs(lg.mean() - 16.0) < 0.15


def test_batched_recipes_agree_table_by_table():
    sizes = dg.batched_sizes(40, 3, lo_log2=0.0, hi_log2=10.0)
    sizes[:3] = [0, 1, 5]
    keys = dg.batched_keys_u32(sizes, 8)
    q = dg.batched_queries_u32(sizes, keys, sizes, 0.5, 9)
    ub = np.concatenate([[0], np.cumsum(sizes)])
    for t in range(len(sizes)):
        kt = dg.uniform_keys_u32(int(sizes[t]), 8, start=int(ub[t]))
        assert np.array_equal(keys[ub[t]:ub[t + 1]], kt)
        qt = dg.batched_table_queries_u32(int(sizes[t]), int(ub[t]), kt, 0.5, 9)
        assert np.array_equal(q[ub[t]:ub[t + 1]], qt)
    # about half the queries are keys of their own table
    assert 0.4 < np.mean(np.isin(q, keys)) < 0.6


def test_batched_sizes_total_and_shape():
    n = dg.batched_sizes(10_000, dg.SEED_BATCH, total=(1 << 30) - 40_000)
    assert n.sum() <= (1 << 30) - 40_000 and n.sum() > (1 << 30) - 50_000 and n.min() >= 1
    raw = dg.batched_table_sizes(10_000, dg.SEED_BATCH)
    assert raw.min() >= 1 << 10 and raw.max() < 1 << 22
    # log-uniform: log2 sizes spread evenly over [10, 22)
    h, _ = np.histogram(np.log2(raw), bins=12, range=(10, 22))
    assert h.min() > 700 and h.max() < 980


def test_zipf_inverse_shortcut_equals_binary_search():
    # the s = 1 shortcut must draw exactly the ranks of the binary search
    for nd in (1, 2, 3, 100, 4000, 1 << 17):
        cdf = dg.zipf_cdf(nd)
        u = dg.unit_double(dg.splitmix64_range(5, dg.STREAM_ZIPF, 0, 1 << 18))
        u = np.concatenate([u, [0.0, np.nextafter(1.0, 0), cdf[0], np.nextafter(cdf[0], 0), 1.0]])
        assert np.array_equal(dg._zipf1_inverse(cdf, u), np.searchsorted(cdf, u, side="right")), nd
