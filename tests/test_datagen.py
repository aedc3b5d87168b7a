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
