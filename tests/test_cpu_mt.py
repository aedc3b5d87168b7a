"""The multithreaded CPU HashGraph against the oracle, byte for byte: the
canonical table for every thread count, key width, id array, load factor and
duplicate multiplicity, and the Probe-Standard counts."""
import numpy as np
import pytest

import cpu_baseline as cmt
from paper_1907_02900_gb300 import datagen as dg


def _same_table(orc, keys, V, seed=0, ids=None, threads=0):
    off, ck, ci = cmt.build(keys, V, seed, ids=ids, threads=threads)
    roff, rk, ri = orc.build(keys, V, seed, ids=ids)
    assert np.array_equal(off, roff), "offsets differ"
    assert np.array_equal(ck, rk), "csr keys differ"
    assert np.array_equal(ci, ri), "csr ids differ"
    return off, ck, ci


@pytest.mark.parametrize("threads", [1, 3, 8])
@pytest.mark.parametrize("n,V", [(1, 1), (33, 7), (5000, 1), (100_000, 100_003), (1 << 17, 1 << 12),
                                 (70_001, 1 << 20)])
def test_build_u32_matches_oracle(orc, n, V, threads):
    _same_table(orc, dg.uniform_keys_u32(n, 21), V, seed=5, threads=threads)


def test_build_u64_explicit_ids_and_duplicates(orc):
    keys = dg.uniform_keys_u64(60_001, 4)
    ids = (np.arange(len(keys), dtype=np.uint64) * 2654435761 % (1 << 32)).astype(np.uint32)
    _same_table(orc, keys, 1 << 15, ids=ids, threads=4)
    for mult in (4, 32, 5000):
        _same_table(orc, dg.dup_keys_u32(80_000, mult, 6), 1 << 16, threads=6)


def test_build_empty_and_all_equal(orc):
    off, ck, ci = cmt.build(np.empty(0, dtype=np.uint32), 9)
    assert np.array_equal(off, np.zeros(10, dtype=np.uint32)) and len(ck) == 0 and len(ci) == 0
    _same_table(orc, np.full(20_000, 77, dtype=np.uint32), 1 << 10, threads=5)


@pytest.mark.parametrize("hit", [0.0, 0.5, 1.0])
def test_probe_matches_oracle(orc, hit):
    keys = dg.dup_keys_u32(50_000, 3, 2)
    q = dg.queries_u32(40_000, keys, hit, 3)
    V = 1 << 14
    off, ck, _ = cmt.build(keys, V, threads=4)
    counts = cmt.probe(off, ck, V, q, threads=4)
    assert np.array_equal(counts, orc.probe(off, ck, q, V))
    assert np.array_equal(counts, orc.multiplicity(keys, q))


def test_invalid_arguments_rejected():
    with pytest.raises(ValueError):
        cmt.build(np.arange(4, dtype=np.uint32), 0)
    with pytest.raises(ValueError):
        cmt.build(np.arange(4, dtype=np.uint32), (1 << 32) + 1)
    with pytest.raises(TypeError):
        cmt.build(np.arange(4, dtype=np.int16), 8)
    assert cmt.max_threads() >= 1
