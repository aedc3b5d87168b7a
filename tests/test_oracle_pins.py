"""Pins of the CPU oracle against facts that do not come from the oracle itself:
published hash values, closed forms, brute force on tiny inputs, and the
invariants the paper states for a HashGraph table."""
import os

import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


# --- Section 2 "Hashing": Murmur hash ------------------------------------
def test_murmur3_published_values(orc):
    rows = _read_fixture("murmur3_x86_32.txt")
    assert len(rows) == 18
    for row in rows:
        data_hex, seed_hex, want_hex = row.split()
        data = b"" if data_hex == "-" else bytes.fromhex(data_hex)
        assert orc.murmur3_x86_32(data, int(seed_hex, 16)) == int(want_hex, 16), row


def test_murmur3_key_paths_match_byte_definition(orc):
    # u32 keys hash their 4 little-endian bytes, u64 keys their 8 bytes.
    k32 = np.array([0, 1, 0x87654321, 0xFFFFFFFF], dtype=np.uint32)
    k64 = np.array([0, 1, 0x0123456789ABCDEF, 2**64 - 1], dtype=np.uint64)
    for seed in (0, 7, 0x9747B28C):
        h32 = orc.hash_keys(k32, seed)
        h64 = orc.hash_keys(k64, seed)
        for k, h in zip(k32, h32):
            assert h == orc.murmur3_x86_32(int(k).to_bytes(4, "little"), seed)
        for k, h in zip(k64, h64):
            assert h == orc.murmur3_x86_32(int(k).to_bytes(8, "little"), seed)


def test_bucket_is_hash_mod_V(orc):
    keys = dg.uniform_keys_u32(1000, 3)
    h = orc.hash_keys(keys, 5).astype(np.uint64)
    for V in (1, 2, 7, 1000, 1 << 20, (1 << 32) - 1):
        assert np.array_equal(orc.buckets(keys, V, 5), h % np.uint64(V))


def test_hash_spreads_keys_like_poisson(orc):
    # Eq. 1: hash(a) mod V should scatter distinct keys like balls into bins.
    n = V = 1 << 16
    keys = dg.sequence_keys_u32(n)
    lens = np.bincount(orc.buckets(keys, V).astype(np.int64), minlength=V)
    assert abs(lens.mean() - 1.0) < 1e-9
    assert 0.95 < lens.var() < 1.05                  # Poisson(1) variance
    assert abs((lens == 0).mean() - np.exp(-1)) < 0.01  # P(empty) = e^-1


# --- Section 3.1/3.2: the CSR table -----------------------------------------
def _numpy_reference_table(keys, V, seed, orc):
    b = orc.buckets(keys, V, seed)
    perm = np.argsort(b, kind="stable")
    offsets = np.searchsorted(b[perm], np.arange(V + 1, dtype=np.uint64), side="left")
    return offsets.astype(np.uint32), keys[perm], perm.astype(np.uint32)


@pytest.mark.parametrize("n,V", [(0, 1), (1, 1), (33, 7), (1000, 1), (1000, 64), (5000, 5003), (4096, 1 << 14)])
def test_build_matches_stable_grouping(orc, n, V):
    keys = dg.uniform_keys_u32(n, 11)
    off, ck, ci = orc.build(keys, V, seed=1)
    roff, rk, ri = _numpy_reference_table(keys, V, 1, orc)
    assert np.array_equal(off, roff) and np.array_equal(ck, rk) and np.array_equal(ci, ri)
    assert orc.check_table(off, ck, ci, keys, V, seed=1) == []


def test_build_u64_and_explicit_ids(orc):
    keys = dg.zipf_keys_u64(3000, 200, 5)
    ids = (np.arange(3000, dtype=np.uint32) * 7 + 3)
    off, ck, ci = orc.build(keys, 512, seed=9, ids=ids)
    roff, rk, rperm = _numpy_reference_table(keys, 512, 9, orc)
    assert np.array_equal(off, roff) and np.array_equal(ck, rk)
    assert np.array_equal(ci, ids[rperm])


def test_table_invariants_detect_planted_mistakes(orc):
    keys = dg.dup_keys_u32(2000, 4, 2)
    off, ck, ci = orc.build(keys, 256)
    assert orc.check_table(off, ck, ci, keys, 256) == []
    # swap two ids inside one bucket -> order violated
    lens = np.diff(off.astype(np.int64))
    v = int(np.argmax(lens))
    ci2 = ci.copy()
    ci2[off[v]], ci2[off[v] + 1] = ci2[off[v] + 1], ci2[off[v]]
    assert orc.check_table(off, ck, ci2, keys, 256) != []
    # move one boundary -> an edge lands outside its bucket
    off2 = off.copy()
    off2[v + 1] += 1
    assert orc.check_table(off2, ck, ci, keys, 256) != []
    # drop the last edge -> offsets no longer end at N
    assert orc.check_table(off[:-1].tolist() + [off[-1] - 1], ck, ci, keys, 256) != []


def test_fig1_worked_example(orc):
    rows = dict(r.split(":", 1) for r in _read_fixture("fig1_example.txt"))
    inputs = np.array([int(x) for x in rows["inputs"].split()], dtype=np.uint32)
    V = int(rows["range"])
    # pick the first seed under which 3 and 10121 collide, as in the figure
    seed = next(s for s in range(1000) if orc.buckets(inputs[:2], V, s)[0] == orc.buckets(inputs[:2], V, s)[1])
    off, ck, ci = orc.build(inputs, V, seed)
    assert off[-1] == int(rows["expect_table_size"])
    v3 = int(orc.buckets(inputs[:1], V, seed)[0])
    seg = ck[off[v3]:off[v3 + 1]]
    assert sorted(seg.tolist()) == sorted([3, 3, 10121]) and list(ci[off[v3]:off[v3 + 1]]) == [0, 1, 2]
    assert (np.diff(off.astype(np.int64)) == 0).any()       # some hash value owns no input


# --- Section 3.4: probing -------------------------------------------------
def test_probe_equals_multiplicity(orc):
    keys = dg.dup_keys_u32(4000, 3, 4)
    q = dg.queries_u32(3000, keys, 0.5, 6)
    for V in (1, 97, 4096):
        off, ck, _ = orc.build(keys, V, 2)
        assert np.array_equal(orc.probe(off, ck, q, V, 2), orc.multiplicity(keys, q))


def test_multiplicity_brute_force(orc):
    keys = dg.dup_keys_u32(300, 5, 1)
    q = dg.queries_u32(200, keys, 0.7, 8)
    brute = (q[:, None] == keys[None, :]).sum(axis=1)
    assert np.array_equal(orc.multiplicity(keys, q), brute)


def test_probe_sequence_input_all_ones(orc):
    keys = dg.sequence_keys_u32(1 << 14)                  # the paper's default input
    off, ck, _ = orc.build(keys, 1 << 13)
    assert np.all(orc.probe(off, ck, keys, 1 << 13) == 1)


def test_probe_guaranteed_misses(orc):
    keys = dg.uniform_keys_u32(5000, 3)
    q = dg.queries_u32(5000, keys, 0.0, 3)
    off, ck, _ = orc.build(keys, 4096)
    assert not np.isin(q, keys).any()
    assert np.all(orc.probe(off, ck, q, 4096) == 0)


# --- Alg. 3: bucket-wise intersection -------------------------------------
@pytest.mark.parametrize("V", [1, 13, 256])
def test_join_count_closed_form_and_brute(orc, V):
    a = dg.dup_keys_u32(700, 6, 1)
    b = dg.dup_keys_u32(500, 3, 2)
    offA, kA, _ = orc.build(a, V, 3)
    offB, kB, _ = orc.build(b, V, 3)
    tot, per = orc.join_count(offA, kA, offB, kB, V)
    assert tot == int(per.sum())
    assert tot == orc.join_size_by_keys(a, b)
    assert tot == int((a[:, None] == b[None, :]).sum())


def test_join_materialize_pairs_and_order(orc):
    a = dg.zipf_keys_u64(600, 50, 1)
    b = dg.uniform_domain_keys_u64(400, 50, 2)
    V = 64
    offA, kA, iA = orc.build(a, V, 5)
    offB, kB, iB = orc.build(b, V, 5)
    pa, pb = orc.join_materialize(offA, kA, iA, offB, kB, iB, V)
    ii, jj = np.nonzero(a[:, None] == b[None, :])
    assert len(pa) == len(ii)
    got = sorted(zip(pa.tolist(), pb.tolist()))
    assert got == sorted(zip(ii.tolist(), jj.tolist()))
    # canonical order: bucket, then position in A's CSR, then position in B's CSR
    posA = np.empty(len(a), np.int64); posA[iA] = np.arange(len(a))
    posB = np.empty(len(b), np.int64); posB[iB] = np.arange(len(b))
    bk = orc.buckets(a[pa], V, 5).astype(np.int64)
    key = np.stack([bk, posA[pa], posB[pb]], axis=1)
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    assert np.array_equal(order, np.arange(len(pa)))


def test_join_count_map_independent(orc):
    # The join size does not depend on the bucket map (Alg. 3 only needs both
    # tables to use the same V and hash).
    a = dg.dup_keys_u32(900, 4, 7)
    b = dg.dup_keys_u32(900, 4, 8)
    sizes = set()
    for V, seed in ((1, 0), (31, 1), (512, 2), (4096, 3)):
        offA, kA, _ = orc.build(a, V, seed)
        offB, kB, _ = orc.build(b, V, seed)
        sizes.add(orc.join_count(offA, kA, offB, kB, V)[0])
    assert len(sizes) == 1


def test_bucket_counts_is_the_histogram_of_the_bucket_map(orc):
    # the large-table checks compare GPU offsets with this histogram's
    # exclusive prefix; it must equal the build's offsets and numpy's count
    keys = dg.dup_keys_u32(50_000, 3, 17)
    for V in (1, 97, 1 << 12):
        c = orc.bucket_counts(keys, V, seed=5)
        assert np.array_equal(c, np.bincount(orc.buckets(keys, V, 5).astype(np.int64), minlength=V))
        off, _, _ = orc.build(keys, V, 5)
        assert np.array_equal(np.concatenate([[0], np.cumsum(c)]).astype(np.uint32), off)
