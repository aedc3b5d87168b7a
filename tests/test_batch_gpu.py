"""Batched tables on the GPU vs the CPU oracle, table by table: every table
of a batch equals the oracle's table of its keys alone (offsets shifted by
the table's first position), every count equals the multiplicity.  Also:
results do not depend on the configuration the autotuner picks, the plain
per-table loop gives the same tables, graph replays see new inputs, and the
GPU input generator draws the host generator's numbers."""
import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def _plan_and_data(hg, sizes, qsizes, seed, V=None, hit=0.5):
    plan = hg.BatchPlan(sizes, qsizes, num_buckets=V, seed=seed)
    keys = dg.batched_keys_u32(sizes, seed + 1)
    queries = dg.batched_queries_u32(qsizes, keys, sizes, hit, seed + 2)
    b = plan.alloc()
    b["keys"].copy_(to_dev(plan.pad_keys(keys)))
    b["queries"].copy_(to_dev(plan.pad_queries(queries)))
    return plan, b, keys, queries


def _check_tables(orc, plan, b, keys, queries, tables, local_offsets=False):
    ub = np.concatenate([[0], np.cumsum(plan.sizes.astype(np.int64))])
    qb = np.concatenate([[0], np.cumsum(plan.qsizes.astype(np.int64))])
    for t in tables:
        off, ck, ci, cnt = (to_np(x) for x in plan.table(b, t))
        kt = keys[ub[t]:ub[t + 1]]
        qt = queries[qb[t]:qb[t + 1]]
        V = plan.num_buckets(t)
        roff, rk, ri = orc.build(kt, V, seed=plan.seed)
        shift = 0 if local_offsets else int(plan.key_begin[t])
        assert np.array_equal(off.astype(np.int64) - shift, roff.astype(np.int64)), t
        assert np.array_equal(ck, rk) and np.array_equal(ci, ri), t
        assert np.array_equal(cnt, orc.multiplicity(kt, qt)), t


def _ragged_sizes():
    s = list(dg.batched_sizes(200, 7, lo_log2=0.0, hi_log2=16.0))
    s[:8] = [0, 1, 2, 3, 4, 5, 0, 7]          # empty tables and every padding length
    q = [int(x) // 2 + (i % 3) for i, x in enumerate(s)]
    q[5] = 0
    return np.array(s, dtype=np.int64), np.array(q, dtype=np.int64)


def test_batch_matches_oracle_table_by_table(hg, orc):
    sizes, qsizes = _ragged_sizes()
    seed = 0x5A17
    plan, b, keys, queries = _plan_and_data(hg, sizes, qsizes, seed)
    plan.run(b)
    assert hg.workspace_status(b["ws"]) == 0
    _check_tables(orc, plan, b, keys, queries, range(plan.T))
    # the closing entry of the offsets array
    assert int(to_np(b["offsets"])[-1]) == plan.total_keys


def test_batch_bucket_counts_and_multiwave(hg, orc):
    # uneven V_t (load factors 1/4 .. 8) and a bin size small enough that the
    # batch needs several waves
    sizes, qsizes = _ragged_sizes()
    V = np.maximum(1, (sizes * np.array([0.25, 1, 3, 8])[np.arange(len(sizes)) % 4]).astype(np.int64))
    seed = 0x5A18
    plan, b, keys, queries = _plan_and_data(hg, sizes, qsizes, seed, V=V)
    plan.set_config(bin_shift=4, threads_per_bin=512)
    assert plan.config()["waves"] > 1
    plan.run(b)
    _check_tables(orc, plan, b, keys, queries, range(plan.T))


def test_batch_results_do_not_depend_on_configuration(hg, orc):
    sizes = dg.batched_sizes(300, 11, total=1 << 21)
    qsizes = sizes.copy()
    seed = 0x5A19
    plan, b, keys, queries = _plan_and_data(hg, sizes, qsizes, seed)
    ref = None
    for s in (9, 10, 11, 12):
        for tpb in (512, 1024):
            plan.set_config(bin_shift=s, threads_per_bin=tpb)
            plan.run(b)
            got = [to_np(b[k]).copy() for k in ("offsets", "csr_keys", "csr_ids", "counts")]
            if ref is None:
                ref = got
                _check_tables(orc, plan, b, keys, queries, [0, 1, 2, int(np.argmax(sizes)), plan.T - 1])
            else:
                for g, r in zip(got, ref):
                    assert np.array_equal(g, r), (s, tpb)
    tuned = plan.autotune(b, reps=1)
    assert tuned["ms"] > 0 and tuned["threads_per_bin"] in (512, 1024)
    plan.run(b)
    for k, r in zip(("offsets", "csr_keys", "csr_ids", "counts"), ref):
        assert np.array_equal(to_np(b[k]), r)


def test_plain_loop_gives_the_same_tables(hg, orc):
    sizes, qsizes = _ragged_sizes()
    seed = 0x5A1A
    plan, b, keys, queries = _plan_and_data(hg, sizes, qsizes, seed)
    plan.run(b)
    batched = {k: to_np(b[k]).copy() for k in ("offsets", "csr_keys", "csr_ids", "counts")}
    plan.run_plain(b)
    _check_tables(orc, plan, b, keys, queries, range(plan.T), local_offsets=True)
    for t in range(plan.T):
        o0, o1 = int(plan.offset_begin[t]), int(plan.offset_begin[t + 1])
        k0, k1 = int(plan.key_begin[t]), int(plan.key_begin[t]) + int(sizes[t])
        assert np.array_equal(to_np(b["offsets"])[o0:o1].astype(np.int64) + k0, batched["offsets"][o0:o1])
        assert np.array_equal(to_np(b["csr_keys"])[k0:k1], batched["csr_keys"][k0:k1])


def test_graph_replay_reads_new_inputs(hg, orc):
    sizes, qsizes = _ragged_sizes()
    seed = 0x5A1B
    plan, b, keys, queries = _plan_and_data(hg, sizes, qsizes, seed)
    plan.run(b)
    keys2 = dg.batched_keys_u32(sizes, seed + 9)
    queries2 = dg.batched_queries_u32(qsizes, keys2, sizes, 0.7, seed + 10)
    b["keys"].copy_(to_dev(plan.pad_keys(keys2)))
    b["queries"].copy_(to_dev(plan.pad_queries(queries2)))
    plan.run(b)   # same buffers: the captured graph is replayed
    _check_tables(orc, plan, b, keys2, queries2, range(0, plan.T, 7))


def test_gpu_datagen_draws_the_host_numbers(hg):
    import paper_1907_02900_gb300.datagen_gpu as dgg
    sizes, qsizes = _ragged_sizes()
    plan = hg.BatchPlan(sizes, qsizes, seed=1)
    b = plan.alloc()
    dgg.fill_batch(plan, b, key_seed=41, query_seed=42, hit_rate=0.5)
    keys = dg.batched_keys_u32(sizes, 41)
    queries = dg.batched_queries_u32(qsizes, keys, sizes, 0.5, 42)
    assert np.array_equal(to_np(b["keys"]), plan.pad_keys(keys))
    assert np.array_equal(to_np(b["queries"]), plan.pad_queries(queries))


@pytest.mark.slow
def test_full_size_batch_sampled_parity(hg, orc):
    """The batched workload at full size (10,000 tables, log-uniform sizes
    scaled to a 2^30 total, 50% hits), autotuned and graph-launched as the
    benchmark runs it; sampled tables (largest, smallest, random) checked
    against the oracle, all counts checked against a property."""
    import paper_1907_02900_gb300.datagen_gpu as dgg
    T = 10_000
    sizes = dg.batched_sizes(T, dg.SEED_BATCH, total=(1 << 30) - 4 * T)
    qsizes = sizes.copy()
    plan = hg.BatchPlan(sizes, qsizes, seed=dg.SEED_BATCH)
    b = plan.alloc()
    dgg.fill_batch(plan, b, key_seed=dg.SEED_BATCH + 1, query_seed=dg.SEED_BATCH + 2, hit_rate=0.5)
    plan.autotune(b, reps=1)
    plan.run(b)
    assert hg.workspace_status(b["ws"]) == 0
    rng = np.random.default_rng(5)
    pick = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), 0, T - 1, *rng.choice(T, 12, replace=False).tolist()})
    ub = np.concatenate([[0], np.cumsum(sizes.astype(np.int64))])
    qub = np.concatenate([[0], np.cumsum(qsizes.astype(np.int64))])
    for t in pick:
        kt = dg.uniform_keys_u32(int(sizes[t]), dg.SEED_BATCH + 1, start=int(ub[t]))
        qt = dg.batched_table_queries_u32(int(qsizes[t]), int(qub[t]), kt, 0.5, dg.SEED_BATCH + 2)
        off, ck, ci, cnt = (to_np(x) for x in plan.table(b, t))
        roff, rk, ri = orc.build(kt, plan.num_buckets(t), seed=dg.SEED_BATCH)
        assert np.array_equal(off.astype(np.int64) - int(plan.key_begin[t]), roff.astype(np.int64)), t
        assert np.array_equal(ck, rk) and np.array_equal(ci, ri), t
        assert np.array_equal(cnt, orc.multiplicity(kt, qt)), t
    # every query: a hit key occurs in its table (count >= 1), a miss never does
    # (misses are drawn from the upper half of the preimages); about half hit
    cnt = to_np(b["counts"])
    qb = plan.query_begin[:-1].astype(np.int64)
    real = np.repeat(qb, qsizes) + (np.arange(int(qsizes.sum())) - np.repeat(np.cumsum(qsizes) - qsizes, qsizes))
    frac = np.mean(cnt[real] > 0)
    assert 0.49 < frac < 0.51
