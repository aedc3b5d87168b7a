"""Parity at the benchmark's full sizes for the join and learned-map workloads.

The oracle cannot build 2^27-key tables in seconds, so these tests check
the GPU results against facts the oracle and the mathematics fix at any size:

* join (Alg. 3): the inner-join size and every bucket's pair count equal
  the closed form sum_k m_A(k) m_B(k) (multiplicities from numpy sorts),
  grouped by the oracle's bucket map; the materialised pairs of sampled
  buckets (the Zipf side's hot bucket among them) equal the oracle's
  bucket-by-bucket intersection of the canonical segments, at the output
  positions the per-bucket counts give; both tables' complete offsets equal
  the oracle's bucket histogram.
* learned map: the complete offsets of a table built with the GPU-trained
  model equal the histogram of the oracle's inference with the same model,
  sampled buckets hold the canonical segments, the probe counts equal the
  Murmur table's for every query and the multiplicity for sampled queries.

Inputs are the benchmark's: 2^27 uint64 keys each, V = 2^27.
"""
import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg
from gpu_util import sampled_reference, to_dev, to_np

pytestmark = pytest.mark.gpu

N = 1 << 27
V = 1 << 27


def _check_table_sampled(t, ref_off, segs):
    off = to_np(t.offsets)
    assert np.array_equal(off, ref_off), "offsets differ from the oracle's bucket histogram"
    for v, (rk, ri) in segs.items():
        s, e = int(off[v]), int(off[v + 1])
        assert np.array_equal(to_np(t.keys[s:e]), rk), f"bucket {v}: keys"
        assert np.array_equal(to_np(t.ids[s:e]), ri), f"bucket {v}: ids"
    return off


def test_join_full_size_zipf_vs_uniform(hg, orc):
    import torch
    distinct = 1 << 24
    a = dg.zipf_keys_u64(N, distinct, dg.SEED_JOIN, 1.0)
    b = dg.uniform_domain_keys_u64(N, distinct, dg.SEED_JOIN + 1)
    # closed form: multiplicities of every key on both sides
    ua, ca = np.unique(a, return_counts=True)
    ub, cb = np.unique(b, return_counts=True)
    common, ia, ib = np.intersect1d(ua, ub, assume_unique=True, return_indices=True)
    prod = ca[ia].astype(np.int64) * cb[ib].astype(np.int64)
    want_total = int(prod.sum())
    cbk = orc.buckets(common, V).astype(np.int64)
    want_per = np.bincount(cbk, weights=prod.astype(np.float64), minlength=V)
    assert want_per.max() < 2 ** 52
    want_per = want_per.astype(np.int64)
    del ua, ub, ca, cb, ia, ib, prod
    hot = int(orc.buckets(dg.scramble64(np.array([1], dtype=np.uint64)), V)[0])   # the rank-1 key's bucket
    rng = np.random.default_rng(5)
    nz = np.nonzero(want_per)[0]
    sample = np.unique(np.concatenate([rng.choice(nz, 200, replace=False), [hot, 0, V - 1]]))
    offA, segA, _ = sampled_reference(orc, a, V, 0, sample)
    offB, segB, _ = sampled_reference(orc, b, V, 0, sample)

    tA = hg.build(to_dev(a), V)
    tB = hg.build(to_dev(b), V)
    _check_table_sampled(tA, offA, segA)
    _check_table_sampled(tB, offB, segB)
    total, per = hg.join_count(tA, tB)
    assert int(total.item()) == want_total
    assert np.array_equal(to_np(per), want_per)
    del per
    torch.cuda.empty_cache()
    # materialised pairs of the sampled buckets, in canonical order at their
    # output positions (exclusive prefix of the per-bucket counts)
    jws = torch.empty(hg.join_workspace_size(tA.cfg, N, N), dtype=torch.uint8, device="cuda")
    for after_count in (True, False):
        if after_count:   # the count pass leaves its per-edge counts in jws for the materialisation
            hg.join_count(tA, tB, per_bucket=False, ws=jws)
        pa, pb = hg.join_materialize(tA, tB, capacity=want_total, ws=jws, after_count=after_count)
        assert hg.workspace_status(jws) == 0
        assert pa.numel() == want_total
        start = np.concatenate([[0], np.cumsum(want_per)])
        for v in sample.tolist():
            ka, ida = segA[v]
            kb, idb = segB[v]
            ra, rb = orc.join_materialize(np.array([0, len(ka)], dtype=np.uint32), ka, ida,
                                          np.array([0, len(kb)], dtype=np.uint32), kb, idb, 1)
            s, e = int(start[v]), int(start[v + 1])
            assert e - s == len(ra), f"bucket {v}: pair count"
            assert np.array_equal(to_np(pa[s:e]), ra) and np.array_equal(to_np(pb[s:e]), rb), f"bucket {v}"
        assert int(want_per[hot]) > 10_000_000          # the hot bucket was among the checked ones
        del pa, pb
        torch.cuda.empty_cache()
    del tA, tB, jws
    torch.cuda.empty_cache()


def test_learned_full_size_lognormal_mixture(hg, orc):
    import torch
    keys = dg.lognormal_mixture_u64(N, dg.SEED_LEARNED)
    q = dg.queries_u64(N, keys, 0.5, dg.SEED_LEARNED + 1)
    dk = to_dev(keys)
    model, diag = hg.learned_train(dk, V)
    assert diag["sample_size"] == N // 100
    blob = to_np(model).view(np.uint8)
    rng = np.random.default_rng(9)
    sample = np.unique(np.concatenate([rng.integers(0, V, 300), [0, V - 1]]))
    roff, segs, bk = sampled_reference(orc, keys, V, 0, sample, model=blob)
    t = hg.build(dk, V, model=model)
    off = _check_table_sampled(t, roff, segs)
    # key-range order: first keys of the non-empty buckets ascend
    ne = np.nonzero(np.diff(off.astype(np.int64)) > 0)[0]
    first = t.keys.view(torch.int64)[torch.from_numpy(off[ne].astype(np.int64)).cuda()].cpu().numpy().view(np.uint64)
    assert np.all(first[1:] >= first[:-1])
    # the judge (Murmur) keeps the learned map on these keys
    chosen, rep = hg.choose_map(dk, V, model)
    print(f"\nlearned: max {rep['learned']['max']:.0f} var {rep['learned']['var']:.4f}; "
          f"murmur: max {rep['murmur']['max']:.0f} var {rep['murmur']['var']:.4f}")
    assert rep["kept"] and chosen is model
    # probe: identical to the Murmur table's counts for every query, the
    # multiplicity for sampled queries
    dq = to_dev(q)
    counts = hg.probe(t, dq, binned=True)
    tm = hg.build(dk, V)
    counts_m = hg.probe(tm, dq, binned=True)
    assert torch.equal(counts.view(torch.int32), counts_m.view(torch.int32))
    del tm, counts_m
    qi = rng.integers(0, N, 200_000)
    sk = np.sort(keys)
    want = (np.searchsorted(sk, q[qi], side="right") - np.searchsorted(sk, q[qi], side="left")).astype(np.uint32)
    assert np.array_equal(to_np(counts)[qi], want)
    del t, dk, dq, counts
    torch.cuda.empty_cache()
