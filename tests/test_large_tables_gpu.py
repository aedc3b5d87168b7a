"""Tables larger than one two-level plan holds: 2^30 and 2^31 uint32 keys
into as many buckets (load factor 1), built with one more relabeling level
(Section 3.3, "Larger Inputs": a stable partition by slab of 2^28 buckets,
then the two-level build of every slab), and 2^28 uint64 keys (two slabs of
2^27 buckets).

The oracle cannot build such tables in seconds, so the checks use what it
fixes at any size: the complete offsets array equals the exclusive prefix of
the oracle's bucket histogram; sampled buckets (across every slab, the slab
edges among them) hold exactly the oracle's canonical segments (keys and
ids in ascending input position); probe counts of sampled queries equal
their multiplicity, and the binned probe equals the direct one for all
queries.  Keys and queries are drawn on the device by the GPU copy of the
input recipes (checked equal to the host recipes below)."""
import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def test_device_recipes_draw_the_host_numbers(hg):
    import paper_1907_02900_gb300.datagen_gpu as dgg
    n, q = (1 << 20) + 5, (1 << 19) + 3
    keys = dgg.uniform_keys_u32(n, 77)
    want = dg.uniform_keys_u32(n, 77)
    assert np.array_equal(to_np(keys), want)
    assert np.array_equal(to_np(dgg.queries_u32(q, keys, 0.5, 78)), dg.queries_u32(q, want, 0.5, 78))


def _segments(orc, keys: np.ndarray, V: int, sample: np.ndarray, chunk: int = 1 << 26):
    """Canonical segment (keys, input positions) of every sampled bucket,
    computed chunk by chunk so that no per-key array of the whole input is
    held at once."""
    mark = np.zeros(V, dtype=bool)
    mark[sample] = True
    parts = {int(v): ([], []) for v in sample}
    for c0 in range(0, len(keys), chunk):
        b = orc.buckets(keys[c0:c0 + chunk], V).astype(np.int64)
        pos = np.nonzero(mark[b])[0]
        bs = b[pos]
        order = np.argsort(bs, kind="stable")
        pos, bs = pos[order], bs[order]
        cuts = np.flatnonzero(np.diff(bs)) + 1
        for grp in np.split(np.arange(len(pos)), cuts):
            if len(grp):
                v = int(bs[grp[0]])
                parts[v][0].append(keys[c0 + pos[grp]])
                parts[v][1].append((c0 + pos[grp]).astype(np.uint32))
    return {v: (np.concatenate(k) if k else np.zeros(0, keys.dtype),
                np.concatenate(i) if i else np.zeros(0, np.uint32)) for v, (k, i) in parts.items()}


def _check_large(hg, orc, keys_d, V, qn=1 << 26):
    import torch
    import paper_1907_02900_gb300.datagen_gpu as dgg
    keys = to_np(keys_d)
    t = hg.build(keys_d, V)
    off = to_np(t.offsets)
    counts = orc.bucket_counts(keys, V)
    want_off = np.zeros(V + 1, dtype=np.uint32)
    np.cumsum(counts, dtype=np.uint32, out=want_off[1:])
    assert np.array_equal(off, want_off), "offsets differ from the oracle's bucket histogram"
    del counts, want_off
    # sampled buckets: random ones plus the first and last bucket of every slab of 2^28
    rng = np.random.default_rng(3)
    slab_edges = [v for s0 in range(0, V, 1 << 28) for v in (s0, s0 + 1, min(s0 + (1 << 28), V) - 1)]
    sample_q = None
    if keys_d.dtype == torch.uint32:
        dq = dgg.queries_u32(qn, keys_d, 0.5, 4242)
        q = to_np(dq)
        qi = rng.integers(0, qn, 20_000)
        sample_q = (qi, q[qi], orc.buckets(q[qi], V).astype(np.int64))
    extra = sample_q[2] if sample_q is not None else np.zeros(0, np.int64)
    sample = np.unique(np.concatenate([rng.integers(0, V, 1500), slab_edges, extra]))
    segs = _segments(orc, keys, V, sample)
    for v in np.unique(np.concatenate([rng.choice(sample, 1500, replace=False), slab_edges])).tolist():
        rk, ri = segs[v]
        s, e = int(off[v]), int(off[v + 1])
        assert np.array_equal(to_np(t.keys[s:e]), rk), f"bucket {v}: keys"
        assert np.array_equal(to_np(t.ids[s:e]), ri), f"bucket {v}: ids"
    if sample_q is not None:
        qi, qs, qb = sample_q
        counts_b = hg.probe(t, dq, binned=True)
        counts_d = hg.probe(t, dq, binned=False)
        assert torch.equal(counts_b.view(torch.int32), counts_d.view(torch.int32))
        got = to_np(counts_b)[qi]
        want = np.array([int((segs[int(bb)][0] == x).sum()) for x, bb in zip(qs, qb)], dtype=np.uint32)
        assert np.array_equal(got, want)
    del t
    torch.cuda.empty_cache()


@pytest.mark.parametrize("log2n", [30, 31])
def test_uint32_tables_beyond_one_two_level_plan(hg, orc, log2n):
    import torch
    import paper_1907_02900_gb300.datagen_gpu as dgg
    n = V = 1 << log2n
    keys_d = dgg.uniform_keys_u32(n, dg.SEED_SCALE + log2n)
    _check_large(hg, orc, keys_d, V)
    del keys_d
    torch.cuda.empty_cache()


def test_uint64_table_of_2e28_keys_in_two_slabs(hg, orc):
    import torch
    n = V = 1 << 28
    keys = dg.uniform_keys_u64(n, 91)
    _check_large(hg, orc, to_dev(keys), V)
    torch.cuda.empty_cache()
