"""Learned bucket map on the GPU vs the CPU oracle: the sample, the knots,
the gradients of the root and leaf losses, convergence of the trained knot
values to the closed-form least-squares optimum, the model blob, and
bit-exact build / probe / join with the learned map.  Also what the trained
model gains: over its own initialisation (loss) and over Murmur (key-range
order of the table)."""
import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg
from gpu_util import to_dev, to_np, table_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lrn(orc):
    import oracle.learned as L
    return L


def _blob_root(blob: np.ndarray):
    hdr = blob[:32].view(np.uint32)
    L = int(hdr[1])
    V = int(blob[8:16].view(np.uint64)[0])
    a, b = blob[16:24].view(np.float32)
    return np.float32(a), np.float32(b), L, V


def _leaves(blob: np.ndarray, L: int):
    rec = np.dtype([("xmin", "<u8"), ("slope", "<f4"), ("icpt", "<f4"), ("base", "<u4"), ("width", "<u4")])
    return np.frombuffer(blob[32:32 + 24 * L].tobytes(), dtype=rec)


@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_sorted_sample_matches_oracle(hg, lrn, kt):
    keys = dg.uniform_keys_u32(300_000, 3) if kt == "u32" else dg.lognormal_mixture_u64(300_000, 3)
    s = to_np(hg.learned_sorted_sample(to_dev(keys), 3000, 77))
    assert np.array_equal(s, lrn.sorted_sample(keys, 3000, 77))


def _train(hg, keys, V, L=256, iters=60):
    model, diag = hg.learned_train(to_dev(keys), V, num_leaves=L, iters=iters)
    return to_np(model).view(np.uint8), diag


def test_knots_blob_and_gradients(hg, lrn):
    keys = dg.lognormal_mixture_u64(400_000, 5)
    V, L = 1 << 19, 256
    blob, diag = _train(hg, keys, V, L)
    a, b, Lb, Vb = _blob_root(blob)
    assert (Lb, Vb) == (L, V)
    S = diag["sample_size"]
    x = lrn.sorted_sample(keys, S, 0x4C524E)
    kb, J = lrn.knots(a, b, L, 1)
    lv = _leaves(blob, L)
    assert np.array_equal(lv["xmin"][:J + 1], kb[:J + 1])            # knots: exact
    # root gradient, double on both sides
    dx = hg.learned_sorted_sample(to_dev(keys), S, 0x4C524E)
    gl, ga, gb = hg.learned_root_grad(1, dx, L, float(a), float(b))
    ol, og = lrn.root_loss_grad(1, x, L, float(a), float(b))
    assert abs(gl - ol) <= 1e-9 * abs(ol) + 1e-12
    assert np.allclose([ga, gb], og, rtol=1e-6, atol=1e-9 * max(abs(og).max(), 1))
    # leaf gradient (fp32 on the GPU vs double in the oracle) at two points
    Y0 = lrn.leaf_init(x, V, L, kb, J)
    rng = np.random.default_rng(1)
    for Y in (Y0, Y0 + rng.normal(0, 5, Y0.shape) * ((np.arange(L + 1) >= 1) & (np.arange(L + 1) <= J))):
        loss_g, g, h = hg.learned_leaf_grad(1, dx, V, float(a), float(b), L, Y)
        loss_o, go, ho = lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, Y)
        scale = max(np.abs(go).max(), 1e-12)
        assert np.max(np.abs(g - go)) <= 1e-4 * scale + 1e-6, np.max(np.abs(g - go)) / scale
        assert np.max(np.abs(h - ho)) <= 1e-4 * max(ho.max(), 1e-12)
        assert abs(loss_g - loss_o) <= 1e-4 * loss_o + 1e-6
    # the trained knot values are the oracle's iteration (double) up to fp32
    # rounding; the projection keeps the loss above the unconstrained optimum
    Yg = diag["Y"]
    loss_0 = lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, Y0)[0]
    assert abs(diag["loss_before"] - loss_0) <= 1e-4 * loss_0
    Yo = lrn.leaf_train(1, x, V, a, b, L, kb, J, Y0, 60)
    Yo_m = np.minimum(np.maximum.accumulate(np.clip(Yo, 0, V)), V)
    err = np.abs(Yg - Yo_m)
    loss_o = lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, Yo)[0]
    loss_lsq = lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, lrn.leaf_lsq(1, x, V, a, b, L, kb, J, Y0))[0]
    print(f"\nknot error vs oracle iteration: max {err.max():.4f} mean {err.mean():.5f} buckets; "
          f"loss {diag['loss_before']:.2f} -> {diag['loss_after']:.2f} (oracle {loss_o:.2f}, "
          f"unconstrained optimum {loss_lsq:.2f})")
    assert np.max(err) < 0.05 + 1e-6 * V
    assert abs(diag["loss_after"] - loss_o) <= 1e-4 * loss_o
    assert loss_lsq <= diag["loss_after"] * (1 + 1e-4) and diag["loss_after"] < diag["loss_before"]
    # the blob is the oracle's blob of the same knots and knot values
    assert np.array_equal(blob, lrn.make_blob(a, b, 1, V, kb, J, Yg))


@pytest.mark.parametrize("kt", ["u32", "u64"])
def test_learned_build_probe_join_match_oracle(hg, orc, lrn, kt):
    if kt == "u64":
        keys = dg.lognormal_mixture_u64(1 << 20, 11)
        q = dg.queries_u64(1 << 20, keys, 0.5, 12)
        other = dg.lognormal_mixture_u64(1 << 19, 13)
    else:
        keys = dg.uniform_keys_u32(1 << 20, 11)
        q = dg.queries_u32(1 << 20, keys, 0.5, 12)
        other = dg.dup_keys_u32(1 << 19, 2, 13)
    V = 1 << 20
    model, _ = hg.learned_train(to_dev(keys), V, num_leaves=1024)
    blob = to_np(model).view(np.uint8)
    for algo in ("v2", "v1"):
        t = hg.build(to_dev(keys), V, model=model, algo=algo)
        off, ck, ci = table_np(t)
        roff, rk, ri = orc.build(keys, V, model=blob)
        assert np.array_equal(off, roff) and np.array_equal(ck, rk) and np.array_equal(ci, ri)
    assert orc.check_table(off, ck, ci, keys, V, model=blob) == []
    # explicit ids: stable partitions, and the pass whose tile leaves no room
    # to stage the model in shared memory
    ids = (np.arange(len(keys), dtype=np.uint64) * np.uint64(2654435761) % np.uint64(1 << 32)).astype(np.uint32)
    ti = hg.build(to_dev(keys), V, model=model, ids=to_dev(ids))
    got_i = table_np(ti)
    want_i = orc.build(keys, V, model=blob, ids=ids)
    assert all(np.array_equal(g, w) for g, w in zip(got_i, want_i))
    for binned in (False, True):
        got = to_np(hg.probe(t, to_dev(q), binned=binned))
        assert np.array_equal(got, orc.multiplicity(keys, q))
    tb = hg.build(to_dev(other), V, model=model)
    total, per = hg.join_count(t, tb)
    assert int(total.item()) == orc.join_size_by_keys(keys, other)
    pa, pb = hg.join_materialize(t, tb)
    offB, kB, iB = orc.build(other, V, model=blob)
    ra, rb = orc.join_materialize(off, ck, ci, offB, kB, iB, V)
    assert np.array_equal(to_np(pa), ra) and np.array_equal(to_np(pb), rb)


def test_bucket_stats_match_numpy(hg, orc):
    keys = dg.dup_keys_u32(200_000, 3, 1)
    V = 50_021
    st = hg.bucket_stats(to_dev(keys), V, seed=4)
    c = np.bincount(orc.buckets(keys, V, 4).astype(np.int64), minlength=V)
    assert st["max"] == c.max() and st["nonempty"] == (c > 0).sum()
    assert abs(st["mean"] - c.mean()) < 1e-9 and abs(st["var"] - c.var()) < 1e-6


def test_learned_gain_over_initialisation_and_murmur(hg, orc, lrn):
    # Skewed keys (lognormal mixture + uniform share, the learned workload's shape).
    keys = dg.lognormal_mixture_u64(1 << 21, 21)
    V = 1 << 21
    dk = to_dev(keys)
    model, diag = hg.learned_train(dk, V, num_leaves=1024)
    # 1. training lowers its objective from the prior (the sample's rank
    #    interpolant); the residual is the rank noise of a 1% sample
    assert diag["loss_after"] < 0.97 * diag["loss_before"]
    # 2. bucket lengths stay close to Murmur's (balls into bins) on these
    #    keys, so Murmur, the judge, keeps the learned map
    chosen, rep = hg.choose_map(dk, V, model)
    sl, sm = rep["learned"], rep["murmur"]
    print(f"\nlearned: max {sl['max']:.0f} var {sl['var']:.3f}   murmur: max {sm['max']:.0f} var {sm['var']:.3f}")
    assert rep["kept"] and chosen is model
    assert sl["var"] <= 1.15 * sm["var"] and sl["max"] <= 4 * sm["max"]
    assert sl["mean"] == sm["mean"] == len(keys) / V
    # 3. key-range order: with the learned map the table is sorted by key up to
    #    ties inside a bucket; with Murmur it is not
    t = hg.build(dk, V, model=model)
    ck = to_np(t.keys)
    off = to_np(t.offsets).astype(np.int64)
    first = ck[off[:-1][np.diff(off) > 0]]
    assert np.all(np.diff(first.astype(np.float64)) >= 0)
    tm = hg.build(dk, V)
    ckm = to_np(tm.keys)
    assert np.mean(np.diff(ckm.astype(np.float64)) >= 0) < 0.6
    # 4. the judge falls back to Murmur for a map that does not fit the keys
    #    (the same model on uniform keys over the whole range)
    other = to_dev(dg.uniform_keys_u64(len(keys), 22))
    chosen2, rep2 = hg.choose_map(other, V, model)
    assert chosen2 is None and not rep2["kept"]
