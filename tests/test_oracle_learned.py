"""Pins of the learned-map oracle (not in the paper; the model is defined in
oracle/hg_oracle_learned.cpp) against definitions and independent
computations: finite differences, explicit least squares, the knot
definition, monotonicity of the bucket map."""
import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg


@pytest.fixture(scope="module")
def lrn(orc):
    import oracle.learned as L
    return L


def _sm64(z):
    z = np.uint64(z)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def test_sample_indices_follow_splitmix64(lrn):
    # independent restatement of the documented draw
    n, S, seed = 1_000_003, 64, 12345
    with np.errstate(over="ignore"):
        st = _sm64(np.uint64(seed) ^ (np.uint64(lrn.SAMPLE_STREAM) * np.uint64(0xD1B54A32D192ED03)))
        x = [_sm64(st + np.uint64(k + 1) * np.uint64(0x9E3779B97F4A7C15)) for k in range(S)]
    want = [(int(v) >> 32) * n >> 32 for v in x]
    assert lrn.sample_indices(n, S, seed).tolist() == want
    big = lrn.sample_indices(1 << 20, 1 << 16, 3)
    assert big.max() < 1 << 20
    assert abs(big.mean() / (1 << 20) - 0.5) < 0.01


def test_sorted_sample(lrn):
    keys = dg.lognormal_mixture_u64(100_000, 4)
    s = lrn.sorted_sample(keys, 1000, 9)
    idx = lrn.sample_indices(len(keys), 1000, 9)
    assert np.array_equal(s, np.sort(keys[idx.astype(np.int64)]))


@pytest.mark.parametrize("kt,a,b,L", [(0, 3.1e-6, -3400.0, 64), (1, 2.2e-6, -2300.0, 1024), (1, 1e-7, -90.0, 16)])
def test_knots_definition(lrn, kt, a, b, L):
    kb, J = lrn.knots(np.float32(a), np.float32(b), L, kt)
    kmax = 0xFFFFFFFF if kt == 0 else (1 << 64) - 1
    assert J == lrn.root_leaf(a, b, L, kt, kmax)
    assert kb[0] == 0
    for j in range(1, J + 1):
        k = int(kb[j])
        assert lrn.root_leaf(a, b, L, kt, k) >= j
        if k > 0:
            assert lrn.root_leaf(a, b, L, kt, k - 1) < j
    assert all(int(kb[j]) == kmax for j in range(J + 1, L + 1))
    assert np.all(np.diff(kb[:J + 1].astype(np.float64)) >= 0)


def _setup(lrn, n=20_000, S=2_000, L=32, V=1 << 14, seed=5):
    keys = dg.lognormal_mixture_u64(n, seed)
    x = lrn.sorted_sample(keys, S, seed)
    a, b = lrn.root_lsq(1, x, L)
    a, b = np.float32(a), np.float32(b)
    kb, J = lrn.knots(a, b, L, 1)
    return keys, x, a, b, kb, J, L, V


def test_leaf_gradient_matches_finite_differences(lrn):
    keys, x, a, b, kb, J, L, V = _setup(lrn)
    Y = lrn.leaf_init(x, V, L, kb, J)
    rng = np.random.default_rng(0)
    Y = Y + rng.normal(0, 3.0, size=Y.shape) * (np.arange(L + 1) <= J)
    loss, g, d = lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, Y)
    for j in [1, J // 2, J]:
        h = 1e-3
        Yp, Ym = Y.copy(), Y.copy()
        Yp[j] += h
        Ym[j] -= h
        lp = lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, Yp)[0]
        lm = lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, Ym)[0]
        assert abs((lp - lm) / (2 * h) - g[j]) <= 1e-6 * max(1.0, abs(g[j]))
        assert abs((lp - 2 * loss + lm) / h ** 2 - d[j]) <= 1e-3 * max(1.0, d[j]) + 1e-4
    assert loss >= 0


def test_leaf_lsq_matches_explicit_least_squares(lrn):
    keys, x, a, b, kb, J, L, V = _setup(lrn, n=5_000, S=600, L=16, V=4096)
    Y0 = lrn.leaf_init(x, V, L, kb, J)
    Y = lrn.leaf_lsq(1, x, V, a, b, L, kb, J, Y0)
    # explicit design matrix over the free knots 1..J
    S = len(x)
    kmax = (1 << 64) - 1
    rows = np.zeros((S, L + 1))
    t = V * (2 * np.arange(S) + 1) / (2 * S)
    for i in range(S):
        j = lrn.root_leaf(a, b, L, 1, int(x[i]))
        w = float(int(kb[j + 1]) - int(kb[j])) if j < J else float(kmax - int(kb[j])) + 1.0
        lam = (int(x[i]) - int(kb[j])) / w if w > 0 else 0.0
        rows[i, j] += 1 - lam
        rows[i, j + 1] += lam
    fixed = np.zeros(L + 1)
    fixed[J + 1:] = V
    free = [j for j in range(1, J + 1) if rows[:, j].any()]
    rhs = t - rows @ fixed
    sol, *_ = np.linalg.lstsq(rows[:, free], rhs, rcond=None)
    assert np.allclose(Y[free], sol, rtol=1e-7, atol=1e-6)
    # stationarity: zero gradient on the free knots at the optimum
    _, g, _ = lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, Y)
    assert np.max(np.abs(g[free])) < 1e-6 * V


def test_root_fit_and_gradient(lrn):
    keys = dg.lognormal_mixture_u64(10_000, 2)
    x = lrn.sorted_sample(keys, 1_000, 2)
    L = 256
    a, b = lrn.root_lsq(1, x, L)
    f = np.array([np.float32(np.float32(np.uint64(v)).view(np.uint32)) for v in x], dtype=np.float64)
    t = L * (2 * np.arange(len(x)) + 1) / (2 * len(x))
    pa, pb = np.polyfit(f, t, 1)
    assert abs(a - pa) <= 1e-9 * abs(pa) + 1e-15 and abs(b - pb) <= 1e-6 * abs(pb) + 1e-9
    loss, g = lrn.root_loss_grad(1, x, L, a, b)
    assert np.all(np.abs(g) < 1e-6 * np.array([np.abs(f).max() * L, L]))
    h = 1e-9 * abs(a)
    lp = lrn.root_loss_grad(1, x, L, a + h, b)[0]
    lm = lrn.root_loss_grad(1, x, L, a - h, b)[0]
    g2 = lrn.root_loss_grad(1, x, L, a * 1.001, b)[1]
    assert g2[0] != 0
    assert abs((lp - lm) / (2 * h) - g[0]) <= 1e-3 * np.abs(f).max() * L


def test_learned_map_is_monotone_and_in_range(orc, lrn):
    keys, x, a, b, kb, J, L, V = _setup(lrn, n=50_000, S=5_000, L=64, V=1 << 16)
    Y = lrn.leaf_lsq(1, x, V, a, b, L, kb, J, lrn.leaf_init(x, V, L, kb, J))
    blob = lrn.make_blob(a, b, 1, V, kb, J, Y)
    probe = np.unique(np.concatenate([keys, np.array([0, 1, 2**63, 2**64 - 1], dtype=np.uint64),
                                      kb.astype(np.uint64)]))
    bk = orc.buckets(probe, V, model=blob)
    assert bk.max() < V
    assert np.all(np.diff(bk.astype(np.int64)) >= 0)            # order preserving
    # buckets are spread: the fit covers [0, V)
    assert bk[0] == 0 and bk[-1] >= V - 2


def test_learned_table_keeps_key_order_across_buckets(orc, lrn):
    keys, x, a, b, kb, J, L, V = _setup(lrn, n=30_000, S=3_000, L=64, V=1 << 15)
    Y = lrn.leaf_lsq(1, x, V, a, b, L, kb, J, lrn.leaf_init(x, V, L, kb, J))
    blob = lrn.make_blob(a, b, 1, V, kb, J, Y)
    off, ck, ci = orc.build(keys, V, model=blob)
    assert orc.check_table(off, ck, ci, keys, V, model=blob) == []
    # an order-preserving map makes the CSR sorted by key up to ties inside a bucket
    owner = np.repeat(np.arange(V), np.diff(off.astype(np.int64)))
    order = np.lexsort((ck, owner))
    assert np.all(np.diff(ck[order].astype(np.float64)) >= 0)
    assert np.array_equal(np.sort(ck), ck[order])
