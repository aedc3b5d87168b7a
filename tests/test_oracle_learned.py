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


@pytest.mark.parametrize("n,S,L", [(5_000, 600, 16), (40_000, 400, 256)])
def test_leaf_lsq_matches_explicit_least_squares(lrn, n, S, L):
    keys, x, a, b, kb, J, L, V = _setup(lrn, n=n, S=S, L=L, V=4096)
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
    free = list(range(1, J + 1))
    rhs = t - rows @ fixed
    # ridge rows sqrt(rho) * (Y_j - Y0_j) for the free knots
    rho = lrn.RIDGE
    R = np.sqrt(rho) * np.eye(len(free))
    sol, *_ = np.linalg.lstsq(np.vstack([rows[:, free], R]), np.concatenate([rhs, np.sqrt(rho) * Y0[free]]), rcond=None)
    assert np.allclose(Y[free], sol, rtol=1e-7, atol=1e-6)
    # stationarity: zero gradient on the free knots at the optimum
    _, g, _ = lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, Y)
    assert np.max(np.abs(g[free])) < 1e-6 * V


def test_leaf_train_steps_and_converges(lrn):
    # sparse: about two samples per leaf, so some knot runs converge slowly
    keys, x, a, b, kb, J, L, V = _setup(lrn, n=40_000, S=500, L=256, V=1 << 14)
    Y0 = lrn.leaf_init(x, V, L, kb, J)
    # one round without projection is the preconditioned gradient step on the free knots only
    _, g, d = lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, Y0)
    step = Y0.copy()
    step[1:J + 1] -= 0.9 * g[1:J + 1] / d[1:J + 1]
    assert np.allclose(lrn.leaf_train(1, x, V, a, b, L, kb, J, Y0, 1, gamma=0.0), step, rtol=0, atol=1e-9 * V)
    # with projection: the same step, then the projection
    want = lrn.leaf_project(V, L, J, Y0, step)
    assert np.allclose(lrn.leaf_train(1, x, V, a, b, L, kb, J, Y0, 1), want, rtol=0, atol=1e-9 * V)
    # unprojected, the iteration is a contraction toward the closed-form optimum
    Yl = lrn.leaf_lsq(1, x, V, a, b, L, kb, J, Y0)
    e = [np.abs(lrn.leaf_train(1, x, V, a, b, L, kb, J, Y0, it, gamma=0.0) - Yl).max() for it in (3, 30, 3000)]
    assert e[0] > e[1] > e[2] and e[2] < 1e-6 * V
    # projected, it lowers the loss from the prior but cannot beat the unconstrained optimum
    Yt = lrn.leaf_train(1, x, V, a, b, L, kb, J, Y0, 40)
    l0, l1, ll = (lrn.leaf_loss_grad(1, x, V, a, b, L, kb, J, Y)[0] for Y in (Y0, Yt, Yl))
    assert ll <= l1 < l0
    Yfull = np.append(Yt[:J + 1], V)
    P0 = np.append(Y0[:J + 1], V)
    assert np.all(np.diff(Yfull) >= 0.5 * np.diff(P0) - 1e-9 * V)


def test_leaf_init_interpolates_the_rank_targets(lrn):
    rng = np.random.default_rng(3)
    x = np.sort(rng.choice(1 << 40, size=200, replace=False).astype(np.uint64))
    S, V = len(x), 1 << 16
    t = V * (2 * np.arange(S) + 1) / (2 * S)
    # knots at sample points hit their targets; midpoints of neighbours give the mean
    kb = np.concatenate([[0], x[::7], (x[10:60:5] // 2 + x[11:61:5] // 2)]).astype(np.uint64)
    kb = np.sort(kb)
    J = len(kb) - 1
    Y = lrn.leaf_init(x, V, J, kb, J)
    assert Y[0] == 0
    for j in range(1, J + 1):
        k = int(kb[j])
        i = int(np.searchsorted(x, kb[j]))
        if i < S and int(x[i]) == k:
            assert abs(Y[j] - t[i]) <= 1e-9 * V
        else:
            lam = (k - int(x[i - 1])) / (int(x[i]) - int(x[i - 1]))
            assert abs(Y[j] - ((1 - lam) * t[i - 1] + lam * t[i])) <= 1e-9 * V
    assert np.all(np.diff(Y) > 0)
    # the ends: below the first sample toward (0, 0), above the last toward (key max + 1, V)
    kb2 = np.array([0, int(x[0]) // 2, int(x[-1]) + ((1 << 64) - 1 - int(x[-1])) // 2], dtype=np.uint64)
    Y2 = lrn.leaf_init(x, V, 2, kb2, 2)
    assert abs(Y2[1] - t[0] * (int(x[0]) // 2) / int(x[0])) <= 1e-9 * V
    assert abs(Y2[2] - (t[-1] + (V - t[-1]) * 0.5)) <= 1e-6 * V
    # knots above J sit at V
    Y3 = lrn.leaf_init(x, V, 5, kb[:6], 3)
    assert np.all(Y3[4:] == V)


def test_leaf_project_is_the_least_feasible_majorant(lrn):
    rng = np.random.default_rng(4)
    V, L, gam = 1000, 12, 0.5
    for trial in range(50):
        J = int(rng.integers(1, L + 1))
        Y0 = np.concatenate([[0.0], np.sort(rng.uniform(0, V, L))])
        Y0[J + 1:] = V
        Y = Y0 + rng.normal(0, 60, L + 1)
        Y[0] = 0
        P = lrn.leaf_project(V, L, J, Y0, Y, gam)
        Z, Zp = Y - gam * Y0, P - gam * Y0
        Zp0, Zj = Zp[:J + 1], Z[:J + 1]
        # feasible: Z' non-decreasing from 0 and capped so that the last leaf keeps its floor
        assert np.all(np.diff(np.concatenate([[0.0], Zp0[1:]])) >= -1e-12)
        assert np.all(Zp0[1:] <= (1 - gam) * V + 1e-9)
        # every value is attained: either the cap or an earlier Z (or 0)
        for j in range(1, J + 1):
            cands = np.concatenate([[0.0], Zj[1:j + 1], [(1 - gam) * V]])
            assert np.min(np.abs(cands - Zp0[j])) <= 1e-9
            assert Zp0[j] >= min(Zj[j], (1 - gam) * V) - 1e-12
        # knots above J untouched; feasible inputs unchanged (idempotent)
        assert np.array_equal(P[J + 1:], Y[J + 1:])
        assert np.allclose(lrn.leaf_project(V, L, J, Y0, P, gam), P, rtol=0, atol=1e-9)


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
