"""Pins of the learned bucket map's inference at the edges of its leaves.

The learned map (not in the paper) sends a key to a leaf with the root
model and to a bucket with the leaf's line (model layout in include/hg.h).
Random keys rarely land on the places where an off-by-one or a wrong clamp
would show, so these tests pick them on purpose:

* hand-built models whose buckets are worked out by hand, in exact
  arithmetic, at key 0, the largest key, the first key of a leaf, the keys
  one below and one above it, the last key of a leaf, the key where the line
  reaches the leaf's width, a negative intercept, a zero-width leaf, the
  clamp below V and the round-to-nearest-even conversion of a key distance
  to float32;
* a trained model (oracle training on a lognormal mixture), checked at
  every leaf edge against a float32 restatement of the inference written
  here with exact integer rounding (not numpy's own uint64 -> float32 cast,
  which may round twice through float64).

The GPU test builds a table from the hand-built model's edge keys and checks
that every key sits in the bucket worked out by hand.
"""
import struct

import numpy as np
import pytest

from paper_1907_02900_gb300 import datagen as dg

MAGIC = 0x4D4C4748
U64MAX = (1 << 64) - 1
U32MAX = (1 << 32) - 1


def make_blob(a, b, key_type, V, leaves):
    """Model blob: header (magic, L, V, a, b, key type, flags) and one
    (xmin, slope, icpt, base, width) record per leaf."""
    buf = bytearray(32 + 24 * len(leaves))
    struct.pack_into("<IIQffII", buf, 0, MAGIC, len(leaves), V, a, b, key_type, 0)
    for j, (xmin, slope, icpt, base, width) in enumerate(leaves):
        struct.pack_into("<QffII", buf, 32 + 24 * j, xmin, slope, icpt, base, width)
    return np.frombuffer(bytes(buf), dtype=np.uint8).copy()


# --- hand-built model 1 (uint64 keys) --------------------------------------
# Root: a = 2^-23, b = -133.  The feature of a key is the bit pattern of
# float32(key) read as an integer; for 2^7 = 128 it is (127 + 7) * 2^23, so
# a * f + b = 134 - 133 = 1 (leaf 1); for 127 it is 0x42FE0000 = 1123942400,
# 1123942400 / 2^23 - 133 = 0.984375 (leaf 0).  Key 0 gives -133 (leaf 0),
# the largest key float32(2^64 - 1) = 2^64, feature 191 * 2^23, 191 - 133 =
# 58 >= L (leaf L - 1 = 1).
# Leaf 0: xmin 0,   slope 1/2, icpt 0, base 0,  width 50
# Leaf 1: xmin 131, slope 1/4, icpt 0, base 50, width 50   (V = 120)
#   keys 128..131 reach leaf 1 but lie at or below its xmin: distance 0.
M1 = dict(a=2.0 ** -23, b=-133.0, key_type=1, V=120,
          leaves=[(0, 0.5, 0.0, 0, 50), (131, 0.25, 0.0, 50, 50)])
M1_EXPECT = {
    0: 0,          # leaf 0, distance 0
    1: 0,          # 0.5 -> 0
    2: 1,          # 1.0 -> 1
    99: 49,        # 49.5 -> 49
    100: 49,       # 50.0 reaches the width: clamped to width - 1 (a clamp to width would give 50)
    127: 49,       # last key the root sends to leaf 0 (0.984375), 63.5 -> clamped
    128: 50,       # first key of leaf 1 by the root, below xmin: distance 0
    130: 50,       # xmin - 1
    131: 50,       # xmin
    132: 50,       # xmin + 1: 0.25
    134: 50,       # distance 3: 0.75 (an off-by-one "+1" would give 1.0 -> 51)
    135: 51,       # distance 4: 1.0 (an off-by-one "-1" would give 0.75 -> 50)
    330: 99,       # distance 199: 49.75 -> 49
    331: 99,       # distance 200: 50.0 = width -> width - 1 (a clamp to width gives 100)
    1 << 40: 99,
    U64MAX: 99,    # largest key: leaf L - 1, far past the width
}

# --- hand-built model 2 (uint64 keys, one leaf; a = b = 0 sends every key
# to leaf 0) --------------------------------------------------------------
# slope 1, icpt 0, xmin 1000, base 0, width 2^26, V = 2^26 + 8:
#   distance 2^24 + 1 rounds to 2^24 in float32 (round to nearest)
#   distance 2^24 + 3 is halfway between 2^24 + 2 and 2^24 + 4: ties to even -> 2^24 + 4
#   distance 2^24 + 5 is halfway between 2^24 + 4 and 2^24 + 6: ties to even -> 2^24 + 4
#   distance 2^24 + 6 is exact
M2 = dict(a=0.0, b=0.0, key_type=1, V=(1 << 26) + 8, leaves=[(1000, 1.0, 0.0, 0, 1 << 26)])
M2_EXPECT = {
    999: 0, 1000: 0, 1001: 1, 1000 + (1 << 24) - 1: (1 << 24) - 1,
    1000 + (1 << 24) + 1: 1 << 24,
    1000 + (1 << 24) + 3: (1 << 24) + 4,
    1000 + (1 << 24) + 5: (1 << 24) + 4,
    1000 + (1 << 24) + 6: (1 << 24) + 6,
    1000 + (1 << 26) - 1: (1 << 26) - 1,
    1000 + (1 << 26): (1 << 26) - 1,     # the width reached: clamped to width - 1
}

# --- hand-built model 3 (uint32 keys): negative intercept, a zero-width
# leaf, the clamp below V ---------------------------------------------------
# Root as model 1 with L = 3: key 127 -> leaf 0, 128..255 -> 1 (134 - 133 = 1,
# feature of 255 = 0x437F0000 -> 134.9921875 - 133 = 1.99), 256 -> 2 (135 - 133),
# 0xFFFFFFFF -> float32 2^32, feature 159 * 2^23 -> 26 -> leaf 2.
# Leaf 0: xmin 10,  slope 1, icpt -2.5, base 0,  width 100
# Leaf 1: xmin 128, slope 1, icpt 0,    base 7,  width 0    (every key -> base)
# Leaf 2: xmin 256, slope 1, icpt 0,    base 30, width 100  (V = 40: base + local >= V -> V - 1)
M3 = dict(a=2.0 ** -23, b=-133.0, key_type=0, V=40,
          leaves=[(10, 1.0, -2.5, 0, 100), (128, 1.0, 0.0, 7, 0), (256, 1.0, 0.0, 30, 100)])
M3_EXPECT = {
    0: 0,      # below xmin: distance 0, -2.5 -> 0
    11: 0,     # -1.5 -> 0
    13: 0,     # 0.5 -> 0
    14: 1,     # 1.5 -> 1
    127: 39,   # distance 117: 114.5 >= width -> local 99; bucket 0 + 99 >= V -> V - 1
    128: 7, 200: 7, 255: 7,    # zero-width leaf
    256: 30, 265: 39, 266: 39, # 30 + 9 = 39 = V - 1; 30 + 10 >= V -> V - 1
    U32MAX: 39,
}


def _check(orc, model, expect):
    blob = make_blob(**model)
    keys = np.array(sorted(expect), dtype=np.uint64 if model["key_type"] == 1 else np.uint32)
    got = orc.buckets(keys, model["V"], model=blob)
    want = np.array([expect[int(k)] for k in keys], dtype=np.uint64)
    bad = [(int(k), int(g), int(w)) for k, g, w in zip(keys, got, want) if g != w]
    assert not bad, f"(key, oracle bucket, hand-worked bucket): {bad}"


def test_hand_built_model_leaf_edges(orc):
    _check(orc, M1, M1_EXPECT)


def test_hand_built_model_float32_rounding_of_the_distance(orc):
    _check(orc, M2, M2_EXPECT)


def test_hand_built_model_u32_intercept_zero_width_and_clamp(orc):
    _check(orc, M3, M3_EXPECT)


# --- float32 restatement with exact rounding ---------------------------------
def f32_round(x: int) -> np.float32:
    """Nearest float32 to the non-negative integer x, ties to even, computed on
    Python integers (exact), then stored (it is representable)."""
    if x == 0:
        return np.float32(0.0)
    e = x.bit_length() - 24
    if e <= 0:
        return np.float32(x)
    q, r = divmod(x, 1 << e)
    half = 1 << (e - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return np.float32(float(q << e))


def f32_mul_add(a: np.float32, x: np.float32, b: np.float32) -> np.float32:
    """a * x + b with a float32 rounding after each operation (no fused
    multiply-add): the products and sums are formed exactly as Python
    fractions of doubles (float32 values multiply exactly in float64) and
    rounded once to float32."""
    p = np.float32(float(a) * float(x))      # exact in float64, one rounding to float32
    return np.float32(float(p) + float(b))   # float32 + float32 is exact in float64


def restated_bucket(blob: np.ndarray, key: int) -> int:
    L = int(blob[4:8].view(np.uint32)[0])
    V = int(blob[8:16].view(np.uint64)[0])
    a, b = blob[16:24].view(np.float32)
    kt = int(blob[24:28].view(np.uint32)[0])
    fk = f32_round(key & (U32MAX if kt == 0 else U64MAX))
    feat = f32_round(int(np.float32(fk).view(np.uint32)))
    r = f32_mul_add(a, feat, b)
    if not r >= 0:
        j = 0
    elif r >= np.float32(L):
        j = L - 1
    else:
        j = int(r)
    rec = blob[32 + 24 * j: 56 + 24 * j]
    xmin = int(rec[0:8].view(np.uint64)[0])
    slope, icpt = rec[8:16].view(np.float32)
    base, width = (int(v) for v in rec[16:24].view(np.uint32))
    local = 0
    if width > 0:
        d = key - xmin if key > xmin else 0
        p = f32_mul_add(slope, f32_round(d), icpt)
        if not p >= 0:
            local = 0
        elif p >= np.float32(width):
            local = width - 1
        else:
            local = min(int(p), width - 1)
    return min(base + local, V - 1)


def test_restatement_agrees_with_hand_worked_values():
    # the restatement itself is pinned by the hand-worked tables above
    for model, expect in ((M1, M1_EXPECT), (M2, M2_EXPECT), (M3, M3_EXPECT)):
        blob = make_blob(**model)
        for k, w in expect.items():
            assert restated_bucket(blob, k) == w, (k, w)


def test_float32_rounding_helper():
    # 2^60 + 2^36 + 1 lies just above the midpoint of two float32 values:
    # rounds up; via float64 first it would land on the midpoint and round to even (down)
    x = (1 << 60) + (1 << 36) + 1
    assert float(f32_round(x)) == float((1 << 60) + (1 << 37))
    assert float(f32_round((1 << 24) + 1)) == float(1 << 24)
    assert float(f32_round((1 << 24) + 3)) == float((1 << 24) + 4)
    assert float(f32_round(U64MAX)) == 2.0 ** 64


@pytest.fixture(scope="module")
def trained_blob(orc):
    import oracle.learned as lrn
    keys = dg.lognormal_mixture_u64(60_000, 31)
    V, L, S = 1 << 16, 64, 6_000
    x = lrn.sorted_sample(keys, S, 0x4C524E)
    a, b = lrn.root_lsq(1, x, L)
    kb, J = lrn.knots(np.float32(a), np.float32(b), L, 1)
    Y = lrn.leaf_lsq(1, x, V, a, b, L, kb, J, lrn.leaf_init(x, V, L, kb, J))
    return lrn.make_blob(a, b, 1, V, kb, J, Y), kb, J, V


def test_trained_model_at_every_leaf_edge(orc, trained_blob):
    """Keys 0, max, and for every reachable leaf j: xmin_j - 1, xmin_j,
    xmin_j + 1 and the last key the root sends to leaf j (xmin_{j+1} - 1)."""
    blob, kb, J, V = trained_blob
    ks = {0, 1, U64MAX, U64MAX - 1}
    for j in range(J + 1):
        x = int(kb[j])
        ks.update(k for k in (x - 1, x, x + 1) if 0 <= k <= U64MAX)
        if j < J:
            ks.add(int(kb[j + 1]) - 1)
    keys = np.array(sorted(ks), dtype=np.uint64)
    got = orc.buckets(keys, V, model=blob)
    want = np.array([restated_bucket(blob, int(k)) for k in keys], dtype=np.uint64)
    bad = [(int(k), int(g), int(w)) for k, g, w in zip(keys, got, want) if g != w]
    assert not bad, bad[:10]
    assert np.all(np.diff(got.astype(np.int64)) >= 0)   # monotone across the edges


@pytest.mark.gpu
@pytest.mark.parametrize("model,expect", [(M1, M1_EXPECT), (M2, M2_EXPECT), (M3, M3_EXPECT)])
def test_gpu_inference_at_hand_worked_edges(hg, model, expect):
    """A table built on the GPU from the edge keys with a hand-built model:
    every key lies in its hand-worked bucket (fused inference in the
    histogram, partition and bin-build kernels), for V1 and V2."""
    import torch
    from gpu_util import to_dev, to_np, table_np
    blob = make_blob(**model)
    dt = np.uint64 if model["key_type"] == 1 else np.uint32
    keys = np.array(sorted(expect), dtype=dt)
    keys = np.concatenate([keys, keys[::-1]])                # every bucket twice, in two orders
    mdl = torch.from_numpy(blob).cuda()
    V = model["V"]
    for algo in ("v2", "v1"):
        t = hg.build(to_dev(keys), V, model=mdl, algo=algo)
        off, ck, _ = table_np(t)
        owner = np.repeat(np.arange(V), np.diff(off.astype(np.int64)))
        got = {int(k): int(v) for k, v in zip(ck, owner)}
        assert got == {int(k): expect[int(k)] for k in keys}, algo
        q = to_dev(keys)
        assert np.all(to_np(hg.probe(t, q, binned=False)) == 2)
