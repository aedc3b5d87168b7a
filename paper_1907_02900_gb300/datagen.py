"""Seeded synthetic inputs shaped like the HashGraph paper's workloads.

This module only draws numbers; it holds none of the hash-table method's
arithmetic (no hash, no bucket map, no table layout).  Both the CPU oracle
tests and the CUDA path take their inputs from here, so the two sides see
identical keys and queries.

Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: output ``i`` of a stream is the SplitMix64 finaliser applied to
``state0 + (i + 1) * gamma``, where ``state0`` is derived from
``(seed, stream)``.  Everything below is integer arithmetic on ``uint64``
(wrapping), except the Zipf table and the lognormal mixture, which use
float64 on the host and are uploaded as-is.

Workload shapes (paper Section 4 and 5):
  * the sequence ``[1 .. N]`` used for the framework comparison,
  * uniform random keys, and keys drawn from ``[1 .. N/d]`` to control the
    average multiplicity ``d`` (Fig. "dup-keys"),
  * two random inputs for the inner join (Section 5, join vs CPU).
"""
from __future__ import annotations

import numpy as np

U64 = np.uint64
_GAMMA = U64(0x9E3779B97F4A7C15)
_STREAM_MUL = U64(0xD1B54A32D192ED03)
MASK32 = U64(0xFFFFFFFF)

# Stream ids (any distinct values work; fixed so that runs are reproducible).
STREAM_KEYS = 1
STREAM_QUERY_HIT = 2
STREAM_QUERY_PICK = 3
STREAM_QUERY_MISS = 4
STREAM_ZIPF = 5
STREAM_MIX_CHOICE = 6
STREAM_MIX_U1 = 7
STREAM_MIX_U2 = 8
STREAM_MIX_PARAMS = 9
STREAM_SIZES = 10


def _u64(x) -> np.ndarray:
    return np.asarray(x, dtype=np.uint64)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser (a bijection on 64-bit words)."""
    z = _u64(z)
    z = (z ^ (z >> U64(30))) * U64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> U64(27))) * U64(0x94D049BB133111EB)
    return z ^ (z >> U64(31))


def stream_state(seed: int, stream: int) -> np.uint64:
    """Initial SplitMix64 state of stream ``stream`` under ``seed``."""
    with np.errstate(over="ignore"):
        s = _u64(seed & 0xFFFFFFFFFFFFFFFF) ^ (_u64(stream) * _STREAM_MUL)
        return U64(_mix64(s))


def splitmix64(seed: int, stream: int, idx) -> np.ndarray:
    """Outputs ``idx`` (array of indices) of SplitMix64 stream ``(seed, stream)``."""
    st = stream_state(seed, stream)
    idx = _u64(idx)
    with np.errstate(over="ignore"):
        return _mix64(st + (idx + U64(1)) * _GAMMA)


def splitmix64_range(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    return splitmix64(seed, stream, np.arange(start, start + count, dtype=np.uint64))


def unit_double(x: np.ndarray) -> np.ndarray:
    """Top 53 bits of a 64-bit word as a double in [0, 1) (exact)."""
    return (_u64(x) >> U64(11)).astype(np.float64) * (2.0 ** -53)


def pick_below(x: np.ndarray, n: int) -> np.ndarray:
    """Map 64-bit words to integers in [0, n) by multiply-shift of the top 32 bits (n <= 2**32)."""
    assert 0 < n <= (1 << 32)
    return ((_u64(x) >> U64(32)) * U64(n)) >> U64(32)


# --- bijective scramblers: make structured integers look uniform while
#     keeping them distinct (own odd multipliers; each step is invertible).
def scramble32(x) -> np.ndarray:
    x = _u64(x) & MASK32
    x = x ^ (x >> U64(15))
    x = (x * U64(0x7A1F3C9B)) & MASK32
    x = x ^ (x >> U64(13))
    x = (x * U64(0x5C2E8D17)) & MASK32
    x = x ^ (x >> U64(16))
    return x.astype(np.uint32)


def scramble64(x) -> np.ndarray:
    x = _u64(x)
    with np.errstate(over="ignore"):
        x = x ^ (x >> U64(31))
        x = x * U64(0x6A09E667F3BCC909)
        x = x ^ (x >> U64(29))
        x = x * U64(0xBB67AE8584CAA73B)
        x = x ^ (x >> U64(32))
    return x


# --- workloads -------------------------------------------------------------
def sequence_keys_u32(n: int) -> np.ndarray:
    """The paper's default input: the sequence 1, 2, ..., n (Section 4)."""
    return np.arange(1, n + 1, dtype=np.uint32)


def uniform_keys_u32(n: int, seed: int, start: int = 0) -> np.ndarray:
    """Uniform random u32 keys: scramble32(u), u uniform in [0, 2**31).

    The preimage of every key lies in the lower half of the u32 domain, so
    ``miss_keys_u32`` (preimages in the upper half) can never hit.
    """
    u = splitmix64_range(seed, STREAM_KEYS, start, n) >> U64(33)
    return scramble32(u)


def miss_keys_u32(idx, seed: int) -> np.ndarray:
    u = (splitmix64(seed, STREAM_QUERY_MISS, idx) >> U64(33)) | U64(1 << 31)
    return scramble32(u)


def queries_u32(q: int, keys: np.ndarray, hit_rate: float, seed: int) -> np.ndarray:
    """Probe queries: a fraction ``hit_rate`` are copies of random build keys
    (``keys[uniform index]``), the rest are guaranteed misses."""
    idx = np.arange(q, dtype=np.uint64)
    thr = U64(int(round(hit_rate * (1 << 53))))
    hit = (splitmix64(seed, STREAM_QUERY_HIT, idx) >> U64(11)) < thr
    out = miss_keys_u32(idx, seed)
    if len(keys) > 0 and hit.any():
        pick = pick_below(splitmix64(seed, STREAM_QUERY_PICK, idx[hit]), len(keys))
        out[hit] = keys[pick.astype(np.int64)]
    return out


def dup_keys_u32(n: int, avg_mult: float, seed: int) -> np.ndarray:
    """Keys drawn uniformly from [1 .. ceil(n / avg_mult)] (Fig. "dup-keys":
    an average of ``avg_mult`` appearances per distinct key)."""
    rng = max(1, int(np.ceil(n / avg_mult)))
    x = splitmix64_range(seed, STREAM_KEYS, 0, n)
    return (pick_below(x, rng) + U64(1)).astype(np.uint32)


def uniform_keys_u64(n: int, seed: int, start: int = 0) -> np.ndarray:
    u = splitmix64_range(seed, STREAM_KEYS, start, n) >> U64(1)
    return scramble64(u)


def queries_u64(q: int, keys: np.ndarray, hit_rate: float, seed: int) -> np.ndarray:
    idx = np.arange(q, dtype=np.uint64)
    thr = U64(int(round(hit_rate * (1 << 53))))
    hit = (splitmix64(seed, STREAM_QUERY_HIT, idx) >> U64(11)) < thr
    miss_pre = (splitmix64(seed, STREAM_QUERY_MISS, idx) >> U64(1)) | U64(1 << 63)
    out = scramble64(miss_pre)
    if len(keys) > 0 and hit.any():
        pick = pick_below(splitmix64(seed, STREAM_QUERY_PICK, idx[hit]), min(len(keys), 1 << 32))
        out[hit] = keys[pick.astype(np.int64)]
    return out


def zipf_cdf(n_distinct: int, s: float = 1.0) -> np.ndarray:
    """Cumulative distribution of Zipf(s) over ranks 1..n_distinct (float64)."""
    w = np.arange(1, n_distinct + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def _zipf1_inverse(cdf: np.ndarray, u: np.ndarray) -> np.ndarray:
    """searchsorted(cdf, u, 'right') for the Zipf(1) CDF, found from a
    closed-form first guess: H_m is close to ln(m + 1/2) + 0.5772, so the
    smallest m with H_m > u * H_n is about exp(u * H_n - 0.5772) - 1/2 and the
    index (m - 1) about floor(exp(u * H_n - 0.5772) - 0.5).  A guess k is kept
    where it is the exact index (cdf[k-1] <= u < cdf[k]); the few others (a
    fraction of a percent) take the binary search."""
    nd = len(cdf)
    h_n = np.log(nd + 0.5) + 0.5772156649015329
    k = np.clip(np.floor(np.exp(u * h_n - 0.5772156649015329) - 0.5), 0, nd - 1).astype(np.int64)
    bad = cdf[k] <= u
    bad |= (k > 0) & (cdf[np.maximum(k - 1, 0)] > u)
    if bad.any():
        k[bad] = np.searchsorted(cdf, u[bad], side="right")
    return k


def zipf_ranks(n: int, n_distinct: int, seed: int, s: float = 1.0, start: int = 0,
               cdf: np.ndarray | None = None) -> np.ndarray:
    """Ranks in [1, n_distinct] drawn by inverse CDF: the rank of u is
    searchsorted(cdf, u, side='right') + 1 (s = 1 uses an exact shortcut)."""
    if cdf is None:
        cdf = zipf_cdf(n_distinct, s)
    u = unit_double(splitmix64_range(seed, STREAM_ZIPF, start, n))
    r = _zipf1_inverse(cdf, u) if s == 1.0 else np.searchsorted(cdf, u, side="right")
    return np.minimum(r, n_distinct - 1).astype(np.uint64) + U64(1)


def zipf_keys_u64(n: int, n_distinct: int, seed: int, s: float = 1.0) -> np.ndarray:
    """u64 keys scramble64(rank), rank ~ Zipf(s) over 1..n_distinct."""
    return scramble64(zipf_ranks(n, n_distinct, seed, s))


def uniform_domain_keys_u64(n: int, n_distinct: int, seed: int) -> np.ndarray:
    """u64 keys scramble64(rank), rank uniform over 1..n_distinct."""
    r = pick_below(splitmix64_range(seed, STREAM_KEYS, 0, n), n_distinct) + U64(1)
    return scramble64(r)


def lognormal_mixture_params(seed: int, clusters: int = 64):
    x = splitmix64_range(seed, STREAM_MIX_PARAMS, 0, 2 * clusters)
    u = unit_double(x)
    mu = 20.0 + 16.0 * u[:clusters]          # ln-space centres in [20, 36)
    sigma = 0.5 + 1.5 * u[clusters:]         # ln-space widths in [0.5, 2.0)
    return mu, sigma


def lognormal_mixture_u64(n: int, seed: int, clusters: int = 64,
                          uniform_frac: float = 0.10) -> np.ndarray:
    """Skewed u64 keys: equal-weight mixture of ``clusters`` lognormals plus a
    ``uniform_frac`` share of uniform u64 words.  float64 on the host
    (Box-Muller normal draws); generated once and uploaded to the device."""
    mu, sigma = lognormal_mixture_params(seed, clusters)
    idx = np.arange(n, dtype=np.uint64)
    choice = splitmix64(seed, STREAM_MIX_CHOICE, idx)
    thr = U64(int(round(uniform_frac * (1 << 53))))
    is_uni = (choice >> U64(11)) < thr
    c = pick_below(scramble64(choice), clusters).astype(np.int64)
    u1 = 1.0 - unit_double(splitmix64(seed, STREAM_MIX_U1, idx))   # (0, 1]
    u2 = unit_double(splitmix64(seed, STREAM_MIX_U2, idx))
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    v = np.floor(np.exp(mu[c] + sigma[c] * z))
    out = np.empty(n, dtype=np.uint64)
    big = v >= 2.0 ** 64
    hi = (v >= 2.0 ** 63) & ~big
    lo = ~(big | hi)
    out[lo] = v[lo].astype(np.uint64)
    out[hi] = (v[hi] - 2.0 ** 63).astype(np.uint64) | U64(1 << 63)
    out[big] = U64(0xFFFFFFFFFFFFFFFF)
    out[is_uni] = splitmix64(seed, STREAM_KEYS, idx[is_uni])
    return out


def batched_table_sizes(t: int, seed: int, lo_log2: float = 10.0, hi_log2: float = 22.0) -> np.ndarray:
    """Table sizes floor(2**(lo + (hi-lo) u)), u uniform: log-uniform 1K..4M."""
    u = unit_double(splitmix64_range(seed, STREAM_SIZES, 0, t))
    return np.floor(np.exp2(lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)


def batched_sizes(t: int, seed: int, total: int | None = None, lo_log2: float = 10.0,
                  hi_log2: float = 22.0) -> np.ndarray:
    """Sizes of t tables, log-uniform over [2**lo, 2**hi); with ``total`` they
    are scaled by total / sum and floored (each at least 1), so the batch holds
    at most ``total`` keys and keeps the log-uniform shape."""
    n = batched_table_sizes(t, seed, lo_log2, hi_log2)
    if total is not None:
        n = np.maximum(1, np.floor(n * (total / float(n.sum())))).astype(np.int64)
        excess = int(n.sum()) - total          # only from the floor of 1, a few keys at most
        if excess > 0:
            n[int(np.argmax(n))] -= excess
    return n


def batched_keys_u32(sizes: np.ndarray, seed: int) -> np.ndarray:
    """Keys of all tables back to back: one uniform u32 stream, table t owns
    the slice [sum(sizes[:t]), sum(sizes[:t+1]))."""
    return uniform_keys_u32(int(np.sum(sizes)), seed)


def batched_queries_u32(qsizes: np.ndarray, keys: np.ndarray, sizes: np.ndarray, hit_rate: float,
                        seed: int) -> np.ndarray:
    """Queries of all tables back to back.  Query j belongs to table t(j); a
    fraction ``hit_rate`` are copies of a uniformly chosen key of that table
    (none if it is empty), the rest are guaranteed misses."""
    qsizes = np.asarray(qsizes, dtype=np.int64)
    sizes = np.asarray(sizes, dtype=np.int64)
    qtot = int(qsizes.sum())
    kbeg = np.concatenate([[0], np.cumsum(sizes)])
    qbeg = np.concatenate([[0], np.cumsum(qsizes)])
    idx = np.arange(qtot, dtype=np.uint64)
    t = np.searchsorted(qbeg, np.arange(qtot, dtype=np.int64), side="right") - 1
    nt = sizes[t].astype(np.uint64)
    thr = U64(int(round(hit_rate * (1 << 53))))
    hit = ((splitmix64(seed, STREAM_QUERY_HIT, idx) >> U64(11)) < thr) & (nt > 0)
    out = miss_keys_u32(idx, seed)
    if hit.any():
        x = splitmix64(seed, STREAM_QUERY_PICK, idx[hit])
        with np.errstate(over="ignore"):
            pick = ((x >> U64(32)) * nt[hit]) >> U64(32)
        out[hit] = keys[(kbeg[t[hit]] + pick.astype(np.int64))]
    return out


def batched_table_queries_u32(q: int, start: int, table_keys: np.ndarray, hit_rate: float,
                              seed: int) -> np.ndarray:
    """The queries of one table of a batch: outputs start .. start+q-1 of the
    batched query recipe (start = the table's first query in the unpadded
    concatenation), hits drawn from ``table_keys``."""
    idx = np.arange(start, start + q, dtype=np.uint64)
    n = len(table_keys)
    thr = U64(int(round(hit_rate * (1 << 53))))
    hit = ((splitmix64(seed, STREAM_QUERY_HIT, idx) >> U64(11)) < thr) & (n > 0)
    out = miss_keys_u32(idx, seed)
    if hit.any():
        pick = pick_below(splitmix64(seed, STREAM_QUERY_PICK, idx[hit]), n)
        out[hit] = table_keys[pick.astype(np.int64)]
    return out


# Seeds of the five measured workloads.
SEED_PLAIN = 0x48470001
SEED_SCALE = 0x48470002
SEED_JOIN = 0x48470003
SEED_BATCH = 0x48470004
SEED_LEARNED = 0x48470005
