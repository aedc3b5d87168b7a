// HashGraph-Probe-New (Alg. 3): intersect the adjacency arrays of two tables
// bucket by bucket.  Both tables are built with the same V and bucket map,
// so equal keys always meet in the same bucket index.
//
// Both CSRs hold their edges in bucket order, so the kernels walk them side
// by side in tiles of A's edges (bucket-major, merge-style) and take every
// edge's bucket from A's offsets instead of evaluating the bucket map:
//   k_join_merge   per edge a of table A: m(a) = number of edges of B's bucket
//                  with key(a); per bucket: sum of m; join total
//   scan of m      -> output position of every A edge (canonical pair order:
//                  bucket, A's CSR position, B's CSR position)
//   k_join_write   every A edge writes its matching (A id, B id) pairs
#include "hg_build.cuh"
#include "hg_trace.h"
#include "hg_scan.cuh"

namespace hg {

// Which tables a workspace's per-edge match counts belong to: written by the
// count, checked by the materialisation that reuses them.
struct JoinStamp {
  uint64_t w[8];
};
constexpr uint64_t kJoinStampMagic = 0x544E434E494F4A48ull;  // "HJOINCNT"

static JoinStamp join_stamp(const hg_table* A, const hg_table* B, uint64_t V) {
  JoinStamp s{};
  s.w[0] = kJoinStampMagic;
  s.w[1] = A->n;
  s.w[2] = B->n;
  s.w[3] = V;
  s.w[4] = (uint64_t)(uintptr_t)A->d_offsets;
  s.w[5] = (uint64_t)(uintptr_t)A->d_keys;
  s.w[6] = (uint64_t)(uintptr_t)B->d_offsets;
  s.w[7] = (uint64_t)(uintptr_t)B->d_keys;
  return s;
}

constexpr int kJoinThreads = 256;
// A tile is kJoinTile consecutive items of the merged sequence "bucket v,
// then its A edges" (bucket v at item offA[v] + v, A edge j of bucket v at
// item j + v + 1): at most kJoinTile A edges and kJoinTile + 1 buckets, so
// its slices of both offset arrays always fit shared memory, however sparse
// or skewed the table.
constexpr uint32_t kJoinTile = 2048;
constexpr uint32_t kJoinPer = kJoinTile / kJoinThreads;
constexpr uint32_t kJoinOffCap = kJoinTile + 2;  // offsets staged per table
constexpr uint32_t kJoinKeyBytes = kJoinTile * 8;  // B keys staged (then the tile's prefix sums)

// Element copies global -> shared that bypass registers (cp.async): a
// thread's copies are all in flight at once; join_copies_wait() completes
// the thread's own copies (a barrier then publishes them to the block).
template <int B>
__device__ __forceinline__ void join_copy(void* dst, const void* src) {
  static_assert(B == 4 || B == 8, "element copy of 4 or 8 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "n"(B)
               : "memory");
}
__device__ __forceinline__ void join_copies_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Merge-path split of every tile boundary w = t * kJoinTile: the bucket v
// holding item w (the last v with offA[v] + v <= w) and the first A edge at
// or after item w.  tv[tiles] closes the last tile.
__global__ void k_join_tiles(const uint32_t* __restrict__ offA, uint64_t V, uint64_t nA, uint64_t tiles,
                             uint2* __restrict__ tv) {
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= tiles;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t w = t * kJoinTile;
    uint64_t v, j;
    if (w >= nA + V) {
      v = V - 1;
      j = nA;
    } else {
      uint64_t lo = 0, hi = V;  // item(lo) <= w < item(hi), item(V) = nA + V
      while (hi - lo > 1) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if ((uint64_t)__ldg(offA + mid) + mid <= w) lo = mid;
        else hi = mid;
      }
      v = lo;
      const uint64_t o = __ldg(offA + v);
      j = w - v > o ? w - v - 1 : o;
    }
    tv[t] = make_uint2((uint32_t)v, (uint32_t)j);
  }
}

// One tile of the two tables: A edges [j0, j1) in buckets v0 .. v1, and the
// offsets of those buckets (and of v1 + 1) staged from both tables.  Ends
// with a barrier.
struct JoinTile {
  uint32_t v0, nv;  // buckets v0 .. v0 + nv - 1
  uint32_t j0, ne;  // A edges j0 .. j0 + ne - 1
};

__device__ __forceinline__ JoinTile join_stage(const uint2* __restrict__ tv, uint64_t t,
                                               const uint32_t* __restrict__ offA,
                                               const uint32_t* __restrict__ offB, uint32_t* oa, uint32_t* ob) {
  const uint2 c = tv[t], d = tv[t + 1];
  JoinTile T;
  T.v0 = c.x;
  T.nv = d.x - c.x + 1;  // <= kJoinTile + 1
  T.j0 = c.y;
  T.ne = d.y - c.y;      // <= kJoinTile
  for (uint32_t k = threadIdx.x; k <= T.nv; k += blockDim.x) {
    join_copy<4>(oa + k, offA + T.v0 + k);
    join_copy<4>(ob + k, offB + T.v0 + k);
  }
  join_copies_wait();
  __syncthreads();
  return T;
}

// Local bucket of A edge j of the tile: the last b < nv with oa[b] <= j
// (oa[0] <= j < oa[nv] holds for every edge of the tile).
__device__ __forceinline__ uint32_t join_local_bucket(const uint32_t* oa, uint32_t nv, uint32_t j) {
  uint32_t lo = 0, hi = nv;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (oa[mid] <= j) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Matches of key among B's edges [s, e) (read from global memory).
template <typename K>
__device__ __forceinline__ uint32_t bucket_matches(const K* __restrict__ keysB, uint32_t s, uint32_t e, K key) {
  uint32_t m = 0, k = s;
  for (; k + 4 <= e; k += 4) {
    const K b0 = __ldg(keysB + k), b1 = __ldg(keysB + k + 1), b2 = __ldg(keysB + k + 2), b3 = __ldg(keysB + k + 3);
    m += (b0 == key) + (b1 == key) + (b2 == key) + (b3 == key);
  }
  for (; k < e; ++k) m += __ldg(keysB + k) == key;
  return m;
}

// Count (merge-style, bucket-major): both tables hold their edges in bucket
// order, so a tile of A's edges meets one contiguous run of B's edges; the
// kernel streams the two CSR arrays side by side, stages the run of B's keys
// when it fits, and never evaluates the bucket map.  Per A edge: m = matches
// in B's bucket (kept for the materialisation); per bucket: the sum of m,
// stored by the tile holding all of the bucket's A edges or added by every
// tile holding some (the array is zeroed first); per tile: its sum added to
// the join total.  bucket_counts null: per-edge counts only.
template <typename K>
__global__ void __launch_bounds__(kJoinThreads) k_join_merge(const uint32_t* __restrict__ offA,
                                                             const K* __restrict__ keysA,
                                                             const uint32_t* __restrict__ offB,
                                                             const K* __restrict__ keysB,
                                                             const uint2* __restrict__ tv, uint64_t tiles,
                                                             uint64_t* __restrict__ m_out,
                                                             unsigned long long* __restrict__ bucket_counts,
                                                             unsigned long long* __restrict__ total,
                                                             JoinStamp stamp, uint64_t* __restrict__ stamp_out) {
  __shared__ uint32_t oa[kJoinOffCap], ob[kJoinOffCap];
  __shared__ __align__(16) uint8_t region[kJoinKeyBytes];  // B keys, then the prefix sums
  __shared__ uint16_t bkt[kJoinTile];
  __shared__ uint32_t msm[kJoinTile];
  __shared__ unsigned long long wsum64[32];
  if (stamp_out && blockIdx.x == 0 && threadIdx.x < 8) stamp_out[threadIdx.x] = stamp.w[threadIdx.x];
  K* const kbs = (K*)region;
  unsigned long long* const psum = (unsigned long long*)region;
  constexpr uint32_t cap_b = kJoinKeyBytes / sizeof(K);
  unsigned long long acc = 0;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const JoinTile T = join_stage(tv, t, offA, offB, oa, ob);
    const uint32_t bb0 = ob[0], nbt = ob[T.nv] - bb0;
    const bool staged = nbt <= cap_b;
    // the tile's A keys (registers) and, when it fits, B's run of keys
    // (copied to shared memory): all loads in flight before the first use
    K ka[kJoinPer];
#pragma unroll
    for (int r = 0; r < (int)kJoinPer; ++r) {
      const uint32_t i = threadIdx.x + r * kJoinThreads;
      ka[r] = i < T.ne ? __ldcs(keysA + T.j0 + i) : K(0);
    }
    if (staged) {
      for (uint32_t k = threadIdx.x; k < nbt; k += blockDim.x) join_copy<sizeof(K)>(kbs + k, keysB + bb0 + k);
      join_copies_wait();
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < (int)kJoinPer; ++r) {
      const uint32_t i = threadIdx.x + r * kJoinThreads;
      if (i >= T.ne) break;
      const uint32_t j = T.j0 + i;
      const K key = ka[r];
      const uint32_t b = join_local_bucket(oa, T.nv, j);
      const uint32_t s = ob[b], e = ob[b + 1];
      uint32_t m = 0;
      if (staged)
        for (uint32_t k = s - bb0; k < e - bb0; ++k) m += kbs[k] == key;
      else
        m = bucket_matches(keysB, s, e, key);
      __stcs(m_out + j, (uint64_t)m);
      msm[i] = m;
      bkt[i] = (uint16_t)b;
    }
    __syncthreads();
    if (!bucket_counts) continue;  // materialisation without a count
    // inclusive prefix sums of m over the tile, kJoinPer entries per thread
    const uint32_t c0 = threadIdx.x * kJoinPer;
    unsigned long long loc = 0;
#pragma unroll
    for (uint32_t k = 0; k < kJoinPer; ++k) loc += c0 + k < T.ne ? msm[c0 + k] : 0u;
    unsigned long long tile_sum;
    unsigned long long run = block_excl_scan<unsigned long long>(loc, wsum64, &tile_sum);
#pragma unroll
    for (uint32_t k = 0; k < kJoinPer; ++k) {
      run += c0 + k < T.ne ? msm[c0 + k] : 0u;
      psum[c0 + k] = run;
    }
    __syncthreads();
    // one thread per bucket segment of the tile (at its last edge)
    for (uint32_t i = threadIdx.x; i < T.ne; i += blockDim.x) {
      const uint32_t b = bkt[i];
      if (i + 1 < T.ne && bkt[i + 1] == b) continue;
      const uint32_t bs = oa[b], be = oa[b + 1];
      const uint32_t first = bs > T.j0 ? min(i, bs - T.j0) : 0u;
      const unsigned long long c = psum[i] - (first ? psum[first - 1] : 0ull);
      if (bs >= T.j0 && be <= T.j0 + T.ne) bucket_counts[T.v0 + b] = c;
      else if (c) atomicAdd(bucket_counts + T.v0 + b, c);
    }
    if (threadIdx.x == 0) acc += tile_sum;
    __syncthreads();
  }
  if (total && threadIdx.x == 0 && acc) atomicAdd(total, acc);
}

// Pairs of a warp's 32 consecutive A edges occupy one contiguous output
// range; it is written in windows of kJoinWin pairs: every lane stages the
// pairs of its edge that fall in the window in shared memory, then the warp
// writes the window out coalesced.
constexpr uint32_t kJoinWin = 256;

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const uint64_t y = __shfl_xor_sync(kFull, x, d);
    x = y < x ? y : x;
  }
  return x;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t x) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const uint64_t y = __shfl_xor_sync(kFull, x, d);
    x = y > x ? y : x;
  }
  return x;
}

template <typename K>
__global__ void __launch_bounds__(kJoinThreads) k_join_write(const uint32_t* __restrict__ offA,
                                                             const K* __restrict__ keysA,
                                                             const uint32_t* __restrict__ idsA,
                                                             const uint32_t* __restrict__ offB,
                                                             const K* __restrict__ keysB,
                                                             const uint32_t* __restrict__ idsB,
                                                             const uint2* __restrict__ tv, uint64_t tiles,
                                                             const uint64_t* __restrict__ moff,
                                                             int64_t* __restrict__ outA,
                                                             int64_t* __restrict__ outB, uint64_t cap,
                                                             const uint32_t* __restrict__ abort) {
  // ids are 32-bit: staged as such, widened to int64 on the way out
  __shared__ uint32_t stage_a[kJoinThreads / 32][kJoinWin];
  __shared__ uint32_t stage_b[kJoinThreads / 32][kJoinWin];
  __shared__ uint32_t oa[kJoinOffCap], ob[kJoinOffCap];
  if (*(volatile const uint32_t*)abort) return;
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t* sa = stage_a[w];
  uint32_t* sb = stage_b[w];
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const JoinTile T = join_stage(tv, t, offA, offB, oa, ob);
    // The warp's groups of 32 consecutive A edges; each lane's output range,
    // key and id of the next group are loaded while the current one is written.
    uint32_t g = w * 32;
    uint64_t n_o = ~0ull, n_oe = 0;
    K n_key = K(0);
    uint32_t n_ida = 0;
    auto fetch = [&](uint32_t gg) {
      const uint32_t i = gg + lane;
      const uint64_t j = (uint64_t)T.j0 + i;
      const bool valid = gg < T.ne && i < T.ne;
      n_o = valid ? moff[j] : ~0ull;
      n_oe = valid ? moff[j + 1] : 0ull;
      n_key = valid ? keysA[j] : K(0);
      n_ida = valid ? idsA[j] : 0u;
    };
    fetch(g);
    for (; g < T.ne; g += nw * 32) {
      const uint32_t i = g + lane;
      const uint64_t j = (uint64_t)T.j0 + i;
      uint64_t o = n_o, oe = n_oe;
      const K key = n_key;
      const uint32_t ida = n_ida;
      fetch(g + nw * 32);
      if (oe > cap) oe = cap;
      uint32_t k = 0, e = 0;
      if (i < T.ne && o < oe) {
        const uint32_t b = join_local_bucket(oa, T.nv, (uint32_t)j);
        k = ob[b];
        e = ob[b + 1];
      }
      const uint64_t lo = warp_min_u64(o), hi = warp_max_u64(oe);
      for (uint64_t w0 = lo; w0 < hi; w0 += kJoinWin) {
        const uint64_t w1 = w0 + kJoinWin < hi ? w0 + kJoinWin : hi;
        while (o < oe && o < w1) {
          while (k < e && __ldg(keysB + k) != key) ++k;
          if (k >= e) {  // unreachable for the tables the counts came from; keeps k inside the bucket
            oe = o;
            break;
          }
          sa[o - w0] = ida;
          sb[o - w0] = __ldg(idsB + k);
          ++o;
          ++k;
        }
        __syncwarp();
        for (uint64_t x = w0 + lane; x < w1; x += 32) {
          outA[x] = (int64_t)sa[x - w0];
          outB[x] = (int64_t)sb[x - w0];
        }
        __syncwarp();
      }
    }
    __syncthreads();  // the staged offsets are rewritten by the next tile
  }
}

__global__ void k_join_finish(const uint64_t* __restrict__ moff, uint64_t nA, uint64_t cap,
                              int64_t* __restrict__ d_total, uint32_t* status, const uint32_t* abort,
                              uint64_t* stamp) {
  stamp[0] = 0;  // the per-edge counts are now output positions: no later call may reuse them
  if (*abort) {
    *d_total = 0;
    return;
  }
  const uint64_t t = moff[nA];
  *d_total = (int64_t)t;
  if (t > cap) set_status(status, HG_ERR_OVERFLOW);
}

// The materialisation after a count: the workspace must hold the per-edge
// match counts of exactly these tables (stamp).  On a mismatch nothing is
// written and the status reads HG_ERR_INVALID_ARG.
__global__ void k_join_check(JoinStamp want, const uint64_t* __restrict__ stamp, uint32_t* abort,
                             uint32_t* status, uint64_t* __restrict__ moff, uint64_t nA) {
  bool ok = true;
  for (int i = 0; i < 8; ++i) ok &= stamp[i] == want.w[i];
  *abort = ok ? 0u : 1u;
  if (ok) moff[nA] = 0;  // closing element of the exclusive scan over nA + 1 entries
  else set_status(status, HG_ERR_INVALID_ARG);
}

struct JoinWs {
  uint64_t* moff;
  uint64_t* part;
  unsigned long long* bucket_counts;
  uint2* tv;       // tile splits (tiles + 1)
  uint64_t tiles;
  size_t total;
};

static JoinWs join_layout(uint8_t* ws, uint64_t nA, uint64_t V) {
  JoinWs w{};
  size_t o = sizeof(WsHeader);
  w.tiles = (nA + V + kJoinTile - 1) / kJoinTile;
  w.moff = (uint64_t*)(ws + o);                  o = align_up(o + (nA + 1) * 8);
  w.part = (uint64_t*)(ws + o);                  o = align_up(o + scan_workspace_bytes<uint64_t>(nA + 1));
  w.bucket_counts = (unsigned long long*)(ws + o); o = align_up(o + V * 8);
  w.tv = (uint2*)(ws + o);                        o = align_up(o + (w.tiles + 1) * 8);
  w.total = o;
  return w;
}

size_t join_workspace_bytes(uint64_t nA, uint64_t V) { return join_layout(nullptr, nA, V).total; }

// Grid of a bucket-major kernel: one wave of resident CTAs (a second,
// partial wave would leave most SMs idle while it runs), at most one per tile.
template <typename F>
static unsigned join_grid(F* kern, uint64_t tiles) {
  static int per_sm = 0;  // per kernel instantiation
  if (per_sm == 0) {
    int x = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&x, kern, kJoinThreads, 0) != cudaSuccess || x <= 0) x = 1;
    per_sm = x;
  }
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)dev_info().sms * per_sm));
}

static hg_status join_tiles(const hg_table* A, uint64_t V, const JoinWs& w, cudaStream_t st) {
  HG_TRACE("k_join_tiles", st);
  const uint64_t g = std::min<uint64_t>((w.tiles + 1 + 255) / 256, (uint64_t)dev_info().sms * 8);
  k_join_tiles<<<(unsigned)g, 256, 0, st>>>(A->d_offsets, V, A->n, w.tiles, w.tv);
  return last_launch_status();
}

// The bucket map is not evaluated: the tables' CSR order gives every edge's
// bucket.  (Map stays in the signature: the tables must come from it.)
template <typename K, typename Map>
hg_status join_count_impl(const hg_config* cfg, const hg_table* A, const hg_table* B, int64_t* d_total,
                          int64_t* d_bucket_counts, uint8_t* ws, cudaStream_t st, Map) {
  const uint64_t V = cfg->num_buckets, nA = A->n;
  JoinWs w = join_layout(ws, nA, V);
  unsigned long long* bc = d_bucket_counts ? (unsigned long long*)d_bucket_counts : w.bucket_counts;
  if (cudaMemsetAsync(bc, 0, V * 8, st) != cudaSuccess) return HG_ERR_CUDA;
  if (cudaMemsetAsync(d_total, 0, 8, st) != cudaSuccess) return HG_ERR_CUDA;
  hg_status rc = join_tiles(A, V, w, st);
  if (rc != HG_OK) return rc;
  {
    HG_TRACE("k_join_merge", st);
    k_join_merge<K><<<join_grid(k_join_merge<K>, w.tiles), kJoinThreads, 0, st>>>(
        A->d_offsets, (const K*)A->d_keys, B->d_offsets, (const K*)B->d_keys, w.tv, w.tiles, w.moff, bc,
        (unsigned long long*)d_total, join_stamp(A, B, V), ((WsHeader*)ws)->join_stamp);
  }
  return last_launch_status();
}

// after_count: the per-edge match counts come from the hg_join_count call
// that last used this workspace on the same tables (checked on the device)
// instead of a second intersection pass.
template <typename K, typename Map>
hg_status join_materialize_impl(const hg_config* cfg, const hg_table* A, const hg_table* B, int64_t* outA,
                                int64_t* outB, uint64_t cap, int64_t* d_total, uint8_t* ws, cudaStream_t st,
                                Map, bool after_count) {
  const uint64_t V = cfg->num_buckets, nA = A->n;
  JoinWs w = join_layout(ws, nA, V);
  WsHeader* hdr = (WsHeader*)ws;
  if (after_count) {
    HG_TRACE("k_join_check", st);
    k_join_check<<<1, 1, 0, st>>>(join_stamp(A, B, V), hdr->join_stamp, &hdr->join_abort, &hdr->status, w.moff, nA);
  } else {
    // every per-edge count is written below; the scan's closing element is zeroed here
    if (cudaMemsetAsync(w.moff + nA, 0, 8, st) != cudaSuccess) return HG_ERR_CUDA;
  }
  if (nA > 0) {
    hg_status rc = join_tiles(A, V, w, st);
    if (rc != HG_OK) return rc;
    if (!after_count) {
      HG_TRACE("k_join_merge", st);
      k_join_merge<K><<<join_grid(k_join_merge<K>, w.tiles), kJoinThreads, 0, st>>>(
          A->d_offsets, (const K*)A->d_keys, B->d_offsets, (const K*)B->d_keys, w.tv, w.tiles, w.moff, nullptr,
          nullptr, JoinStamp{}, nullptr);
    }
    rc = device_excl_scan<uint64_t>(w.moff, nA + 1, w.part, st);
    if (rc != HG_OK) return rc;
    {
      HG_TRACE("k_join_write", st);
      k_join_write<K><<<join_grid(k_join_write<K>, w.tiles), kJoinThreads, 0, st>>>(
          A->d_offsets, (const K*)A->d_keys, A->d_ids, B->d_offsets, (const K*)B->d_keys, B->d_ids, w.tv, w.tiles,
          w.moff, outA, outB, cap, &hdr->join_abort);
    }
  }
  {
    HG_TRACE("k_join_finish", st);
    k_join_finish<<<1, 1, 0, st>>>(w.moff, nA, cap, d_total, &hdr->status, &hdr->join_abort, hdr->join_stamp);
  }
  return last_launch_status();
}

#define HG_INST(K, M)                                                                                          \
  template hg_status join_count_impl<K, M>(const hg_config*, const hg_table*, const hg_table*, int64_t*,       \
                                           int64_t*, uint8_t*, cudaStream_t, M);                              \
  template hg_status join_materialize_impl<K, M>(const hg_config*, const hg_table*, const hg_table*, int64_t*, \
                                                 int64_t*, uint64_t, int64_t*, uint8_t*, cudaStream_t, M, bool);
HG_INST(uint32_t, MurmurMap)
HG_INST(uint64_t, MurmurMap)
HG_INST(uint32_t, LearnedMap)
HG_INST(uint64_t, LearnedMap)
#undef HG_INST

}  // namespace hg
