// HashGraph-Probe-New (Alg. 3): intersect the adjacency arrays of two tables
// bucket by bucket.  Both tables are built with the same V and bucket map,
// so equal keys always meet in the same bucket index.
//
//   k_join_elem    per edge a of table A: m(a) = number of edges of B's bucket
//                  with key(a); heavy A buckets also get their sum by atomics
//   k_join_bucket  per bucket: sum of m over a light A bucket; join total
//   scan of m      -> output position of every A edge (canonical pair order:
//                  bucket, A's CSR position, B's CSR position)
//   k_join_write   every A edge writes its matching (A id, B id) pairs
#include "hg_build.cuh"
#include "hg_trace.h"
#include "hg_scan.cuh"

namespace hg {

constexpr uint32_t kJoinLightA = 64;  // A bucket length summed by one thread
constexpr int kJoinThreads = 256;

template <typename K, typename Map>
__global__ void __launch_bounds__(kJoinThreads) k_join_elem(const uint32_t* __restrict__ offA,
                                                            const K* __restrict__ keysA, uint64_t nA,
                                                            const uint32_t* __restrict__ offB,
                                                            const K* __restrict__ keysB,
                                                            uint64_t* __restrict__ m_out,
                                                            unsigned long long* __restrict__ bucket_counts,
                                                            Map map) {
  map.init();
  const uint32_t lane = lane_id();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < nA; base += stride) {
    const uint64_t j = base + lane;
    const bool valid = j < nA;
    uint32_t v = 0, m = 0;
    bool heavy = false;
    if (valid) {
      const K key = keysA[j];
      v = map(key);
      const uint32_t s = __ldg(offB + v), e = __ldg(offB + v + 1);
      for (uint32_t k = s; k < e; ++k) m += __ldg(keysB + k) == key;
      m_out[j] = m;
      heavy = (__ldg(offA + v + 1) - __ldg(offA + v)) > kJoinLightA;
    }
    if (bucket_counts) {
      uint32_t hm = __ballot_sync(kFull, heavy);
      while (hm) {
        const int l = __ffs(hm) - 1;
        const uint32_t vv = __shfl_sync(kFull, v, l);
        const bool mine = heavy && v == vv;
        const uint32_t grp = __ballot_sync(kFull, mine);
        const unsigned long long s = warp_sum((unsigned long long)(mine ? m : 0u));
        if ((int)lane == l && s) atomicAdd(bucket_counts + vv, s);
        hm &= ~grp;
      }
    }
  }
}

// Light buckets: one thread sums m over the bucket's A edges.  Every bucket
// then adds its count to the block's share of the join total.
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

__global__ void __launch_bounds__(kJoinThreads) k_join_bucket(const uint32_t* __restrict__ offA, uint64_t V,
                                                              const uint64_t* __restrict__ m,
                                                              unsigned long long* __restrict__ bucket_counts,
                                                              unsigned long long* __restrict__ total,
                                                              JoinStamp stamp, uint64_t* __restrict__ stamp_out) {
  __shared__ unsigned long long wsum[32];
  if (blockIdx.x == 0 && threadIdx.x < 8) stamp_out[threadIdx.x] = stamp.w[threadIdx.x];
  unsigned long long acc = 0;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = offA[v], e = offA[v + 1];
    unsigned long long c;
    if (e - s <= kJoinLightA) {
      c = 0;
      for (uint32_t j = s; j < e; ++j) c += m[j];
      bucket_counts[v] = c;
    } else {
      c = bucket_counts[v];
    }
    acc += c;
  }
  acc = warp_sum(acc);
  if (lane_id() == 0) wsum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long x = threadIdx.x < (blockDim.x >> 5) ? wsum[threadIdx.x] : 0ull;
    x = warp_sum(x);
    if (threadIdx.x == 0 && x) atomicAdd(total, x);
  }
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

template <typename K, typename Map>
__global__ void __launch_bounds__(kJoinThreads) k_join_write(const K* __restrict__ keysA,
                                                             const uint32_t* __restrict__ idsA, uint64_t nA,
                                                             const uint32_t* __restrict__ offB,
                                                             const K* __restrict__ keysB,
                                                             const uint32_t* __restrict__ idsB,
                                                             const uint64_t* __restrict__ moff,
                                                             int64_t* __restrict__ outA,
                                                             int64_t* __restrict__ outB, uint64_t cap,
                                                             const uint32_t* __restrict__ abort, Map map) {
  __shared__ int64_t stage_a[kJoinThreads / 32][kJoinWin];
  __shared__ int64_t stage_b[kJoinThreads / 32][kJoinWin];
  if (*(volatile const uint32_t*)abort) return;
  map.init();
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  int64_t* sa = stage_a[w];
  int64_t* sb = stage_b[w];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < nA; base += stride) {
    const uint64_t j = base + lane;
    const bool valid = j < nA;
    uint64_t o = valid ? moff[j] : ~0ull, oe = valid ? moff[j + 1] : 0ull;
    if (oe > cap) oe = cap;
    K key = K(0);
    int64_t ida = 0;
    uint32_t k = 0, e = 0;
    if (valid && o < oe) {
      key = keysA[j];
      ida = idsA[j];
      const uint32_t v = map(key);
      k = __ldg(offB + v);
      e = __ldg(offB + v + 1);
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
      for (uint64_t i = w0 + lane; i < w1; i += 32) {
        outA[i] = sa[i - w0];
        outB[i] = sb[i - w0];
      }
      __syncwarp();
    }
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
  size_t total;
};

static JoinWs join_layout(uint8_t* ws, uint64_t nA, uint64_t V) {
  JoinWs w{};
  size_t o = sizeof(WsHeader);
  w.moff = (uint64_t*)(ws + o);                  o = align_up(o + (nA + 1) * 8);
  w.part = (uint64_t*)(ws + o);                  o = align_up(o + scan_workspace_bytes<uint64_t>(nA + 1));
  w.bucket_counts = (unsigned long long*)(ws + o); o = align_up(o + V * 8);
  w.total = o;
  return w;
}

size_t join_workspace_bytes(uint64_t nA, uint64_t V) { return join_layout(nullptr, nA, V).total; }

template <typename K, typename Map>
hg_status join_count_impl(const hg_config* cfg, const hg_table* A, const hg_table* B, int64_t* d_total,
                          int64_t* d_bucket_counts, uint8_t* ws, cudaStream_t st, Map map) {
  const uint64_t V = cfg->num_buckets, nA = A->n;
  JoinWs w = join_layout(ws, nA, V);
  unsigned long long* bc = d_bucket_counts ? (unsigned long long*)d_bucket_counts : w.bucket_counts;
  if (cudaMemsetAsync(bc, 0, V * 8, st) != cudaSuccess) return HG_ERR_CUDA;
  if (cudaMemsetAsync(d_total, 0, 8, st) != cudaSuccess) return HG_ERR_CUDA;
  const int sms = dev_info().sms;
  if (nA > 0) {
    const unsigned g = (unsigned)std::min<uint64_t>((nA + kJoinThreads - 1) / kJoinThreads, (uint64_t)sms * 16);
    {
      HG_TRACE("k_join_elem", st);
      k_join_elem<K, Map><<<g, kJoinThreads, 0, st>>>(A->d_offsets, (const K*)A->d_keys, nA, B->d_offsets,
                                                      (const K*)B->d_keys, w.moff, bc, map);
    }
  }
  const unsigned gb = (unsigned)std::min<uint64_t>((V + kJoinThreads - 1) / kJoinThreads, (uint64_t)sms * 16);
  {
    HG_TRACE("k_join_bucket", st);
    k_join_bucket<<<gb, kJoinThreads, 0, st>>>(A->d_offsets, V, w.moff, bc, (unsigned long long*)d_total,
                                               join_stamp(A, B, V), ((WsHeader*)ws)->join_stamp);
  }
  return last_launch_status();
}

// after_count: the per-edge match counts come from the hg_join_count call
// that last used this workspace on the same tables (checked on the device)
// instead of a second intersection pass.
template <typename K, typename Map>
hg_status join_materialize_impl(const hg_config* cfg, const hg_table* A, const hg_table* B, int64_t* outA,
                                int64_t* outB, uint64_t cap, int64_t* d_total, uint8_t* ws, cudaStream_t st,
                                Map map, bool after_count) {
  const uint64_t V = cfg->num_buckets, nA = A->n;
  JoinWs w = join_layout(ws, nA, V);
  WsHeader* hdr = (WsHeader*)ws;
  const int sms = dev_info().sms;
  const unsigned g = (unsigned)std::min<uint64_t>(std::max<uint64_t>(1, (nA + kJoinThreads - 1) / kJoinThreads),
                                                  (uint64_t)sms * 16);
  if (after_count) {
    HG_TRACE("k_join_check", st);
    k_join_check<<<1, 1, 0, st>>>(join_stamp(A, B, V), hdr->join_stamp, &hdr->join_abort, &hdr->status, w.moff, nA);
  } else {
    if (cudaMemsetAsync(w.moff, 0, (nA + 1) * 8, st) != cudaSuccess) return HG_ERR_CUDA;
    if (nA > 0) {
      HG_TRACE("k_join_elem", st);
      k_join_elem<K, Map><<<g, kJoinThreads, 0, st>>>(A->d_offsets, (const K*)A->d_keys, nA, B->d_offsets,
                                                      (const K*)B->d_keys, w.moff, nullptr, map);
    }
  }
  if (nA > 0) {
    hg_status rc = device_excl_scan<uint64_t>(w.moff, nA + 1, w.part, st);
    if (rc != HG_OK) return rc;
    {
      HG_TRACE("k_join_write", st);
      k_join_write<K, Map><<<g, kJoinThreads, 0, st>>>((const K*)A->d_keys, A->d_ids, nA, B->d_offsets,
                                                       (const K*)B->d_keys, B->d_ids, w.moff, outA, outB, cap,
                                                       &hdr->join_abort, map);
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
