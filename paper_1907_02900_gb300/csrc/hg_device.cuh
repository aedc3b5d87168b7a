// Device-side building blocks of the GB300 HashGraph library.
//
// Everything here is sm_103a device code: the Murmur3 bucket map (Eq. 1),
// the learned bucket map, warp/block scans, the stable block-wide ranking
// of the stable partition steps, and bounded TMA bulk-copy waits.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hg_internal.h"

namespace hg {

constexpr int kWarp = 32;
constexpr uint32_t kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// MurmurHash3 x86_32 over the 4 or 8 little-endian bytes of a key (the hash
// the paper names in Section 2, "Hashing").  Keys are whole 4-byte blocks,
// so there is never a tail.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mm3_mix_block(uint32_t h, uint32_t k) {
  k *= 0xcc9e2d51u;
  k = __funnelshift_l(k, k, 15);
  k *= 0x1b873593u;
  h ^= k;
  h = __funnelshift_l(h, h, 13);
  return h * 5u + 0xe6546b64u;
}
__device__ __forceinline__ uint32_t mm3_finish(uint32_t h, uint32_t len) {
  h ^= len;
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ uint32_t murmur3(uint32_t key, uint32_t seed) {
  return mm3_finish(mm3_mix_block(seed, key), 4u);
}
__device__ __forceinline__ uint32_t murmur3(uint64_t key, uint32_t seed) {
  uint32_t h = mm3_mix_block(seed, (uint32_t)key);
  h = mm3_mix_block(h, (uint32_t)(key >> 32));
  return mm3_finish(h, 8u);
}

// h mod d for 32-bit h and 1 <= d < 2^32 without a divide: division by an
// invariant integer (Granlund and Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994, unsigned case): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, the quotient is
// (t + ((h - t) >> sh1)) >> sh2 for t = high32(m h), sh1 = min(l, 1),
// sh2 = max(l - 1, 0).  One 32-bit high multiply and one multiply-subtract.
// Powers of two (up to 2^32) use a mask.  fastmod_params() sets it up.
struct FastMod {
  uint32_t d, m, sh1, sh2;
  uint32_t mask;
  uint32_t pow2;
  __device__ __forceinline__ uint32_t operator()(uint32_t h) const {
    if (pow2) return h & mask;
    const uint32_t t = __umulhi(m, h);
    return h - ((t + ((h - t) >> sh1)) >> sh2) * d;
  }
};
// Host side: the constants for divisor d (1 <= d < 2^32).
inline void fastmod_params(uint32_t d, uint32_t* m, uint32_t* sh1, uint32_t* sh2) {
  uint32_t l = 0;
  while (l < 32 && (1ull << l) < d) ++l;
  *m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);  // < 2^32 for every d >= 1
  *sh1 = l < 1 ? l : 1u;
  *sh2 = l > 1 ? l - 1 : 0u;
}

// Bucket maps: operator()(key, pos) gives the bucket of the key at input
// position pos (plain maps ignore the position; the batched map finds the
// key's table from it); out_id(pos) is the id stored for the element whose
// carried id is pos (plain maps store it unchanged).
// Eq. 1: bucket = hash(key) mod V.
// slab_base: first bucket of the slab a build works on (the map returns the
// bucket minus slab_base; 0 for a whole table).
// kSkewed: the map may send most queries to a few buckets (an order-
// preserving map does, with keys outside the fitted range); the probe then
// merges its counts back with a balanced merge.
struct MurmurMap {
  static constexpr bool kNeedsPos = false;
  static constexpr bool kSkewed = false;
  static constexpr size_t kStageBytes = 0;  // shared memory stage() can use
  uint32_t seed;
  uint32_t slab_base;
  FastMod mod;
  __device__ __forceinline__ void init() {}
  __device__ __forceinline__ void stage(uint8_t*, size_t) {}
  template <typename K>
  __device__ __forceinline__ uint32_t operator()(K key, uint32_t /*pos*/ = 0) const {
    return mod(murmur3(key, seed)) - slab_base;
  }
  __device__ __forceinline__ uint32_t out_id(uint32_t id) const { return id; }
};

// Batched tables (not in the paper): many tables share one bucket space.
// Table t owns the global buckets [base_t, base_t + V_t] and the input
// positions [begin_t, begin_{t+1}), of which the first len_t hold its keys
// and the rest (fewer than 4) only align the next table to 16 bytes.  The
// bucket of the key at position p is base_t + murmur3(key) mod V_t (Eq. 1
// per table) for the table t holding p; an alignment position goes to the
// spare bucket base_t + V_t, which no hash reaches, so table t's V_t + 1
// offsets and its edges are exactly those of a standalone build.  t is found
// through a page directory (the table holding the first position of every
// page of 2^page_shift positions) and a short forward walk.  One instance
// serves one launch sequence that sees the positions pos_base + [0, n) and
// the buckets bucket_base + [0, V).
struct BatchedMap {
  static constexpr bool kNeedsPos = true;
  static constexpr bool kSkewed = false;
  static constexpr size_t kStageBytes = 0;
  uint32_t seed;
  uint32_t page_shift;
  uint64_t pos_base;
  uint32_t bucket_base;
  const uint64_t* begin;  // [T+1] first position of each table
  const uint32_t* len;    // [T] positions of each table that hold keys
  const uint32_t* page;   // table holding position (p << page_shift)
  const uint4* desc;      // per table: {global bucket base, V_t, fastmod m, sh1 | sh2 << 8}
  // The table of the last lookup, kept by each thread: the elements one
  // thread handles mostly belong to the same (large) table, so most lookups
  // become one comparison.  c_lo: the table's first position relative to
  // pos_base (modulo 2^32); c_n: its positions; c_len: those holding keys.
  // All tests are on pos - c_lo, which stays correct when c_lo wraps.
  mutable uint32_t c_lo, c_n, c_len;
  mutable uint4 c_d;
  __device__ __forceinline__ void init() {
    c_lo = 0u;
    c_n = 0u;  // empty range: the first lookup misses
  }
  __device__ __forceinline__ void stage(uint8_t*, size_t) {}
  __device__ __forceinline__ uint32_t table_of(uint64_t p) const {
    uint32_t t = __ldg(page + (p >> page_shift));
    while (__ldg((const unsigned long long*)begin + t + 1) <= p) ++t;
    return t;
  }
  __device__ __forceinline__ void lookup(uint32_t pos) const {
    if (pos - c_lo < c_n) return;  // inside the cached table
    const uint64_t p = pos_base + pos;
    const uint32_t t = table_of(p);
    const uint64_t b0 = __ldg((const unsigned long long*)begin + t);
    const uint64_t b1 = __ldg((const unsigned long long*)begin + t + 1);
    c_lo = (uint32_t)(b0 - pos_base);
    c_n = (uint32_t)(b1 - b0);
    c_len = __ldg(len + t);
    c_d = __ldg(desc + t);
  }
  template <typename K>
  __device__ __forceinline__ uint32_t operator()(K key, uint32_t pos) const {
    lookup(pos);
    if (pos - c_lo >= c_len) return c_d.x - bucket_base + c_d.y;
    // murmur3 mod V_t (see FastMod)
    const uint32_t h = murmur3(key, seed), t = __umulhi(c_d.z, h);
    const uint32_t local = h - ((t + ((h - t) >> (c_d.w & 255u))) >> (c_d.w >> 8)) * c_d.y;
    return c_d.x - bucket_base + local;
  }
  // ids are stored table-local: position minus the table's first position
  __device__ __forceinline__ uint32_t out_id(uint32_t pos) const {
    lookup(pos);
    return pos - c_lo;
  }
};

// ---------------------------------------------------------------------------
// Learned bucket map (not in the paper).  Two-layer piecewise-linear CDF
// model stored as a blob in device memory:
//   header 32 B: u32 magic, u32 L, u64 V, f32 root_a, f32 root_b, u32 key_type, u32 flags
//   leaf   24 B: u64 xmin, f32 slope, f32 icpt, u32 base, u32 width
// Root: leaf = clamp(floor(a * f(key) + b), 0, L-1) with the monotone feature
// f(key) = fp32(bits(fp32(key))).  Leaf j: bucket = base_j +
// clamp(floor(slope_j * fp32(key - xmin_j) + icpt_j), 0, width_j - 1).  All
// fp32 operations are explicitly round-to-nearest and unfused, so results
// are identical to any IEEE implementation of the same steps.
// ---------------------------------------------------------------------------
struct LearnedLeaf {
  uint64_t xmin;
  float slope;
  float icpt;
  uint32_t base;
  uint32_t width;
};
static_assert(sizeof(LearnedLeaf) == 24, "leaf layout");
constexpr uint32_t kModelMagic = 0x4D4C4748u;  // "HGLM"
constexpr size_t kModelHeaderBytes = 32;

__device__ __forceinline__ float rmi_feature(uint32_t key) {
  return __uint2float_rn(__float_as_uint(__uint2float_rn(key)));
}
__device__ __forceinline__ float rmi_feature(uint64_t key) {
  return __uint2float_rn(__float_as_uint(__ull2float_rn(key)));
}

constexpr uint32_t kStageLeaves = 1024;  // leaf records a kernel can stage in shared memory

struct LearnedMap {
  static constexpr bool kNeedsPos = false;
  static constexpr bool kSkewed = true;
  static constexpr size_t kStageBytes = kStageLeaves * sizeof(LearnedLeaf);
  const uint8_t* blob;  // device pointer
  uint64_t Vcap;        // buckets of the table being built (host-provided bound)
  uint32_t slab_base;   // first bucket of the slab being built (subtracted from the result)
  float a, b, Lf;
  uint32_t L;
  uint64_t V, vmax;
  const LearnedLeaf* leaves;
  uint32_t sleaves;     // shared-memory address of the staged leaves (0: not staged)
  __device__ __forceinline__ void init() {
    L = __ldg((const uint32_t*)(blob + 4));
    V = __ldg((const unsigned long long*)(blob + 8));
    a = __ldg((const float*)(blob + 16));
    b = __ldg((const float*)(blob + 20));
    Lf = __uint2float_rn(L);
    vmax = V < Vcap ? V : Vcap;
    leaves = (const LearnedLeaf*)(blob + kModelHeaderBytes);
    sleaves = 0;
  }
  // Copies the leaf records into `smem` (16-byte aligned, `bytes` long)
  // when they fit, so that inference reads them from shared memory.  Every
  // thread of the block must call it (after init()); it ends with a barrier.
  __device__ __forceinline__ void stage(uint8_t* smem, size_t bytes) {
    if ((size_t)L * sizeof(LearnedLeaf) <= bytes) {
      const unsigned long long* src = (const unsigned long long*)leaves;
      unsigned long long* dst = (unsigned long long*)smem;
      for (uint32_t i = threadIdx.x; i < L * 3; i += blockDim.x) dst[i] = __ldg(src + i);
      sleaves = (uint32_t)__cvta_generic_to_shared(smem);
    }
    __syncthreads();
  }
  template <typename K>
  __device__ __forceinline__ uint32_t leaf_of(K key) const {
    float r = __fadd_rn(__fmul_rn(a, rmi_feature(key)), b);
    if (!(r >= 0.0f)) return 0;
    if (r >= Lf) return L - 1;
    return (uint32_t)r;
  }
  __device__ __forceinline__ uint32_t out_id(uint32_t id) const { return id; }
  template <typename K>
  __device__ __forceinline__ uint32_t operator()(K key, uint32_t /*pos*/ = 0) const {
    // a leaf record is 24 bytes at an 8-byte boundary: three 8-byte loads,
    // from shared memory when staged
    const uint32_t j = leaf_of(key);
    uint64_t xmin;
    uint2 si, bw;
    if (sleaves) {
      const uint32_t a0 = sleaves + j * (uint32_t)sizeof(LearnedLeaf);
      asm("ld.shared.u64 %0, [%1];" : "=l"(xmin) : "r"(a0));
      asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(si.x), "=r"(si.y) : "r"(a0 + 8));
      asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(bw.x), "=r"(bw.y) : "r"(a0 + 16));
    } else {
      const unsigned long long* rec = (const unsigned long long*)(leaves + j);
      xmin = __ldg(rec);
      si = __ldg((const uint2*)(rec + 1));
      bw = __ldg((const uint2*)(rec + 2));
    }
    const float slope = __uint_as_float(si.x), icpt = __uint_as_float(si.y);
    const uint32_t base = bw.x, width = bw.y;
    uint32_t local = 0;
    if (width > 0) {
      uint64_t k = (uint64_t)key;
      uint64_t d = k > xmin ? k - xmin : 0ull;
      float p = __fadd_rn(__fmul_rn(slope, __ull2float_rn(d)), icpt);
      if (!(p >= 0.0f)) local = 0;
      else if (p >= __uint2float_rn(width)) local = width - 1;
      else local = min((uint32_t)p, width - 1);
    }
    const uint64_t bk = (uint64_t)base + local;
    return (uint32_t)(bk < vmax ? bk : vmax - 1) - slab_base;
  }
};

// ---------------------------------------------------------------------------
// Device status word (first bytes of every workspace).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(uint32_t* st, uint32_t code) {
  if (st) atomicCAS(st, 0u, code);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Scans.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(kFull, v, o);
    if ((int)lane_id() >= o) v += u;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Exclusive block scan of one value per thread.  wsum: smem[32].  Returns
// the exclusive prefix; *total receives the block sum.  Contains two
// __syncthreads and leaves wsum reusable after a third.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* wsum, T* total) {
  const int lane = lane_id(), w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  T incl = warp_incl_scan(v);
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    T x = lane < nw ? wsum[lane] : T(0);
    x = warp_incl_scan(x);
    wsum[lane] = x;
  }
  __syncthreads();
  T base = (w ? wsum[w - 1] : T(0)) + incl - v;
  if (total) *total = wsum[nw - 1];
  __syncthreads();
  return base;
}

// Exclusive block scan without the trailing barrier: wsum may be reused only
// after the caller's next __syncthreads.
template <typename T>
__device__ __forceinline__ T block_excl_scan_nt(T v, T* wsum) {
  const int lane = lane_id(), w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  T incl = warp_incl_scan(v);
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    T x = lane < nw ? wsum[lane] : T(0);
    x = warp_incl_scan(x);
    wsum[lane] = x;
  }
  __syncthreads();
  return (w ? wsum[w - 1] : T(0)) + incl - v;
}

// In-place exclusive scan of a[0..m) in shared memory by the whole block
// (sums carried in 32 bits).  Returns the total.  wsum: smem u32[32].
template <typename T>
__device__ __forceinline__ uint32_t block_excl_scan_smem(T* a, int m, uint32_t* wsum) {
  const int nt = blockDim.x;
  const int per = (m + nt - 1) / nt;
  const int b = threadIdx.x * per;
  const int e = min(b + per, m);
  uint32_t s = 0;
  for (int i = b; i < e; ++i) s += (uint32_t)a[i];
  uint32_t total;
  uint32_t base = block_excl_scan<uint32_t>(s, wsum, &total);
  for (int i = b; i < e; ++i) {
    const uint32_t x = (uint32_t)a[i];
    a[i] = (T)base;
    base += x;
  }
  __syncthreads();
  return total;
}

// Lanes of the warp whose digit (BITS bits) equals this lane's, among the
// lanes with valid set; an invalid lane gets only itself.  One ballot per
// digit bit (measured faster on GB300 than the hardware match instruction,
// which HG_MATCH_BALLOT=0 selects).
#ifndef HG_MATCH_BALLOT
#define HG_MATCH_BALLOT 1
#endif
template <int BITS>
__device__ __forceinline__ uint32_t warp_peers(uint32_t d, bool valid) {
#if HG_MATCH_BALLOT
  uint32_t m = __ballot_sync(kFull, valid);
#pragma unroll
  for (int b = 0; b < BITS; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t v = __ballot_sync(kFull, bit);
    m &= bit ? v : ~v;
  }
  return valid ? m : (1u << (threadIdx.x & 31u));
#else
  return __match_any_sync(kFull, valid ? d : (0x10000u + (threadIdx.x & 31u)));
#endif
}

// ---------------------------------------------------------------------------
// Stable block-wide ranking by a small digit (ndig <= 256).
//
// The block's element sequence (length n <= NW*32*IPT) is split into NW
// contiguous warp segments of 32*IPT elements; in round r lane l of warp w
// holds element w*32*IPT + r*32 + l.  Inside a warp, equal digits of one
// round are grouped with __match_any_sync and ranked by lane; a per-(digit,
// warp) counter carries the running count from round to round, so ranks
// follow the sequence order.  Then each digit's thread turns its row of
// warp counters into an exclusive prefix, a block scan over the digit totals
// gives every digit its start, and (digit start + warp prefix + rank in
// warp) is the element's position in the stably sorted sequence.
// Counters live at wc[d*(NW+1) + w]: the odd row stride puts the leaders of
// different digits, and the threads of different digits, in different
// shared-memory banks; slot NW of each row receives the digit's start.
//   dig[r]   digit of the element held in round r (ignored when invalid)
//   dest[r]  out: position of that element in the stably sorted sequence
//   wc       smem u32[ndig*(NW+1)] (scratch)
//   dstart   smem u32[ndig] out: first sorted position of each digit (or null)
//   wsum     smem u32[32] (scratch)
// Requires ndig <= blockDim.x.  Contains __syncthreads; every thread of the
// block must call it.
// ---------------------------------------------------------------------------
template <int NW>
__host__ __device__ constexpr int rank_row() {
  return NW + 1 + (NW & 1);  // odd row stride with a spare slot after the NW counters
}

template <int IPT, int NW>
__device__ __forceinline__ void block_stable_rank(const uint32_t (&dig)[IPT], uint32_t n,
                                                  uint32_t (&dest)[IPT], int ndig, uint32_t* wc,
                                                  uint32_t* dstart, uint32_t* wsum) {
  constexpr int S = rank_row<NW>();
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int m = ndig * S;
  for (int i = threadIdx.x; i < m; i += blockDim.x) wc[i] = 0;
  __syncthreads();
  const uint32_t seg0 = (uint32_t)w * (32u * IPT);
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    if (seg0 + (uint32_t)r * 32u < n) {  // warp-uniform
      const bool valid = idx < n;
      const uint32_t d = dig[r];
      const uint32_t peers = warp_peers<8>(d, valid);
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (valid && lane == leader) {
        old = wc[d * S + w];
        wc[d * S + w] = old + __popc(peers);
      }
      old = __shfl_sync(kFull, old, leader);
      dest[r] = old + __popc(peers & lt);
      __syncwarp();
    } else {
      dest[r] = 0;
    }
  }
  __syncthreads();
  uint32_t tot = 0;
  const int t = threadIdx.x;
  if (t < ndig) {
    uint32_t c[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) c[k] = wc[t * S + k];
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      wc[t * S + k] = tot;
      tot += c[k];
    }
  }
  const uint32_t start = block_excl_scan<uint32_t>(tot, wsum, (uint32_t*)nullptr);
  if (t < ndig) {
    wc[t * S + NW] = start;
    if (dstart) dstart[t] = start;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    if (idx < n) dest[r] += wc[dig[r] * S + NW] + wc[dig[r] * S + w];
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// TMA bulk copies (cp.async.bulk) into shared memory with mbarrier
// completion, and bounded waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for phase `parity` of `bar`, giving up after kWaitLimitNs.  Returns a
// block-uniform verdict (every thread must call).  On failure it records
// HG_ERR_TIMEOUT, waits once more (bounded) so that no copy is still landing
// in shared memory, and the caller must return.
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s
__device__ __forceinline__ bool mbar_wait_block(uint64_t* bar, uint32_t parity, uint32_t* status,
                                                uint64_t limit_ns = kWaitLimitNs) {
  bool ok = mbar_try_wait(bar, parity);
  if (!ok) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
      if (mbar_try_wait(bar, parity)) {
        ok = true;
        break;
      }
      if ((it & 255u) == 0 && globaltimer_ns() - t0 > limit_ns) break;
    }
  }
  ok = __syncthreads_and(ok);
  if (!ok) {
    set_status(status, HG_ERR_TIMEOUT);
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity) && globaltimer_ns() - t0 < limit_ns) {
    }
  }
  return ok;
}

// Copy elements [k0, k1) of a device array g (element size ES bytes; the
// base need only be ES-aligned) into smem so that smem[x - a0] holds element
// x, where a0 is the last element at or below k0 whose address is 16-byte
// aligned.  When g itself is not 16-byte aligned and k0 lies before its first
// aligned element q, a0 = q - 16/ES lies below the array start (unsigned
// arithmetic wraps; indexes x - a0 stay small).  One TMA bulk copy (issued by
// thread 0 together with the barrier's expected byte count) brings the
// elements from b0 = max(a0, q) up to the last 16-byte boundary at or below
// k1; elements of [k0, k1) outside it (fewer than 16 bytes at the end, and at
// the start only before q) are loaded by the caller with load_edges() after
// the wait.  Elements between a0 and k0 that the copy brings along are inside
// the array and unused.  Staging buffers hold 16/ES spare elements.  Indexes
// are 32-bit (every array here has fewer than 2^32 elements).  (Arrays that
// start inside another array, such as one slab of a larger build, need the
// unaligned case.)
template <int ES>
struct TileSpan {
  uint32_t a0;    // element a0 sits at smem[0]
  uint32_t k0, end;
  uint32_t b0;    // first element of the bulk copy
  uint32_t body;  // elements copied by TMA: [b0, b0 + body)
  __device__ __forceinline__ uint32_t bytes() const { return body * ES; }
  __device__ __forceinline__ uint32_t dst() const { return b0 - a0; }   // smem index of b0
  __device__ __forceinline__ uint32_t lead() const { return k0 - a0; }  // smem index of k0
  __device__ __forceinline__ bool edges() const { return b0 > k0 || b0 + body < end; }
};
// Index of the first element of g with a 16-byte aligned address (computed
// once per kernel).
template <int ES, typename T>
__device__ __forceinline__ uint32_t align_first(const T* g) {
  return (uint32_t)((16 - ((uintptr_t)g & 15)) & 15) / ES;
}
template <int ES>
__device__ __forceinline__ TileSpan<ES> tile_span(uint32_t q, uint64_t k0_, uint64_t k1_) {
  constexpr uint32_t pm = 16 / ES - 1;
  const uint32_t k0 = (uint32_t)k0_, k1 = (uint32_t)k1_;
  TileSpan<ES> s;
  s.k0 = k0;
  s.end = k1;
  s.a0 = k0 - ((k0 - q) & pm);
  s.b0 = s.a0 > k0 ? s.a0 + pm + 1 : s.a0;  // a0 wrapped below the array start: the copy starts at q
  const uint32_t b1 = k1 - ((k1 - q) & pm);
  if (b1 > s.b0 && b1 <= k1) {
    s.body = b1 - s.b0;
  } else {
    s.b0 = k0;
    s.body = 0;
  }
  return s;
}
template <int ES, typename T>
__device__ __forceinline__ void load_edges(T* smem, const T* g, const TileSpan<ES>& s) {
  for (uint64_t x = s.k0 + threadIdx.x; x < s.b0; x += blockDim.x) smem[(uint32_t)x - s.a0] = g[x];
  for (uint64_t x = (uint64_t)s.b0 + s.body + threadIdx.x; x < s.end; x += blockDim.x)
    smem[(uint32_t)x - s.a0] = g[x];
}

}  // namespace hg
