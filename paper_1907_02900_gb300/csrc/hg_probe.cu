// HashGraph-Probe-Standard (Section 3.4): map the query to its bucket, read
// the bucket's two offsets, scan the bucket's edges and count every key equal
// to the query (all instances, Section 5.2).
#include "hg_build.cuh"
#include "hg_trace.h"
#include "hg_probe.cuh"

namespace hg {

// Table loads: read-only path by default; HG_PROBE_LD = 1 caches them in L2
// only, 2 reads them without allocating in L1 (variants for measurement).
#ifndef HG_PROBE_LD
#define HG_PROBE_LD 0
#endif
template <typename T>
__device__ __forceinline__ T probe_ld(const T* p) {
#if HG_PROBE_LD == 1
  return __ldcg(p);
#else
  return __ldg(p);
#endif
}
#if HG_PROBE_LD == 2
template <>
__device__ __forceinline__ uint4 probe_ld<uint4>(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
template <>
__device__ __forceinline__ uint32_t probe_ld<uint32_t>(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
template <>
__device__ __forceinline__ uint64_t probe_ld<uint64_t>(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
#endif

// One query per thread.  The grid is one wave of resident CTAs that sweeps
// the queries in order (query base + threadIdx.x at sweep k, base =
// (k * gridDim.x + blockIdx.x) * blockDim.x), so with grouped queries all
// CTAs work inside one or two groups at any time and each group's slice of
// the table stays in L2 while it is needed: the table is read from DRAM
// once.  (A grid of two waves sweeps every group twice and reads the table
// twice.)  Each thread loads its next query one sweep ahead, so the query's
// DRAM latency is not on its chain of dependent loads.  The kernel is bound
// by L1 request throughput: a warp's random loads touch 32 sectors each.
// Bucket keys read in aligned 16-byte pieces (4-byte keys only: with 8-byte
// keys a piece holds two and measured no faster).  0 switches it off.
#ifndef HG_PROBE_VEC
#define HG_PROBE_VEC 1
#endif

template <typename K, typename Map>
__global__ void __launch_bounds__(kProbeThreads) k_probe(const K* __restrict__ q, uint64_t nq,
                                                         const uint32_t* __restrict__ off,
                                                         const K* __restrict__ ck,
                                                         uint32_t* __restrict__ out, uint32_t nquads,
                                                         const uint32_t* __restrict__ qpos, Map map,
                                                         uint64_t map_buckets) {
  map.init();
  constexpr bool kVec = HG_PROBE_VEC && sizeof(K) == 4;
  // last offset of the table (0 switches the piecewise loads off: keys not 16-byte aligned)
  const uint32_t vec_end = (kVec && (uintptr_t)ck % 16 == 0) ? __ldg(off + map_buckets) : 0u;
  const uint64_t bd = blockDim.x;
  const uint64_t span = (uint64_t)gridDim.x * bd;
  uint64_t base = (uint64_t)blockIdx.x * bd;
  K next = base + threadIdx.x < nq ? __ldcs(q + base + threadIdx.x) : K(0);
  for (; base < nq; base += span) {
    const uint64_t i = base + threadIdx.x;
    const K key = next;
    next = i + span < nq ? __ldcs(q + i + span) : K(0);
    if (i >= nq) continue;
    // The two offsets of a bucket come from one aligned 16-byte load (a random
    // access costs a whole sector either way, so one request beats two); only
    // a bucket in the last slot of its quad needs a second load.
    const uint32_t b = map(key, qpos ? __ldg(qpos + i) : (uint32_t)i);
    const uint32_t r = b & 3u;
    uint32_t s, e;
    if ((b >> 2) < nquads) {
      const uint4 o4 = probe_ld(reinterpret_cast<const uint4*>(off) + (b >> 2));
      s = r == 0 ? o4.x : r == 1 ? o4.y : r == 2 ? o4.z : o4.w;
      e = r == 0 ? o4.y : r == 1 ? o4.z : r == 2 ? o4.w : probe_ld(off + b + 1);
    } else {  // quad not wholly inside the offsets array (or array not 16-byte aligned)
      s = probe_ld(off + b);
      e = probe_ld(off + b + 1);
    }
    uint32_t cnt = 0;
    if (kVec && s < e && vec_end != 0) {
      // The bucket's keys in aligned 16-byte pieces: a bucket of up to 16/kb
      // keys usually costs one load request instead of one per key.  A piece
      // that reaches past the bucket is read only while it stays inside the
      // table's last offset (vec_end), so no load leaves the keys array.
      constexpr uint32_t EPQ = 16 / sizeof(K);
      for (uint32_t j = s & ~(EPQ - 1); j < e; j += EPQ) {
        if (j + EPQ <= vec_end) {
          const uint4 v = probe_ld(reinterpret_cast<const uint4*>(ck + j));
          const K* kv = reinterpret_cast<const K*>(&v);
#pragma unroll
          for (uint32_t l = 0; l < EPQ; ++l) cnt += (j + l >= s) & (j + l < e) & (kv[l] == key);
        } else {
          for (uint32_t l = max(j, s); l < e; ++l) cnt += probe_ld(ck + l) == key;
        }
      }
    } else if (s < e) {
      cnt = probe_ld(ck + s) == key;
      uint32_t j = s + 1;
      // four independent loads in flight per round for long buckets
      for (; j + 4 <= e; j += 4) {
        const K a0 = probe_ld(ck + j), a1 = probe_ld(ck + j + 1), a2 = probe_ld(ck + j + 2), a3 = probe_ld(ck + j + 3);
        cnt += (a0 == key) + (a1 == key) + (a2 == key) + (a3 == key);
      }
      for (; j < e; ++j) cnt += probe_ld(ck + j) == key;
    }
    __stcs(out + i, cnt);
  }
}

template <typename K, typename Map>
hg_status probe_launch(const K* q, uint64_t nq, const uint32_t* off, const K* ck, uint32_t* out,
                       uint64_t V, cudaStream_t st, Map map, const uint32_t* qpos) {
  if (nq == 0) return HG_OK;
  // quads of offsets wholly inside the V+1 entries (none if not 16-byte aligned)
  const uint32_t nquads = ((uintptr_t)off % 16 == 0) ? (uint32_t)((V + 1) / 4) : 0u;
  const int sms = dev_info().sms;
  auto kern = k_probe<K, Map>;
  static int per_sm = 0;  // resident CTAs per SM of this instantiation
  if (per_sm == 0) {
    int x = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&x, kern, kProbeThreads, 0) != cudaSuccess || x <= 0) x = 4;
    per_sm = x;
  }
  const uint64_t want = (nq + kProbeThreads - 1) / kProbeThreads;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * per_sm));
  {
    HG_TRACE("k_probe", st);
    kern<<<grid, kProbeThreads, 0, st>>>(q, nq, off, ck, out, nquads, qpos, map, V);
  }
  return last_launch_status();
}

#define HG_INST(K, M) \
  template hg_status probe_launch<K, M>(const K*, uint64_t, const uint32_t*, const K*, uint32_t*, uint64_t, \
                                        cudaStream_t, M, const uint32_t*);
HG_INST(uint32_t, MurmurMap)
HG_INST(uint64_t, MurmurMap)
HG_INST(uint32_t, LearnedMap)
HG_INST(uint64_t, LearnedMap)
HG_INST(uint32_t, BatchedMap)
#undef HG_INST

}  // namespace hg
