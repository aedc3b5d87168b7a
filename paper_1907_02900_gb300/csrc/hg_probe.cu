// HashGraph-Probe-Standard (Section 3.4): map the query to its bucket, read
// the bucket's two offsets, scan the bucket's edges and count every key equal
// to the query (all instances, Section 5.2).
#include "hg_build.cuh"
#include "hg_trace.h"
#include "hg_probe.cuh"

namespace hg {

// Each thread probes QPT queries whose loads are issued together, so that
// several independent random reads are in flight per thread.
template <typename K, typename Map, int QPT>
__global__ void __launch_bounds__(kProbeThreads) k_probe(const K* __restrict__ q, uint64_t nq,
                                                         const uint32_t* __restrict__ off,
                                                         const K* __restrict__ ck,
                                                         uint32_t* __restrict__ out, uint32_t nquads,
                                                         const uint32_t* __restrict__ qpos, Map map) {
  map.init();
  const uint64_t bd = blockDim.x;
  const uint64_t span = (uint64_t)gridDim.x * bd * QPT;
  for (uint64_t base = (uint64_t)blockIdx.x * bd * QPT + threadIdx.x; base < nq; base += span) {
    K key[QPT];
    uint32_t s[QPT], e[QPT], c[QPT];
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      const uint64_t i = base + k * bd;
      key[k] = i < nq ? __ldcs(q + i) : K(0);
    }
    // The two offsets of a bucket come from one aligned 16-byte load (a random
    // DRAM access costs a whole burst, so one request beats two); only a
    // bucket in the last slot of its quad needs a second load.
    uint32_t bq[QPT];
    uint4 o4[QPT];
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      const uint64_t i = base + k * bd;
      bq[k] = i < nq ? map(key[k], qpos ? __ldg(qpos + i) : (uint32_t)i) : 0u;
      if ((bq[k] >> 2) < nquads) {
        o4[k] = __ldg(reinterpret_cast<const uint4*>(off) + (bq[k] >> 2));
      } else {  // quad not wholly inside the offsets array (or array not 16-byte aligned)
        o4[k] = make_uint4(0u, 0u, 0u, 0u);
        const uint32_t r = bq[k] & 3u;
        const uint32_t lo = __ldg(off + bq[k]), hi = __ldg(off + bq[k] + 1);
        if (r == 0) { o4[k].x = lo; o4[k].y = hi; }
        else if (r == 1) { o4[k].y = lo; o4[k].z = hi; }
        else if (r == 2) { o4[k].z = lo; o4[k].w = hi; }
        else { o4[k].w = lo; }
      }
    }
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      const uint64_t i = base + k * bd;
      const uint32_t r = bq[k] & 3u;
      const uint32_t lo = r == 0 ? o4[k].x : r == 1 ? o4[k].y : r == 2 ? o4[k].z : o4[k].w;
      const uint32_t hi = r == 0 ? o4[k].y : r == 1 ? o4[k].z : r == 2 ? o4[k].w : __ldg(off + bq[k] + 1);
      s[k] = i < nq ? lo : 0u;
      e[k] = i < nq ? hi : 0u;
    }
    K first[QPT];
#pragma unroll
    for (int k = 0; k < QPT; ++k) first[k] = s[k] < e[k] ? __ldg(ck + s[k]) : K(0);
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      uint32_t cnt = (s[k] < e[k] && first[k] == key[k]) ? 1u : 0u;
      uint32_t j = s[k] + 1;
      // four independent loads in flight per round for long buckets
      for (; j + 4 <= e[k]; j += 4) {
        const K a0 = __ldg(ck + j), a1 = __ldg(ck + j + 1), a2 = __ldg(ck + j + 2), a3 = __ldg(ck + j + 3);
        cnt += (a0 == key[k]) + (a1 == key[k]) + (a2 == key[k]) + (a3 == key[k]);
      }
      for (; j < e[k]; ++j) cnt += __ldg(ck + j) == key[k];
      c[k] = cnt;
    }
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      const uint64_t i = base + k * bd;
      if (i < nq) __stcs(out + i, c[k]);
    }
  }
}

template <typename K, typename Map>
hg_status probe_launch(const K* q, uint64_t nq, const uint32_t* off, const K* ck, uint32_t* out,
                       uint64_t V, cudaStream_t st, Map map, const uint32_t* qpos) {
  if (nq == 0) return HG_OK;
  // quads of offsets wholly inside the V+1 entries (none if not 16-byte aligned)
  const uint32_t nquads = ((uintptr_t)off % 16 == 0) ? (uint32_t)((V + 1) / 4) : 0u;
  const int sms = dev_info().sms;
  const uint64_t per_block = (uint64_t)kProbeThreads * kProbeQPT;
  const uint64_t want = (nq + per_block - 1) / per_block;
  const unsigned grid = (unsigned)std::min<uint64_t>(want, (uint64_t)sms * 16);
  {
    HG_TRACE("k_probe", st);
    k_probe<K, Map, kProbeQPT><<<grid, kProbeThreads, 0, st>>>(q, nq, off, ck, out, nquads, qpos, map);
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
