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
                                                         uint32_t* __restrict__ out, Map map) {
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
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      const uint64_t i = base + k * bd;
      if (i < nq) {
        const uint32_t b = map(key[k]);
        s[k] = __ldg(off + b);
        e[k] = __ldg(off + b + 1);
      } else {
        s[k] = e[k] = 0;
      }
    }
    K first[QPT];
#pragma unroll
    for (int k = 0; k < QPT; ++k) first[k] = s[k] < e[k] ? __ldg(ck + s[k]) : K(0);
#pragma unroll
    for (int k = 0; k < QPT; ++k) {
      uint32_t cnt = (s[k] < e[k] && first[k] == key[k]) ? 1u : 0u;
      for (uint32_t j = s[k] + 1; j < e[k]; ++j) cnt += __ldg(ck + j) == key[k];
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
                       cudaStream_t st, Map map) {
  if (nq == 0) return HG_OK;
  const int sms = dev_info().sms;
  const uint64_t per_block = (uint64_t)kProbeThreads * kProbeQPT;
  const uint64_t want = (nq + per_block - 1) / per_block;
  const unsigned grid = (unsigned)std::min<uint64_t>(want, (uint64_t)sms * 16);
  {
    HG_TRACE("k_probe", st);
    k_probe<K, Map, kProbeQPT><<<grid, kProbeThreads, 0, st>>>(q, nq, off, ck, out, map);
  }
  return last_launch_status();
}

#define HG_INST(K, M) \
  template hg_status probe_launch<K, M>(const K*, uint64_t, const uint32_t*, const K*, uint32_t*, cudaStream_t, M);
HG_INST(uint32_t, MurmurMap)
HG_INST(uint64_t, MurmurMap)
HG_INST(uint32_t, LearnedMap)
HG_INST(uint64_t, LearnedMap)
#undef HG_INST

}  // namespace hg
