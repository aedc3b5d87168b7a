// Probe launch declaration.
#pragma once

#include <algorithm>

#include "hg_device.cuh"

namespace hg {

// Probe geometry (compile-time; the defaults are the tuned values).
#ifndef HG_PROBE_THREADS
#define HG_PROBE_THREADS 256
#endif
constexpr int kProbeThreads = HG_PROBE_THREADS;

// qpos (optional): input position of each query, for maps that need it
// (queries probed in a permuted order); null means query i is at position i.
template <typename K, typename Map>
hg_status probe_launch(const K* q, uint64_t nq, const uint32_t* off, const K* ck, uint32_t* out,
                       uint64_t V, cudaStream_t st, Map map, const uint32_t* qpos = nullptr);

}  // namespace hg
