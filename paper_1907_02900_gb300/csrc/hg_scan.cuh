// Device-wide exclusive prefix sum (the "PrefixSum" of Alg. 1 and Alg. 2):
// per-tile reduction, one-CTA scan of the tile sums, per-tile scan + base.
#pragma once

#include "hg_device.cuh"
#include "hg_trace.h"

namespace hg {

constexpr int kScanThreads = 1024, kScanIPT = 8, kScanTile = kScanThreads * kScanIPT;

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(const T* __restrict__ a, uint64_t m,
                                                                T* __restrict__ part) {
  __shared__ T wsum[32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  T s = 0;
#pragma unroll
  for (int r = 0; r < kScanIPT; ++r) {
    const uint64_t i = base + (uint64_t)r * kScanThreads + threadIdx.x;
    if (i < m) s += a[i];
  }
  s = warp_sum(s);
  if (lane_id() == 0) wsum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    T x = threadIdx.x < (blockDim.x >> 5) ? wsum[threadIdx.x] : T(0);
    x = warp_sum(x);
    if (threadIdx.x == 0) part[blockIdx.x] = x;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_top(T* part, uint64_t np, T* total) {
  __shared__ T wsum[32];
  const uint64_t per = (np + blockDim.x - 1) / blockDim.x;
  const uint64_t b = threadIdx.x * per, e = min(b + per, np);
  T s = 0;
  for (uint64_t i = b; i < e; ++i) s += part[i];
  T tot;
  T base = block_excl_scan<T>(s, wsum, &tot);
  for (uint64_t i = b; i < e; ++i) {
    const T x = part[i];
    part[i] = base;
    base += x;
  }
  if (total && threadIdx.x == 0) *total = tot;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(T* __restrict__ a, uint64_t m,
                                                             const T* __restrict__ part) {
  __shared__ T wsum[32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanIPT;
  T v[kScanIPT];
  T s = 0;
#pragma unroll
  for (int r = 0; r < kScanIPT; ++r) {
    v[r] = base + r < m ? a[base + r] : T(0);
    s += v[r];
  }
  T run = block_excl_scan<T>(s, wsum, (T*)nullptr) + part[blockIdx.x];
#pragma unroll
  for (int r = 0; r < kScanIPT; ++r) {
    if (base + r < m) a[base + r] = run;
    run += v[r];
  }
}

template <typename T>
inline size_t scan_workspace_bytes(uint64_t m) {
  return align_up(((m + kScanTile - 1) / kScanTile + 1) * sizeof(T));
}

// In-place exclusive scan of a[0..m); the grand total goes to *total when given.
template <typename T>
inline hg_status device_excl_scan(T* a, uint64_t m, T* part, cudaStream_t st, T* total = nullptr) {
  if (m == 0) return HG_OK;
  const uint64_t nb = (m + kScanTile - 1) / kScanTile;
  {
    HG_TRACE("k_scan_partials", st);
    k_scan_partials<T><<<(unsigned)nb, kScanThreads, 0, st>>>(a, m, part);
  }
  {
    HG_TRACE("k_scan_top", st);
    k_scan_top<T><<<1, 1024, 0, st>>>(part, nb, total);
  }
  {
    HG_TRACE("k_scan_apply", st);
    k_scan_apply<T><<<(unsigned)nb, kScanThreads, 0, st>>>(a, m, part);
  }
  return last_launch_status();
}

}  // namespace hg
