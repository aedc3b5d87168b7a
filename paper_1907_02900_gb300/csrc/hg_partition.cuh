// Tile-level stable partition and in-shared-memory counting sort, shared by
// the build, the overflow path and the V1 fix-up.
#pragma once

#include "hg_device.cuh"

namespace hg {

// Stable partition of one tile (held in registers, IPT items per thread in
// block_stable_rank order) into global memory through running per-digit
// cursors: element j of the digit-sorted tile goes to
// cursor[d] + (j - dstart[d]).  The tile is staged in digit order in shared
// memory first, so global writes come out as contiguous runs per digit.
// Afterwards cursor[d] has advanced by the tile's count of digit d.
template <typename K, int IPT, int NW>
__device__ __forceinline__ void tile_partition_out(const K (&key)[IPT], const uint32_t (&val)[IPT],
                                                   const uint32_t (&dig)[IPT], uint32_t n, int ndig,
                                                   K* sk, uint32_t* sv, uint8_t* sd, uint32_t* wc,
                                                   uint32_t* dstart, uint32_t* cursor,
                                                   uint32_t* wsum, K* __restrict__ out_k,
                                                   uint32_t* __restrict__ out_v) {
  uint32_t dest[IPT];
  block_stable_rank<IPT, NW, uint32_t>(dig, n, dest, ndig, wc, dstart, wsum);
  const uint32_t seg0 = (threadIdx.x >> 5) * (32u * IPT), lane = lane_id();
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    if (idx < n) {
      sk[dest[r]] = key[r];
      sv[dest[r]] = val[r];
      sd[dest[r]] = (uint8_t)dig[r];
    }
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
    const uint32_t d = sd[j];
    const uint32_t g = cursor[d] + (j - dstart[d]);
    out_k[g] = sk[j];
    out_v[g] = sv[j];
  }
  __syncthreads();
  for (int d = threadIdx.x; d < ndig; d += blockDim.x) {
    const uint32_t end = (d + 1 < ndig) ? dstart[d + 1] : n;
    cursor[d] += end - dstart[d];
  }
  __syncthreads();
}

// Stable counting sort of tile positions 0..n-1 by a local bucket index
// lb[p] < nb (nb <= 65536), by two least-significant-digit passes of 8 bits
// (one pass when nb <= 256).  Returns the array holding the sorted
// positions (tmp or perm).  wc: smem CT[256*NW].
template <int IPT, int NW, typename CT>
__device__ __forceinline__ const uint16_t* sort_positions_by_bucket(const uint16_t* lb, uint32_t n,
                                                                    uint32_t nb, uint16_t* tmp,
                                                                    uint16_t* perm, CT* wc,
                                                                    uint32_t* wsum) {
  const uint32_t seg0 = (threadIdx.x >> 5) * (32u * IPT), lane = lane_id();
  uint32_t d[IPT], dest[IPT];
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    d[r] = idx < n ? (uint32_t)(lb[idx] & 255u) : 0u;
  }
  block_stable_rank<IPT, NW, CT>(d, n, dest, nb < 256 ? (int)nb : 256, wc, (uint32_t*)nullptr, wsum);
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    if (idx < n) tmp[dest[r]] = (uint16_t)idx;
  }
  __syncthreads();
  if (nb <= 256) return tmp;
  uint32_t p[IPT];
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    p[r] = idx < n ? tmp[idx] : 0u;
    d[r] = idx < n ? (uint32_t)(lb[p[r]] >> 8) : 0u;
  }
  block_stable_rank<IPT, NW, CT>(d, n, dest, (int)((nb + 255) >> 8), wc, (uint32_t*)nullptr, wsum);
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    if (idx < n) perm[dest[r]] = (uint16_t)p[r];
  }
  __syncthreads();
  return perm;
}

// CSR offsets of one bucket range from the sorted bucket sequence: bucket v
// (local) starts at the number of elements whose bucket is below v.  The
// thread handling sorted element j writes the offsets of every bucket in
// (bucket(j-1), bucket(j)]; j == n closes the range.
__device__ __forceinline__ void write_offsets_from_sorted(const uint16_t* lb, const uint16_t* sorted,
                                                          uint32_t n, uint32_t nb, uint64_t bucket0,
                                                          uint32_t start,
                                                          uint32_t* __restrict__ offsets) {
  for (uint32_t j = threadIdx.x; j <= n; j += blockDim.x) {
    const int64_t cur = j < n ? (int64_t)lb[sorted[j]] : (int64_t)nb;
    const int64_t prev = j > 0 ? (int64_t)lb[sorted[j - 1]] : -1;
    const int64_t hi = cur < (int64_t)nb - 1 ? cur : (int64_t)nb - 1;
    for (int64_t v = prev + 1; v <= hi; ++v) offsets[bucket0 + (uint64_t)v] = start + j;
  }
}

}  // namespace hg
