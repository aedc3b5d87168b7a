// Tile-level partitions (stable, and in any order) and in-shared-memory
// counting sorts, shared by the build, the query grouping, the oversized-bin
// path and the V1 fix-up.
#pragma once

#include "hg_device.cuh"


namespace hg {

// Shared-memory words of block_stable_rank's counter matrix for 256 digits.
template <int NW>
__host__ __device__ constexpr int rank_words() {
  return 256 * rank_row<NW>();
}

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
  block_stable_rank<IPT, NW>(dig, n, dest, ndig, wc, dstart, wsum);
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

// The same stable tile partition with fewer barriers (six per tile):
// per-digit output bases are computed once as delta[d] = cursor[d] - start[d]
// while the cursors advance in the same step, and the counter matrix is
// cleared after its last read, so it is already zero for the next tile.
// Preconditions: wc[0 .. 256*rank_row<NW>()) is zero and 16-byte aligned;
// ndig <= blockDim.x.
// IMPLICIT: val[r] is the element's index in the tile (< 2^16) and its id is
// id_base + val[r]; the index and the digit then share one shared-memory
// word (sd is unused).
template <typename K, int IPT, int NW, bool IMPLICIT>
__device__ __forceinline__ void tile_partition_fast(const K (&key)[IPT], const uint32_t (&val)[IPT],
                                                    const uint32_t (&dig)[IPT], uint32_t n, int ndig, K* sk,
                                                    uint32_t* sv, uint8_t* sd, uint32_t* wc, uint32_t* delta,
                                                    uint32_t* cursor, uint32_t* wsum, K* __restrict__ out_k,
                                                    uint32_t* __restrict__ out_v, uint32_t id_base) {
  constexpr int S = rank_row<NW>();
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const uint32_t seg0 = (uint32_t)w * (32u * IPT);
  const uint32_t lt = lanemask_lt();
  // Ranks inside each round come from warp_peers (computed for all rounds
  // first: they are independent); then, round by round, every lane reads
  // its digit's warp counter and the round's leader (lowest lane of its
  // peer group) stores the advanced count, ordered by __syncwarp.
  uint32_t rank[IPT];
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    rank[r] = seg0 + (uint32_t)r * 32u < n ? warp_peers<8>(dig[r], idx < n) : 0u;  // warp-uniform test
  }
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    if (seg0 + (uint32_t)r * 32u < n) {  // warp-uniform
      const bool valid = seg0 + (uint32_t)r * 32u + lane < n;
      const uint32_t d = dig[r], peers = rank[r];
      const uint32_t old = wc[d * S + w];
      __syncwarp();
      if (valid && (peers & lt) == 0u) wc[d * S + w] = old + __popc(peers);
      rank[r] = old + __popc(peers & lt);
      __syncwarp();
    }
  }
  __syncthreads();
  const int t = threadIdx.x;
  uint32_t tot = 0;
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
  const uint32_t start = block_excl_scan_nt<uint32_t>(tot, wsum);
  if (t < ndig) {
    wc[t * S + NW] = start;
    delta[t] = cursor[t] - start;
    cursor[t] += tot;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    if (idx < n) {
      const uint32_t d = dig[r];
      const uint32_t dest = wc[d * S + NW] + wc[d * S + w] + rank[r];
      sk[dest] = key[r];
      if (IMPLICIT) {
        sv[dest] = val[r] | (d << 16);
      } else {
        sv[dest] = val[r];
        sd[dest] = (uint8_t)d;
      }
    }
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
    if (IMPLICIT) {
      const uint32_t x = sv[j];
      const uint32_t g = delta[x >> 16] + j;
      out_k[g] = sk[j];
      out_v[g] = id_base + (x & 0xffffu);
    } else {
      const uint32_t g = delta[sd[j]] + j;
      out_k[g] = sk[j];
      out_v[g] = sv[j];
    }
  }
  // (16-byte stores; 256 * S words are allocated, a multiple of four)
  for (int i = threadIdx.x; i < (ndig * S + 3) / 4; i += blockDim.x)
    reinterpret_cast<uint4*>(wc)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
}

// Partition of one tile in which equal digits need not keep their order:
// every element takes its rank from a shared-memory atomic on its digit's
// counter, so the tile costs one atomic per element and a 256-entry scan
// instead of the ballots and per-warp counters of tile_partition_fast.
// Used only where the bin build restores the canonical order by id.
// Preconditions: tcnt[0 .. 256) is zero; ndig <= blockDim.x.  IMPLICIT as
// for tile_partition_fast.
// tile_counts (optional): receives the tile's count of every digit (16-bit).
template <typename K, int IPT, int NW, bool IMPLICIT>
__device__ __forceinline__ void tile_partition_any(const K (&key)[IPT], const uint32_t (&val)[IPT],
                                                   const uint32_t (&dig)[IPT], uint32_t n, int ndig, K* sk,
                                                   uint32_t* sv, uint8_t* sd, uint32_t* tcnt, uint32_t* delta,
                                                   uint32_t* cursor, uint32_t* wsum, K* __restrict__ out_k,
                                                   uint32_t* __restrict__ out_v, uint32_t id_base,
                                                   uint16_t* __restrict__ tile_counts = nullptr) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const uint32_t seg0 = (uint32_t)w * (32u * IPT);
  uint32_t rank[IPT];
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    rank[r] = idx < n ? atomicAdd(&tcnt[dig[r]], 1u) : 0u;
  }
  __syncthreads();
  const int t = threadIdx.x;
  const uint32_t tot = t < ndig ? tcnt[t] : 0u;
  if (tile_counts != nullptr && t < ndig) tile_counts[t] = (uint16_t)tot;
  const uint32_t start = block_excl_scan_nt<uint32_t>(tot, wsum);
  if (t < ndig) {
    tcnt[t] = start;
    delta[t] = cursor[t] - start;
    cursor[t] += tot;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    if (idx < n) {
      const uint32_t d = dig[r];
      const uint32_t dest = tcnt[d] + rank[r];
      sk[dest] = key[r];
      if (IMPLICIT) {
        sv[dest] = val[r] | (d << 16);
      } else {
        sv[dest] = val[r];
        sd[dest] = (uint8_t)d;
      }
    }
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
    if (IMPLICIT) {
      const uint32_t x = sv[j];
      const uint32_t g = delta[x >> 16] + j;
      out_k[g] = sk[j];
      out_v[g] = id_base + (x & 0xffffu);
    } else {
      const uint32_t g = delta[sd[j]] + j;
      out_k[g] = sk[j];
      out_v[g] = sv[j];
    }
  }
  for (int i = t; i < 256; i += blockDim.x) tcnt[i] = 0;
  __syncthreads();
}

// Stable counting sort of tile positions 0..n-1 by a local bucket index
// lb[p] < nb (nb <= 65536), by two least-significant-digit passes that split
// the index bits evenly (one pass when nb <= 256).  Returns the array
// holding the sorted positions (tmp or perm).  wc: smem u32[rank_words<NW>()].
template <int IPT, int NW>
__device__ __forceinline__ const uint16_t* sort_positions_by_bucket(const uint16_t* lb, uint32_t n,
                                                                    uint32_t nb, uint16_t* tmp,
                                                                    uint16_t* perm, uint32_t* wc,
                                                                    uint32_t* wsum) {
  const uint32_t seg0 = (threadIdx.x >> 5) * (32u * IPT), lane = lane_id();
  uint32_t bits = 0;
  while ((1u << bits) < nb) ++bits;
  const uint32_t lo_bits = nb <= 256 ? bits : (bits + 1) / 2;
  const uint32_t lo_mask = (1u << lo_bits) - 1u;
  uint32_t d[IPT], dest[IPT];
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    d[r] = idx < n ? ((uint32_t)lb[idx] & lo_mask) : 0u;
  }
  block_stable_rank<IPT, NW>(d, n, dest, nb <= 256 ? (int)nb : (int)(1u << lo_bits), wc, (uint32_t*)nullptr, wsum);
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
    d[r] = idx < n ? ((uint32_t)lb[p[r]] >> lo_bits) : 0u;
  }
  block_stable_rank<IPT, NW>(d, n, dest, (int)(((nb - 1) >> lo_bits) + 1), wc, (uint32_t*)nullptr, wsum);
#pragma unroll
  for (int r = 0; r < IPT; ++r) {
    const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
    if (idx < n) perm[dest[r]] = (uint16_t)p[r];
  }
  __syncthreads();
  return perm;
}

}  // namespace hg
