// HashGraph build: V2 (Alg. 2, two-level, shared-memory bins) and V1 (Alg. 1).
//
// V2 on GB300 is organised as three streaming passes plus an on-chip finish:
//   k_hist       per input chunk g: histogram of bins (bin = bucket >> s),
//                bins held in shared memory (Alg. 2 Phase 1, "Bin Counting")
//   k_colscan    per bin: exclusive prefix over chunks; bin totals
//   k_scan_bins  exclusive scan of bin totals -> bin starts (Phase 2 prefix
//                sum); the order mode (see below)
//   k_partition  pass A: chunk -> super-bins (256-way partition);
//                pass B: (super-bin, chunk) -> bins (<=256-way partition)
//                (Phase 2, "Bin Placement and Data Reorganization")
//   k_binbuild   per bin, in shared memory: local bucket index, counting
//                sort, CSR offsets and edges (Phase 3, "HashGraph Creation")
//   k_binbuild_big  bins larger than shared memory, streamed by one CTA each
// The table comes out in the canonical order (bucket, then input position)
// without atomics deciding any position: either both partitions are stable
// and the bin build ranks each bucket by bin position, or (implicit ids and
// every bin in shared memory: order mode 0) the partitions rank tiles in any
// order and the bin build ranks each bucket by id, which is the position.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <unordered_map>

#include "hg_build.cuh"
#include "hg_trace.h"
#include "hg_partition.cuh"
#include "hg_scan.cuh"
#include "hg_probe.cuh"

namespace hg {

// ===========================================================================
// Plan
// ===========================================================================
static int ceil_log2_u64(uint64_t x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

// stream_runs' shared memory after the cursors: tile keys and ids, four u16
// tile arrays, the ranking counters and a scan scratch (last 128 bytes)
__host__ __device__ inline size_t big_rest_bytes(int kb) {
  return align_up((size_t)kBigTile * (kb + 4) + 4 * (size_t)kBigTile * 2, 16) + (size_t)rank_words<kBinNW>() * 4 +
         32 * 4;
}

size_t big_smem_bytes(int kb, uint32_t nb) { return align_up((size_t)nb * 4, 16) + big_rest_bytes(kb) + 64; }

size_t part_smem_bytes(int kb, bool ids_in, int ipt, bool item_list, int nw) {
  const size_t tile = (size_t)nw * 32 * ipt;
  const size_t tb = tile + 16;
  const size_t rw = (size_t)256 * (nw + 1 + (nw & 1));  // rank_words<nw>()
  size_t b = 2 * tb * kb + (ids_in ? 2 * tb * 4 : 0) + tile * (kb + 4 + 1) + rw * 4 +
             2 * 256 * 4;
  return align_up(b, 16) + (item_list ? 2 * kMaxItemsPerCta * 4 : 0) + 32 * 4 + 2 * 8 + 64;
}

bool make_plan_v2(const hg_config* cfg, uint64_t n, Plan* p) {
  const DevInfo& di = dev_info();
  p->kb = cfg->key_type == HG_KEY_U64 ? 8 : 4;
  p->n = n;
  p->V = cfg->num_buckets;
  p->emax = p->kb == 4 ? kBinEmaxU32 : kBinEmaxU64;
  p->tpb = cfg->threads_per_bin;  // 0 (automatic), 512 or 1024
  const uint64_t V = p->V;
  int s;
  if (cfg->bin_shift) {
    s = (int)cfg->bin_shift;
  } else {
    const double target = 0.75 * p->emax;
    const double bpb = n ? target * (double)V / (double)n : (double)V;
    s = bpb <= 1.0 ? 0 : (int)std::floor(std::log2(bpb));
  }
  if (!cfg->bin_shift) s = std::min(s, (int)kMaxBinShift);
  s = std::max(s, ceil_log2_u64(V) - (int)kMaxBinsLog2);
  s = std::max(s, 0);
  if (s > (int)kMaxBinShift) return false;
  p->s = (uint32_t)s;
  const uint64_t nbins = ((V - 1) >> s) + 1;
  if (nbins > (1ull << kMaxBinsLog2)) return false;
  p->nbins = (uint32_t)nbins;
  const int lb = ceil_log2_u64(nbins);
  p->sshift = lb > 8 ? (uint32_t)(lb - 8) : 0u;
  p->nsb = (uint32_t)(((nbins - 1) >> p->sshift) + 1);
  const int sms = std::max(di.sms, 1);
  uint64_t chunk = std::max<uint64_t>(kPartTile, (n + 2 * sms - 1) / (2 * sms));
  chunk = (chunk + 15) / 16 * 16;
  p->chunk = chunk;
  p->G = (uint32_t)std::max<uint64_t>(1, (n + chunk - 1) / chunk);
  size_t o = sizeof(WsHeader);
  p->o_H = o;   o = align_up(o + (size_t)p->G * p->nbins * 4);
  p->o_C = o;   o = align_up(o + (size_t)p->G * p->nsb * 4);
  p->o_CT = o;  o = align_up(o + (size_t)p->nsb * 4);
  p->o_T = o;   o = align_up(o + (size_t)p->nbins * 4);
  p->o_BS = o;  o = align_up(o + ((size_t)p->nbins + 1) * 4);
  p->o_ovf = o; o = align_up(o + (size_t)p->nbins * 4);
  // a huge bin holds more than kHugeSeg edges, so there are at most n / kHugeSeg
  // of them and their segments number at most 2 n / kHugeSeg
  p->max_rows = (uint32_t)(2 * (n / kHugeSeg) + 2);
  p->o_hlist = o;   o = align_up(o + (size_t)(n / kHugeSeg + 1) * 3 * 4);
  p->o_rowdesc = o; o = align_up(o + (size_t)p->max_rows * 2 * 4);
  p->o_rowcnt = o;  o = align_up(o + (size_t)p->max_rows * ((size_t)1 << p->s) * 4);
  p->o_bk = o;  o = align_up(o + ((size_t)n + 16) * p->kb);
  p->o_bi = o;  o = align_up(o + ((size_t)n + 16) * 4);
  p->total = o;
  return true;
}

// ===========================================================================
// Kernels
// ===========================================================================
template <typename K>
__device__ __forceinline__ void unpack16(const uint4& x, K (&k)[16 / sizeof(K)]);
template <>
__device__ __forceinline__ void unpack16<uint32_t>(const uint4& x, uint32_t (&k)[4]) {
  k[0] = x.x; k[1] = x.y; k[2] = x.z; k[3] = x.w;
}
template <>
__device__ __forceinline__ void unpack16<uint64_t>(const uint4& x, uint64_t (&k)[2]) {
  k[0] = ((uint64_t)x.y << 32) | x.x;
  k[1] = ((uint64_t)x.w << 32) | x.z;
}

// Shared memory of k_hist: the histogram (at least 1 KB), then the bucket
// map's staged tables (Map::kStageBytes).
__host__ __device__ inline size_t hist_stage_offset(uint32_t nbins) {
  return align_up((size_t)(nbins < 256u ? 256u : nbins) * 4, 16);
}

// Phase 1: per-chunk bin histogram in shared memory; per super-bin sums.
template <typename K, typename Map>
__global__ void __launch_bounds__(kHistThreads) k_hist(const K* __restrict__ keys, uint64_t n,
                                                       uint64_t chunk, uint32_t s, uint32_t nbins,
                                                       uint32_t sshift, uint32_t nsb,
                                                       uint32_t* __restrict__ H,
                                                       uint32_t* __restrict__ C, Map map,
                                                       uint32_t stage_bytes) {
  extern __shared__ __align__(16) uint32_t hist[];
  map.init();
  map.stage((uint8_t*)hist + hist_stage_offset(nbins), stage_bytes);
  for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  constexpr int per = 16 / sizeof(K);
  const uint64_t c0 = (uint64_t)blockIdx.x * chunk;
  const uint64_t c1 = min(c0 + chunk, n);
  // 16-byte vector loads between the first and the last 16-byte address
  // boundary of the chunk (keys may start anywhere: a slab of a larger
  // build), single loads before and after
  const uint64_t off = ((uintptr_t)keys / sizeof(K)) % per;
  const uint64_t y0 = (c0 + off + per - 1) / per * per, y1 = (c1 + off) / per * per;
  const uint64_t b0 = y1 > y0 ? y0 - off : c1, b1 = y1 > y0 ? y1 - off : c1;
  const uint4* kv = reinterpret_cast<const uint4*>(keys + b0);
  const uint64_t nv = (b1 - b0) / per;
  const uint32_t bd = blockDim.x;
  uint64_t v = threadIdx.x;
  for (; v + 3 * (uint64_t)bd < nv; v += 4 * (uint64_t)bd) {
    uint4 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = __ldcs(kv + v + u * bd);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      K k[per];
      unpack16<K>(x[u], k);
      const uint32_t p0 = (uint32_t)(b0 + (v + u * bd) * per);
#pragma unroll
      for (int e = 0; e < per; ++e) atomicAdd(&hist[map(k[e], p0 + e) >> s], 1u);
    }
  }
  for (; v < nv; v += bd) {
    K k[per];
    unpack16<K>(__ldcs(kv + v), k);
    const uint32_t p0 = (uint32_t)(b0 + v * per);
#pragma unroll
    for (int e = 0; e < per; ++e) atomicAdd(&hist[map(k[e], p0 + e) >> s], 1u);
  }
  for (uint64_t i = c0 + threadIdx.x; i < b0; i += bd) atomicAdd(&hist[map(keys[i], (uint32_t)i) >> s], 1u);
  for (uint64_t i = b1 + threadIdx.x; i < c1; i += bd) atomicAdd(&hist[map(keys[i], (uint32_t)i) >> s], 1u);
  __syncthreads();
  uint32_t* row = H + (uint64_t)blockIdx.x * nbins;
  for (uint32_t i = threadIdx.x; i < nbins; i += bd) row[i] = hist[i];
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5, nw = bd >> 5;
  const uint32_t bps = 1u << sshift;
  for (uint32_t sb = w; sb < nsb; sb += nw) {
    uint32_t sum = 0;
    for (uint32_t j = lane; j < bps; j += 32) {
      const uint32_t b = (sb << sshift) + j;
      if (b < nbins) sum += hist[b];
    }
    sum = warp_sum(sum);
    if (lane == 0) C[(uint64_t)blockIdx.x * nsb + sb] = sum;
  }
}

// Exclusive prefix down every column of a rows x cols table, in place;
// column totals to coltot (may be null).  A CTA takes 32 consecutive columns
// (lane = column) and splits the rows into 32 segments (warp = segment), so
// every row access of a warp is one coalesced 128-byte line: segment sums,
// a scan of each column's 32 segment sums, then the segment rewritten with
// its prefix.  Launch with colscan_launch().
constexpr int kColScanThreads = 1024;
__global__ void __launch_bounds__(kColScanThreads) k_colscan(uint32_t* __restrict__ tab, uint32_t rows,
                                                             uint32_t cols, uint32_t* __restrict__ coltot) {
  __shared__ uint32_t seg[32][33];
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const uint32_t c = blockIdx.x * 32u + lane;
  const uint32_t R = (rows + 31u) / 32u;
  const uint32_t r0 = min(w * R, rows), r1 = min(r0 + R, rows);
  uint32_t* p = tab + c;
  uint32_t sum = 0;
  if (c < cols)
    for (uint32_t r = r0; r < r1; ++r) sum += p[(uint64_t)r * cols];
  seg[w][lane] = sum;
  __syncthreads();
  {  // warp w scans column w's 32 segment sums (lane = segment)
    const uint32_t v = seg[lane][w];
    const uint32_t incl = warp_incl_scan(v);
    seg[lane][w] = incl - v;
  }
  __syncthreads();
  if (c >= cols) return;
  uint32_t run = seg[w][lane];
  for (uint32_t r = r0; r < r1; ++r) {
    const uint32_t v = p[(uint64_t)r * cols];
    p[(uint64_t)r * cols] = run;
    run += v;
  }
  if (coltot && w == 31) coltot[c] = run;
}

static void colscan_launch(uint32_t* tab, uint32_t rows, uint32_t cols, uint32_t* coltot, cudaStream_t st) {
  k_colscan<<<(cols + 31) / 32, kColScanThreads, 0, st>>>(tab, rows, cols, coltot);
}

// Bins above kHugeSeg edges: list entries (bin, first row, rows) and one
// row (bin, segment) per kHugeSeg-edge segment.  Null list: no such split.
struct HugeArgs {
  uint32_t* list;
  uint32_t* count;
  uint32_t* rows;
  uint32_t* rowdesc;
  uint32_t max_rows;
  uint32_t* status;
};

// Exclusive scan of the bin totals (one CTA); list of bins too large for the
// shared-memory bin build (huge ones split into segments); closing CSR
// offset offsets[V] = n; with wide_count, the number of bins of more than
// wide_lo and at most emax edges (the bin build's single-buffered launch).
__global__ void __launch_bounds__(1024) k_scan_bins(const uint32_t* __restrict__ T, uint32_t nbins,
                                                    uint32_t* __restrict__ BS, uint32_t emax,
                                                    uint32_t* __restrict__ ovf_list,
                                                    uint32_t* __restrict__ ovf_count,
                                                    uint32_t* __restrict__ offsets, uint64_t V,
                                                    uint32_t n_end, HugeArgs h, uint32_t* order,
                                                    uint32_t wide_lo = 0, uint32_t* wide_count = nullptr) {
  // Each warp scans a contiguous range of whole 32-bin rows (lane = bin of
  // the row), so every access is coalesced: the range's sum, an exclusive
  // scan of the warp sums, then the range again from its base.
  __shared__ uint32_t wbase[32];
  __shared__ uint32_t wtotal;
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t rows = (nbins + 31u) / 32u, per = (rows + nw - 1) / nw;
  const uint32_t row0 = min(w * per, rows), row1 = min(row0 + per, rows);
  uint32_t part = 0;
  for (uint32_t r = row0; r < row1; ++r) {
    const uint32_t i = r * 32u + lane;
    part += i < nbins ? T[i] : 0u;
  }
  part = warp_sum(part);
  if (lane == 0) wbase[w] = part;
  __syncthreads();
  if (w == 0) {
    const uint32_t v = lane < nw ? wbase[lane] : 0u;
    const uint32_t incl = warp_incl_scan(v);
    if (lane < nw) wbase[lane] = incl - v;
    if (lane == 31) wtotal = incl;
  }
  __syncthreads();
  uint32_t base = wbase[w];
  for (uint32_t r = row0; r < row1; ++r) {
    const uint32_t i = r * 32u + lane;
    const uint32_t t = i < nbins ? T[i] : 0u;
    const uint32_t incl = warp_incl_scan(t);
    if (i < nbins) BS[i] = base + incl - t;
    base += __shfl_sync(kFull, incl, 31);
    if (wide_count && i < nbins && t > wide_lo && t <= emax) atomicAdd(wide_count, 1u);
    if (i >= nbins || t <= emax) continue;
    if (order) *order = 1u;  // this bin is built outside shared memory: stable partitions needed
    if (h.list == nullptr || t <= kHugeSeg) {
      ovf_list[atomicAdd(ovf_count, 1u)] = i;
      continue;
    }
    const uint32_t nr = (t + kHugeSeg - 1) / kHugeSeg;
    const uint32_t q0 = atomicAdd(h.rows, nr);
    if (q0 + nr > h.max_rows) {  // cannot happen: the bound counts every huge bin
      set_status(h.status, HG_ERR_OVERFLOW);
      continue;
    }
    const uint32_t k = atomicAdd(h.count, 1u);
    h.list[3 * k] = i;
    h.list[3 * k + 1] = q0;
    h.list[3 * k + 2] = nr;
    for (uint32_t x = 0; x < nr; ++x) {
      h.rowdesc[2 * (q0 + x)] = i;
      h.rowdesc[2 * (q0 + x) + 1] = x;
    }
  }
  if (threadIdx.x == 0) {
    BS[nbins] = wtotal;
    offsets[V] = n_end;
  }
}

// Phase 2 (both passes).  Pass A: items are input chunks; digit = super-bin.
// Pass B: items are (super-bin, group of gg consecutive chunks) sub-ranges of
// pass A's output, contiguous in memory; digit = bin inside the super-bin.
// A group's elements are in input order, so one running cursor per bin,
// started at the bin start plus the earlier chunks' counts, keeps the pass
// stable when its tiles are.  Tiles stream through shared memory by TMA bulk
// copies, double-buffered; each tile is partitioned (stably, or in any order
// with ANY) and written out as contiguous runs.
template <typename K>
struct PartArgs {
  const K* in_k;
  const uint32_t* in_i;  // null: ids are input positions
  K* out_k;
  uint32_t* out_i;
  uint64_t n, chunk;
  uint32_t G, s, sshift, nbins, nsb;
  uint32_t gg, ngroups;  // pass B: chunks per item, items per super-bin
  const uint32_t* H;   // per (chunk, bin) exclusive column prefix
  const uint32_t* C;   // per (chunk, super-bin) exclusive column prefix
  const uint32_t* CT;  // per super-bin totals
  const uint32_t* BS;  // bin starts
  uint32_t* status;
  uint32_t stage_bytes;  // shared memory after the kernel's own, for the bucket map's tables
  // order mode word (null: always stable); see k_partition
  const uint32_t* order;
  // optional: per tile (tiles start at multiples of the kernel's tile size),
  // the tile's count of every digit, nbins 16-bit entries per tile
  uint16_t* tile_counts;
};

// ANY: tiles ranked by shared-memory atomics, equal digits in any order
// (tile_partition_any).  With a.order set, the build launches both variants
// and the one that does not match the order mode written by k_scan_bins
// returns at once: the unordered one runs only when every bin fits the
// shared-memory bin build, which then restores the canonical order by id.
template <typename K, typename Map, bool PASS_B, int IPT, int NW, int MINB, bool ANY>
__global__ void __launch_bounds__(NW * 32, MINB) k_partition(PartArgs<K> a, Map map) {
  if (a.order != nullptr && ((*(volatile const uint32_t*)a.order == 0u) != ANY)) return;
  constexpr uint32_t TILE = NW * 32 * IPT;
  constexpr uint32_t TB = TILE + 16;
  static_assert(TILE <= 65536, "tile indexes are packed into 16 bits");
  const bool has_ids = PASS_B || a.in_i != nullptr;
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* sp = smem;
  // staging buffer b of keys at kin0 + b * TB, of ids at iin0 + b * TB
  K* const kin0 = (K*)sp; sp += 2 * TB * sizeof(K);
  uint32_t* const iin0 = has_ids ? (uint32_t*)sp : nullptr;
  if (has_ids) sp += 2 * TB * 4;
  K* sk = (K*)sp; sp += TILE * sizeof(K);
  uint32_t* sv = (uint32_t*)sp; sp += TILE * 4;
  uint32_t* wc = (uint32_t*)sp; sp += rank_words<NW>() * 4;
  uint32_t* dstart = (uint32_t*)sp; sp += 256 * 4;
  uint32_t* cursor = (uint32_t*)sp; sp += 256 * 4;
  uint8_t* sd = sp; sp += TILE;
  sp = (uint8_t*)(((uintptr_t)sp + 15) & ~(uintptr_t)15);
  uint32_t* ilo = (uint32_t*)sp; sp += PASS_B ? kMaxItemsPerCta * 4 : 0;
  uint32_t* ihi = (uint32_t*)sp; sp += PASS_B ? kMaxItemsPerCta * 4 : 0;
  uint32_t* wsum = (uint32_t*)sp; sp += 32 * 4;
  uint64_t* bar = (uint64_t*)sp; sp += 2 * 8;
  uint8_t* stage = sp;  // a.stage_bytes (16-byte aligned)

  map.init();
  map.stage(stage, a.stage_bytes);
  const uint32_t koff = align_first<sizeof(K)>(a.in_k), ioff = has_ids ? align_first<4>(a.in_i) : 0u;
  for (int i = threadIdx.x; i < rank_words<NW>(); i += blockDim.x) wc[i] = 0;
  const uint64_t nitems = PASS_B ? (uint64_t)a.nsb * a.ngroups : (uint64_t)a.G;
  if (PASS_B) {
    // input ranges of this CTA's items, gathered once (keeps global loads out
    // of the tile loop's control path)
    for (uint64_t j = threadIdx.x, item = blockIdx.x + j * gridDim.x; item < nitems;
         j += blockDim.x, item = blockIdx.x + j * gridDim.x) {
      const uint32_t sb = (uint32_t)(item / a.ngroups), grp = (uint32_t)(item % a.ngroups);
      const uint32_t g0 = grp * a.gg, g1 = min(g0 + a.gg, a.G);
      const uint32_t base = a.BS[sb << a.sshift];
      ilo[j] = base + a.C[(uint64_t)g0 * a.nsb + sb];
      ihi[j] = base + (g1 < a.G ? a.C[(uint64_t)g1 * a.nsb + sb] : a.CT[sb]);
    }
  }
  // This CTA's items are blockIdx.x + j * gridDim.x for j = 0, 1, ...; the
  // tile stream walks them by j (32-bit), tiles of TILE elements.
  const uint32_t nmine = blockIdx.x < nitems ? (uint32_t)((nitems - blockIdx.x + gridDim.x - 1) / gridDim.x) : 0u;
  auto item_range = [&](uint32_t j, uint64_t& i0, uint64_t& i1) {
    if (!PASS_B) {
      i0 = ((uint64_t)blockIdx.x + (uint64_t)j * gridDim.x) * a.chunk;
      i1 = min(i0 + a.chunk, a.n);
    } else {
      i0 = ilo[j];
      i1 = ihi[j];
    }
  };
  struct Ref {
    uint32_t j;
    bool ok;
    uint64_t t0, t1;
  };
  auto first_from = [&](uint32_t j) -> Ref {
    for (; j < nmine; ++j) {
      uint64_t i0, i1;
      item_range(j, i0, i1);
      if (i1 > i0) return Ref{j, true, i0, min(i0 + TILE, i1)};
    }
    return Ref{0, false, 0, 0};
  };
  auto next_of = [&](const Ref& r) -> Ref {
    uint64_t i0, i1;
    item_range(r.j, i0, i1);
    if (r.t1 < i1) return Ref{r.j, true, r.t1, min(r.t1 + TILE, i1)};
    return first_from(r.j + 1);
  };
  auto issue = [&](const Ref& r, int buf) {
    if (threadIdx.x == 0) {
      const TileSpan<sizeof(K)> sk_ = tile_span<sizeof(K)>(koff, r.t0, r.t1);
      uint32_t bytes = sk_.bytes();
      TileSpan<4> si_{};
      if (has_ids) {
        si_ = tile_span<4>(ioff, r.t0, r.t1);
        bytes += si_.bytes();
      }
      mbar_arrive_expect_tx(&bar[buf], bytes);
      if (sk_.body) tma_load_1d(kin0 + buf * TB + sk_.dst(), a.in_k + sk_.b0, sk_.bytes(), &bar[buf]);
      if (has_ids && si_.body) tma_load_1d(iin0 + buf * TB + si_.dst(), a.in_i + si_.b0, si_.bytes(), &bar[buf]);
    }
  };

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();

  Ref cur = first_from(0);
  if (!cur.ok) return;
  issue(cur, 0);
  uint32_t cur_j = ~0u, sb = 0;
  int ndig = 0;
  const uint32_t seg0 = (threadIdx.x >> 5) * (32u * IPT), lane = lane_id();
  for (uint32_t it = 0; cur.ok; ++it) {
    const int buf = it & 1;
    const Ref nxt = next_of(cur);
    if (nxt.ok) issue(nxt, buf ^ 1);
    if (!mbar_wait_block(&bar[buf], (it >> 1) & 1u, a.status)) return;
    const TileSpan<sizeof(K)> sk_ = tile_span<sizeof(K)>(koff, cur.t0, cur.t1);
    TileSpan<4> si_{};
    if (has_ids) si_ = tile_span<4>(ioff, cur.t0, cur.t1);
    // elements outside the 16-byte boundaries (only where a tile starts or
    // ends unaligned) come in by plain loads; the barrier is needed only then
    bool sync_needed = sk_.edges() || (has_ids && si_.edges());
    load_edges<sizeof(K)>(kin0 + buf * TB, a.in_k, sk_);
    if (has_ids) load_edges<4>(iin0 + buf * TB, a.in_i, si_);
    if (cur.j != cur_j) {  // cursors are first read after tile_partition_fast's first barrier
      cur_j = cur.j;
      const uint32_t item = blockIdx.x + cur.j * gridDim.x;
      if (!PASS_B) {
        ndig = (int)a.nsb;
        for (int d = threadIdx.x; d < ndig; d += blockDim.x)
          cursor[d] = a.BS[(uint32_t)d << a.sshift] + a.C[(uint64_t)item * a.nsb + d];
      } else {
        sb = item / a.ngroups;
        const uint32_t g = (item - sb * a.ngroups) * a.gg;
        const uint32_t b0 = sb << a.sshift;
        ndig = (int)min(1u << a.sshift, a.nbins - b0);
        for (int d = threadIdx.x; d < ndig; d += blockDim.x)
          cursor[d] = a.BS[b0 + d] + a.H[(uint64_t)g * a.nbins + b0 + d];
      }
    }
    if (sync_needed) __syncthreads();  // block-uniform condition
    const uint32_t cnt = (uint32_t)(cur.t1 - cur.t0);
    const K* kk = kin0 + buf * TB + sk_.lead();
    const uint32_t* ii = has_ids ? iin0 + buf * TB + si_.lead() : nullptr;
    K key[IPT];
    uint32_t val[IPT], dig[IPT];
#pragma unroll
    for (int r = 0; r < IPT; ++r) {
      const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
      if (idx < cnt) {
        key[r] = kk[idx];
        val[r] = has_ids ? ii[idx] : idx;
        const uint32_t bucket = map(key[r], has_ids ? val[r] : (uint32_t)(cur.t0 + idx));
        dig[r] = PASS_B ? (bucket >> a.s) - (sb << a.sshift) : bucket >> (a.s + a.sshift);
      } else {
        key[r] = 0;
        val[r] = 0;
        dig[r] = 0;
      }
    }
    if (ANY) {
      if (has_ids)
        tile_partition_any<K, IPT, NW, false>(key, val, dig, cnt, ndig, sk, sv, sd, wc, dstart, cursor, wsum,
                                              a.out_k, a.out_i, 0u);
      else
        tile_partition_any<K, IPT, NW, true>(key, val, dig, cnt, ndig, sk, sv, sd, wc, dstart, cursor, wsum,
                                             a.out_k, a.out_i, (uint32_t)cur.t0,
                                             a.tile_counts ? a.tile_counts + (cur.t0 / TILE) * a.nbins : nullptr);
    } else {
      if (has_ids)
        tile_partition_fast<K, IPT, NW, false>(key, val, dig, cnt, ndig, sk, sv, sd, wc, dstart, cursor, wsum,
                                               a.out_k, a.out_i, 0u);
      else
        tile_partition_fast<K, IPT, NW, true>(key, val, dig, cnt, ndig, sk, sv, sd, wc, dstart, cursor, wsum,
                                              a.out_k, a.out_i, (uint32_t)cur.t0);
    }
    cur = nxt;
  }
}

// Phase 3: build every bin in shared memory.  Persistent CTAs (one or two
// per SM) take bins round-robin; with two staging buffers the next bin's
// keys and ids are fetched by TMA while the current one is sorted.  Bins
// above emax are skipped here.
template <typename K>
struct BinArgs {
  const K* in_k;
  const uint32_t* in_i;
  K* csr_k;
  uint32_t* csr_i;
  uint32_t* offsets;
  const uint32_t* T;
  const uint32_t* BS;
  uint64_t V;
  uint32_t nbins, s, emax;
  uint32_t emin;      // bins of at most emin edges are another launch's; 0: no lower bound (empty
                      // bins are built too: their buckets' offsets must be written)
  uint32_t pos_base;  // added to every offset written (position of element 0 in the CSR arrays)
  int nbuf;  // staging buffers: 2 = next bin prefetched during this one
  uint32_t* status;
  const uint32_t* order;  // order mode word (null: partitions were stable); see k_partition
  const uint32_t* gate;  // null, or a count written by k_scan_bins: the launch returns when it is 0
};

// Whether the bin build recomputes an edge's bucket rather than keeping it
// in shared memory between its two uses (cheap maps only).
template <typename Map>
struct recompute_bucket {
  static constexpr bool value = false;
};
template <>
struct recompute_bucket<MurmurMap> {
  static constexpr bool value = true;
};


// Sorts the slots opos[beg, end) of one bucket (end - beg <= 32 * KR) by
// position, with one warp: every lane holds up to KR positions, counts the
// bucket's positions below each of them (all lanes read the same slot, a
// broadcast) and, once every lane has read them all, stores each at its rank.
// Positions are distinct, so the ranks are a permutation of the slots.
template <int KR>
__device__ __forceinline__ void warp_rank_positions(uint16_t* opos, uint32_t beg, uint32_t end, uint32_t lane) {
  uint32_t p[KR], r[KR];
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const uint32_t i = beg + lane + 32u * k;
    p[k] = i < end ? (uint32_t)opos[i] : 0xffffffffu;
    r[k] = 0;
  }
  for (uint32_t i = beg; i < end; ++i) {
    const uint32_t x = opos[i];
#pragma unroll
    for (int k = 0; k < KR; ++k) r[k] += x < p[k];
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < KR; ++k)
    if (beg + lane + 32u * k < end) opos[beg + r[k]] = (uint16_t)p[k];
  __syncwarp();
}

// The same ranking by id instead of bin position, for bins whose tiles were
// partitioned in any order (the ids are then input positions, distinct):
// every lane holds up to KR (slot, id) pairs, counts the bucket's ids below
// each of them (all lanes read the same slot and id, broadcasts) and stores
// each slot at its rank.
template <int KR>
__device__ __forceinline__ void warp_rank_ids(uint16_t* opos, const uint32_t* ii, uint32_t beg, uint32_t end,
                                              uint32_t lane) {
  uint32_t p[KR], id[KR], r[KR];
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const uint32_t i = beg + lane + 32u * k;
    p[k] = i < end ? (uint32_t)opos[i] : 0u;
    id[k] = i < end ? ii[p[k]] : 0xffffffffu;
    r[k] = 0;
  }
  for (uint32_t i = beg; i < end; ++i) {
    const uint32_t x = ii[opos[i]];
#pragma unroll
    for (int k = 0; k < KR; ++k) r[k] += x < id[k];
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < KR; ++k)
    if (beg + lane + 32u * k < end) opos[beg + r[k]] = (uint16_t)p[k];
  __syncwarp();
}

// Compile-time switches (the defaults are the measured choices): the
// single-buffered second bin-build launch for bins above the double-buffered
// size, and the register ranking by id of buckets of 33 .. kBinRankBucket
// edges when the partitions ranked tiles in any order.
#ifndef HG_BIN_WIDE
#define HG_BIN_WIDE 1
#endif
#ifndef HG_ANY_WARP_RANK
#define HG_ANY_WARP_RANK 1
#endif

// Shared memory of k_binbuild: staging buffers of keys and ids, the local
// bucket array (LB), slot order (u16), packed u16 bucket counters, the list
// of long buckets, kBinBitmapWarps position bitmaps and small control state.
size_t bin_smem_bytes(int kb, uint32_t emax, uint32_t s, int nbuf, bool lb) {
  size_t b = (size_t)nbuf * (emax + 16) * (kb + 4) + (lb ? (size_t)emax * 2 : 0) + (size_t)emax * 2 +
             (((size_t)1 << s) + 1) / 2 * 4 + ((size_t)emax / (kBinSmallBucket + 1) + 2) * 2;
  b = align_up(b, 16) + (size_t)kBinBitmapWarps * ((emax + 31) / 32) * 4;
  return align_up(b, 16) + 32 * 4 + 16 + 2 * kMaxBinsPerCta * 4 + 2 * 8 + 64;
}

// Per bin (E <= emax edges, nb local buckets):
//   1. local bucket of every edge; bucket counts by shared-memory atomics
//      (counts do not depend on order); two 16-bit counters per word
//   2. exclusive scan of the counts -> bucket starts, packed the same way
//   3. every edge claims a slot of its bucket with an atomic increment; the
//      slot order inside a bucket is arbitrary at this point
//   4. buckets above kBinSmallBucket edges sort their slots by position in
//      the bin: up to kBinRankBucket edges one warp ranks a bucket's
//      positions in registers, longer buckets use per-warp position bitmaps;
//      the position is input order when both partition passes were stable
//   5. the edges are written out in slot order, and the bin's offsets
//      (both coalesced)
// LB: the local buckets of step 1 are kept for step 3 (else recomputed).
// ANY: the partitions ranked tiles in any order (see k_partition), so the
// bin positions no longer follow the input order; every bucket of two or
// more edges is then ranked by id (an input position, distinct) instead:
// in registers by one warp for 33 .. kBinRankBucket edges (step 4), edge by
// edge otherwise (step 5).
// A bin takes this kernel when E <= emax and, for emin > 0, E > emin: one
// launch (emin = 0) covers every bin that fits its double-buffered staging,
// empty ones included, a second, single-buffered launch (twice the staging
// room) the larger ones up to its own emax.
template <typename K, typename Map, int NWB, int MINB, bool LB, bool ANY>
__global__ void __launch_bounds__(NWB * 32, MINB) k_binbuild(BinArgs<K> a, Map map) {
  if (a.order != nullptr && ((*(volatile const uint32_t*)a.order == 0u) != ANY)) return;
  if (a.gate != nullptr && *(volatile const uint32_t*)a.gate == 0u) return;  // no bin for this launch
  constexpr uint32_t NBM = kBinBitmapWarps;
  const uint32_t EB = a.emax + 16;
  const int nbuf = a.nbuf;
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* sp = smem;
  // staging buffer b of keys at kin0 + b * EB, of ids at iin0 + b * EB
  K* const kin0 = (K*)sp; sp += (size_t)nbuf * EB * sizeof(K);
  uint32_t* const iin0 = (uint32_t*)sp; sp += (size_t)nbuf * EB * 4;
  uint16_t* lb = (uint16_t*)sp; sp += LB ? (size_t)a.emax * 2 : 0;
  uint16_t* opos = (uint16_t*)sp; sp += (size_t)a.emax * 2;
  uint32_t* cnt = (uint32_t*)sp; sp += (((size_t)1 << a.s) + 1) / 2 * 4;
  uint16_t* heavy = (uint16_t*)sp; sp += (size_t)(a.emax / (kBinSmallBucket + 1) + 2) * 2;
  sp = (uint8_t*)(((uintptr_t)sp + 15) & ~(uintptr_t)15);
  const uint32_t bm_words = (a.emax + 31) / 32;
  uint32_t* bitmaps = (uint32_t*)sp;  // NBM bitmaps of bm_words words
  sp += (size_t)NBM * bm_words * 4;
  sp = (uint8_t*)(((uintptr_t)sp + 15) & ~(uintptr_t)15);
  uint32_t* wsum = (uint32_t*)sp; sp += 32 * 4;
  uint32_t* nheavy = (uint32_t*)sp; sp += 16;
  uint32_t* bl_start = (uint32_t*)sp; sp += kMaxBinsPerCta * 4;  // this CTA's bins: start, size
  uint32_t* bl_size = (uint32_t*)sp; sp += kMaxBinsPerCta * 4;
  uint64_t* bar = (uint64_t*)sp;

  map.init();
  const uint32_t koff = align_first<sizeof(K)>(a.in_k), ioff = align_first<4>(a.in_i);
  // Bins blockIdx.x, +gridDim.x, ...: starts and sizes gathered once, so the
  // loop below needs no global loads to find its next bin.
  const uint32_t nmine = blockIdx.x < a.nbins ? (a.nbins - blockIdx.x + gridDim.x - 1) / gridDim.x : 0u;
  for (uint32_t j = threadIdx.x; j < nmine; j += blockDim.x) {
    const uint32_t bb = blockIdx.x + j * gridDim.x;
    bl_start[j] = a.BS[bb];
    bl_size[j] = a.T[bb];
  }
  __syncthreads();
  auto skip = [&](uint32_t j) {
    while (j < nmine && (bl_size[j] > a.emax || (a.emin != 0 && bl_size[j] <= a.emin))) ++j;
    return j;
  };
  auto issue = [&](uint32_t j, int buf) {
    if (threadIdx.x == 0) {
      const uint64_t k0 = bl_start[j], k1 = k0 + bl_size[j];
      const TileSpan<sizeof(K)> sk_ = tile_span<sizeof(K)>(koff, k0, k1);
      const TileSpan<4> si_ = tile_span<4>(ioff, k0, k1);
      mbar_arrive_expect_tx(&bar[buf], sk_.bytes() + si_.bytes());
      if (sk_.body) tma_load_1d(kin0 + (size_t)buf * EB + sk_.dst(), a.in_k + sk_.b0, sk_.bytes(), &bar[buf]);
      if (si_.body) tma_load_1d(iin0 + (size_t)buf * EB + si_.dst(), a.in_i + si_.b0, si_.bytes(), &bar[buf]);
    }
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t jb = skip(0);
  if (jb >= nmine) return;
  issue(jb, 0);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  for (uint32_t it = 0; jb < nmine; ++it) {
    const uint32_t b = blockIdx.x + jb * gridDim.x;
    const int buf = nbuf == 2 ? (int)(it & 1) : 0;
    const uint32_t jb_next = skip(jb + 1);
    if (nbuf == 2 && jb_next < nmine) issue(jb_next, buf ^ 1);
    const uint64_t bucket0 = (uint64_t)b << a.s;
    const uint32_t nb = (uint32_t)min((uint64_t)1 << a.s, a.V - bucket0);
    const uint32_t nwords = (nb + 1) >> 1;
    for (uint32_t w = threadIdx.x; w < nwords; w += blockDim.x) cnt[w] = 0;
    if (threadIdx.x == 0) *nheavy = 0;
    const uint32_t parity = nbuf == 2 ? (it >> 1) & 1u : it & 1u;
    if (!mbar_wait_block(&bar[buf], parity, a.status)) return;
    const uint32_t E = bl_size[jb], start = bl_start[jb];
    const TileSpan<sizeof(K)> sk_ = tile_span<sizeof(K)>(koff, start, (uint64_t)start + E);
    const TileSpan<4> si_ = tile_span<4>(ioff, start, (uint64_t)start + E);
    K* const kb_ = kin0 + (size_t)buf * EB;
    uint32_t* const ib_ = iin0 + (size_t)buf * EB;
    load_edges<sizeof(K)>(kb_, a.in_k, sk_);
    load_edges<4>(ib_, a.in_i, si_);
    if (sk_.edges() || si_.edges())
      __syncthreads();  // edge elements came in by plain loads (block-uniform condition)
    const K* kk = kb_ + sk_.lead();
    const uint32_t* ii = ib_ + si_.lead();
    // 1. local buckets and counts
    for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
      const uint32_t l = map(kk[e], ii[e]) - (uint32_t)bucket0;
      if (LB) lb[e] = (uint16_t)l;
      atomicAdd(&cnt[l >> 1], 1u << ((l & 1u) << 4));
    }
    __syncthreads();
    // 2. exclusive scan of the counts; buckets above kBinSmallBucket edges
    //    are listed for the bitmap sort
    {
      const uint32_t per = (nwords + blockDim.x - 1) / blockDim.x;
      const uint32_t w0 = min(threadIdx.x * per, nwords), w1 = min(w0 + per, nwords);
      uint32_t sum = 0;
      for (uint32_t w = w0; w < w1; ++w) {
        const uint32_t x = cnt[w];
        sum += (x & 0xffffu) + (x >> 16);
      }
      uint32_t base = block_excl_scan_nt<uint32_t>(sum, wsum);
      for (uint32_t w = w0; w < w1; ++w) {
        const uint32_t x = cnt[w], lo = x & 0xffffu, hi = x >> 16;
        if ((HG_ANY_WARP_RANK || !ANY) && lo > kBinSmallBucket) heavy[atomicAdd(nheavy, 1u)] = (uint16_t)(2 * w);
        if ((HG_ANY_WARP_RANK || !ANY) && hi > kBinSmallBucket) heavy[atomicAdd(nheavy, 1u)] = (uint16_t)(2 * w + 1);
        cnt[w] = base | ((base + lo) << 16);
        base += lo + hi;
      }
    }
    __syncthreads();
    // 3. slots
    for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
      const uint32_t l = LB ? (uint32_t)lb[e] : map(kk[e], ii[e]) - (uint32_t)bucket0;
      const uint32_t sh = (l & 1u) << 4;
      const uint32_t old = atomicAdd(&cnt[l >> 1], 1u << sh);
      opos[(old >> sh) & 0xffffu] = (uint16_t)e;
    }
    __syncthreads();
    // 4. long buckets (every counter now holds its bucket's end): slots
    //    sorted by position, in registers by one warp per bucket (every warp
    //    takes buckets) up to kBinRankBucket edges, else with per-warp
    //    position bitmaps on the first NBM warps
    const uint32_t nh = *nheavy;
    if (nh > 0) {
      const uint32_t nw = blockDim.x >> 5;
      for (uint32_t h = warp; h < nh; h += nw) {
        const uint32_t v = heavy[h];
        const uint32_t end = (cnt[v >> 1] >> ((v & 1u) << 4)) & 0xffffu;
        const uint32_t beg = v ? (cnt[(v - 1) >> 1] >> (((v - 1) & 1u) << 4)) & 0xffffu : 0u;
        if (ANY) {  // by id; longer buckets are ranked edge by edge in step 5
          if (end - beg <= 64) warp_rank_ids<2>(opos, ii, beg, end, lane);
          else if (end - beg <= 128) warp_rank_ids<4>(opos, ii, beg, end, lane);
          else if (end - beg <= kBinRankBucket) warp_rank_ids<kBinRankBucket / 32>(opos, ii, beg, end, lane);
        } else {
          if (end - beg <= 64) warp_rank_positions<2>(opos, beg, end, lane);
          else if (end - beg <= 128) warp_rank_positions<4>(opos, beg, end, lane);
          else if (end - beg <= kBinRankBucket) warp_rank_positions<kBinRankBucket / 32>(opos, beg, end, lane);
        }
      }
    }
    if (!ANY && nh > 0 && warp < NBM) {
      // each of the first NBM warps owns one bitmap of E bits
      const uint32_t nbits_words = (E + 31) >> 5;
      uint32_t* bm = bitmaps + warp * bm_words;
      for (uint32_t h = warp; h < nh; h += NBM) {
        const uint32_t v = heavy[h];
        const uint32_t end = (cnt[v >> 1] >> ((v & 1u) << 4)) & 0xffffu;
        const uint32_t beg = v ? (cnt[(v - 1) >> 1] >> (((v - 1) & 1u) << 4)) & 0xffffu : 0u;
        if (end - beg <= kBinRankBucket) continue;  // ranked above
        for (uint32_t k = lane; k < nbits_words; k += 32) bm[k] = 0;
        __syncwarp();
        for (uint32_t i = beg + lane; i < end; i += 32) {
          const uint32_t p = opos[i];
          atomicOr(&bm[p >> 5], 1u << (p & 31u));
        }
        __syncwarp();
        uint32_t run = beg;
        for (uint32_t k0 = 0; k0 < nbits_words; k0 += 32) {
          uint32_t word = k0 + lane < nbits_words ? bm[k0 + lane] : 0u;
          const uint32_t c = __popc(word);
          const uint32_t incl = warp_incl_scan(c);
          uint32_t pos = run + incl - c;
          while (word) {
            const uint32_t bit = __ffs(word) - 1;
            opos[pos++] = (uint16_t)(((k0 + lane) << 5) + bit);
            word &= word - 1;
          }
          run += __shfl_sync(kFull, incl, 31);
        }
        __syncwarp();
      }
    }
    if (nh > 0) __syncthreads();  // block-uniform: every thread read the same count
    // 5. edges in canonical order: the edge in slot j of a bucket of at most
    //    kBinSmallBucket edges goes to the bucket's start plus the number of
    //    its edges with a smaller position (positions are distinct, so the
    //    ranks are a permutation of the bucket's slots; the stores of a warp
    //    stay within a few sectors); a long bucket is already in order.  With
    //    ANY every bucket is ranked by id the same way.
    //    Then the bin's offsets (bucket v starts where bucket v - 1 ends).
    // Whether slot j's bucket [beg, end) still needs ranking here (longer
    // ones were put in order in step 4), and its rank.
    auto loose = [&](uint32_t beg, uint32_t end) {
      const uint32_t n = end - beg;
      if (n < 2) return false;
      if (ANY) return !HG_ANY_WARP_RANK || n <= kBinSmallBucket || n > kBinRankBucket;
      return n <= kBinSmallBucket;
    };
    auto rank_of = [&](uint32_t beg, uint32_t end, uint32_t p, uint32_t id) {
      uint32_t dst = beg;
      if (ANY)
        for (uint32_t i = beg; i < end; ++i) dst += ii[opos[i]] < id;
      else
        for (uint32_t i = beg; i < end; ++i) dst += opos[i] < p;
      return dst;
    };
    for (uint32_t j = threadIdx.x; j < E; j += blockDim.x) {
      const uint32_t p = opos[j];
      const K key = kk[p];
      const uint32_t id = ii[p];
      const uint32_t l = LB ? (uint32_t)lb[p] : map(key, id) - (uint32_t)bucket0;
      const uint32_t end = (cnt[l >> 1] >> ((l & 1u) << 4)) & 0xffffu;
      const uint32_t beg = l ? (cnt[(l - 1) >> 1] >> (((l - 1) & 1u) << 4)) & 0xffffu : 0u;
      const uint32_t dst = loose(beg, end) ? rank_of(beg, end, p, id) : j;
      a.csr_k[start + dst] = key;
      a.csr_i[start + dst] = map.out_id(id);
    }
    for (uint32_t v = threadIdx.x; v < nb; v += blockDim.x) {
      const uint32_t first = v ? (cnt[(v - 1) >> 1] >> (((v - 1) & 1u) << 4)) & 0xffffu : 0u;
      a.offsets[bucket0 + v] = a.pos_base + start + first;
    }
    __syncthreads();
    if (nbuf == 1 && jb_next < nmine) issue(jb_next, 0);
    jb = jb_next;
  }
}

// Bin-build launch configuration: 512-thread CTAs two to an SM, single
// buffered, when two fit with bins large enough for this build; otherwise
// one CTA per SM (1024 threads unless 512 were asked for), double buffered
// when that fits.
struct BinCfg {
  uint32_t tpb, per_sm, emax;
  int nbuf;
  bool lb;
  size_t smem;
  uint32_t emax_wide;  // largest bin of the single-buffered second launch (<= emax: none)
  size_t smem_wide;
};
// Two 512-thread CTAs per SM (local buckets recomputed, no prefetch) measured
// slower than one 1024-thread CTA that keeps them and prefetches the next bin
// (2.42 against 2.27 ms at 2^28 keys); HG_BIN_TWO_PER_SM=1 selects them.
#ifndef HG_BIN_TWO_PER_SM
#define HG_BIN_TWO_PER_SM 0
#endif
static BinCfg bin_config(const Plan& p, bool recompute) {
  const DevInfo& di = dev_info();
  BinCfg c{};
  if (HG_BIN_TWO_PER_SM && p.tpb != 1024 && di.smem_per_sm > 0) {
    const bool lb = !recompute;
    const double mean = p.nbins ? (double)p.n / (double)p.nbins : 0.0;
    const size_t sm_cap = (size_t)di.smem_per_sm / 2 - (size_t)di.smem_reserved;
    uint32_t e = p.emax;
    while (e > 1024 && (bin_smem_bytes(p.kb, e, p.s, 1, lb) > sm_cap ||
                        bin_smem_bytes(p.kb, e, p.s, 1, lb) > (size_t)di.max_smem_optin))
      e -= 32;
    // bins of a uniform build are Poisson: allow five standard deviations
    if (bin_smem_bytes(p.kb, e, p.s, 1, lb) <= sm_cap && (double)e >= mean + 5.0 * std::sqrt(mean) + 16.0) {
      c.tpb = 512;
      c.per_sm = 2;
      c.emax = e;
      c.nbuf = 1;
      c.lb = lb;
      c.smem = bin_smem_bytes(p.kb, e, p.s, 1, lb);
      return c;
    }
  }
  c.tpb = p.tpb == 512 ? 512u : 1024u;
  c.per_sm = 1;
  c.emax = p.emax;
  c.lb = true;
  c.nbuf = 2;
  c.smem = bin_smem_bytes(p.kb, p.emax, p.s, 2, true);
  if (c.smem > (size_t)di.max_smem_optin) {
    c.nbuf = 1;
    c.smem = bin_smem_bytes(p.kb, p.emax, p.s, 1, true);
  }
  // the largest bin one single-buffered CTA can hold (slot indexes are 16-bit)
  c.emax_wide = 0;
  c.smem_wide = 0;
  if (HG_BIN_WIDE && c.nbuf == 2 && di.max_smem_optin > 0) {
    uint32_t e = 65504;
    while (e > p.emax && bin_smem_bytes(p.kb, e, p.s, 1, true) > (size_t)di.max_smem_optin) e -= 32;
    if (e > p.emax) {
      c.emax_wide = e;
      c.smem_wide = bin_smem_bytes(p.kb, e, p.s, 1, true);
    }
  }
  return c;
}

// Streams edges [start, start + len) of a bin in tiles of kBigTile, sorts
// every tile stably by local bucket and appends each run at its bucket's
// cursor (cur: absolute CSR positions of the bin's nb buckets, advanced).
// Tiles follow input order and each is sorted stably, so every bucket keeps
// ascending input position.
template <typename K, typename Map, int NW>
__device__ __forceinline__ void stream_runs(const BinArgs<K>& a, const Map& map, uint32_t start, uint32_t len,
                                            uint64_t bucket0, uint32_t nb, uint32_t* cur, uint8_t* sp) {
  constexpr int IPT = kBigTile / (NW * 32);
  K* tk = (K*)sp; sp += (size_t)kBigTile * sizeof(K);
  uint32_t* ti = (uint32_t*)sp; sp += (size_t)kBigTile * 4;
  uint16_t* lb = (uint16_t*)sp; sp += kBigTile * 2;
  uint16_t* tmp = (uint16_t*)sp; sp += kBigTile * 2;
  uint16_t* perm = (uint16_t*)sp; sp += kBigTile * 2;
  uint16_t* slb = (uint16_t*)sp; sp += kBigTile * 2;
  sp = (uint8_t*)(((uintptr_t)sp + 15) & ~(uintptr_t)15);
  uint32_t* wc = (uint32_t*)sp; sp += rank_words<NW>() * 4;
  uint32_t* wsum = (uint32_t*)sp;
  for (uint32_t t0 = 0; t0 < len; t0 += kBigTile) {
    const uint32_t cnt = min((uint32_t)kBigTile, len - t0);
    for (uint32_t e = threadIdx.x; e < cnt; e += blockDim.x) {
      const K key = a.in_k[start + t0 + e];
      const uint32_t id = a.in_i[start + t0 + e];
      tk[e] = key;
      ti[e] = id;
      lb[e] = (uint16_t)(map(key, id) - (uint32_t)bucket0);
    }
    __syncthreads();
    const uint16_t* sorted = sort_positions_by_bucket<IPT, NW>(lb, cnt, nb, tmp, perm, wc, wsum);
    for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) slb[j] = lb[sorted[j]];
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) {
      const uint16_t l = slb[j];
      uint32_t lo = 0, hi = j;  // first index with slb == l
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (slb[mid] < l) lo = mid + 1; else hi = mid;
      }
      const uint32_t g = cur[l] + (j - lo);
      const uint32_t p = sorted[j];
      a.csr_k[g] = tk[p];
      a.csr_i[g] = map.out_id(ti[p]);
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) {
      const uint16_t l = slb[j];
      if (j + 1 == cnt || slb[j + 1] != l) {
        uint32_t lo = 0, hi = j;
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          if (slb[mid] < l) lo = mid + 1; else hi = mid;
        }
        cur[l] += j - lo + 1;
      }
    }
    __syncthreads();
  }
}

// Local-bucket counts of edges [start, start + len) of a bin into cur[]
// (zeroed first).  Equal buckets of a warp are merged by __match_any_sync,
// so a bucket holding most of the bin (duplicates) costs one shared-memory
// atomic per warp instead of one per edge.
template <typename K, typename Map>
__device__ __forceinline__ void count_local(const BinArgs<K>& a, const Map& map, uint32_t start, uint32_t len,
                                            uint64_t bucket0, uint32_t nb, uint32_t* cur) {
  for (uint32_t v = threadIdx.x; v < nb; v += blockDim.x) cur[v] = 0;
  __syncthreads();
  const uint32_t lane = lane_id();
  for (uint32_t base = threadIdx.x & ~31u; base < len; base += blockDim.x) {
    const uint32_t e = base + lane;
    const bool valid = e < len;
    const uint32_t l = valid ? map(a.in_k[start + e], a.in_i[start + e]) - (uint32_t)bucket0 : 0xffffffffu;
    const uint32_t peers = __match_any_sync(kFull, l);
    if (valid && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&cur[l], (uint32_t)__popc(peers));
  }
  __syncthreads();
}

// Bins too large for shared memory (duplicates, skew, tiny V) with at most
// kHugeSeg edges: one CTA per bin counts its local buckets, writes the bin's
// offsets and streams the bin (stream_runs).
template <typename K, typename Map>
__global__ void __launch_bounds__(kBinNW * 32, 1) k_binbuild_big(BinArgs<K> a, const uint32_t* ovf_list,
                                                               const uint32_t* ovf_count, Map map) {
  extern __shared__ __align__(16) uint8_t smem[];
  map.init();
  const uint32_t nbmax = 1u << a.s;
  uint32_t* cur = (uint32_t*)smem;
  uint8_t* rest = smem + align_up((size_t)nbmax * 4, 16);
  uint32_t* wsum = (uint32_t*)(rest + big_rest_bytes(sizeof(K)) - 32 * 4);
  const uint32_t novf = *ovf_count;
  for (uint32_t k = blockIdx.x; k < novf; k += gridDim.x) {
    const uint32_t b = ovf_list[k];
    const uint32_t E = a.T[b], start = a.BS[b];
    const uint64_t bucket0 = (uint64_t)b << a.s;
    const uint32_t nb = (uint32_t)min((uint64_t)nbmax, a.V - bucket0);
    count_local(a, map, start, E, bucket0, nb, cur);
    block_excl_scan_smem(cur, (int)nb, wsum);
    for (uint32_t v = threadIdx.x; v < nb; v += blockDim.x) {
      a.offsets[bucket0 + v] = a.pos_base + start + cur[v];
      cur[v] += start;
    }
    __syncthreads();
    stream_runs<K, Map, kBinNW>(a, map, start, E, bucket0, nb, cur, rest);
  }
}

// Bins above kHugeSeg edges, split into segments of kHugeSeg edges (rows).
// 1. every row's local-bucket counts, one CTA per row
template <typename K, typename Map>
__global__ void __launch_bounds__(kBinNW * 32, 1) k_huge_count(BinArgs<K> a, const uint32_t* __restrict__ rows,
                                                             const uint32_t* __restrict__ rowdesc,
                                                             uint32_t* __restrict__ rowcnt, Map map) {
  extern __shared__ __align__(16) uint32_t hcur[];
  map.init();
  const uint32_t nbmax = 1u << a.s;
  const uint32_t R = *rows;
  for (uint32_t r = blockIdx.x; r < R; r += gridDim.x) {
    const uint32_t b = rowdesc[2 * r], sg = rowdesc[2 * r + 1];
    const uint32_t off = sg * kHugeSeg;
    const uint32_t len = min(kHugeSeg, a.T[b] - off);
    const uint64_t bucket0 = (uint64_t)b << a.s;
    const uint32_t nb = (uint32_t)min((uint64_t)nbmax, a.V - bucket0);
    count_local(a, map, a.BS[b] + off, len, bucket0, nb, hcur);
    for (uint32_t v = threadIdx.x; v < nb; v += blockDim.x) rowcnt[(uint64_t)r * nbmax + v] = hcur[v];
    __syncthreads();
  }
}

// 2. per huge bin: bucket totals over its rows, exclusive scan -> the bin's
//    offsets; every row's counts become its absolute CSR cursors
template <typename K>
__global__ void __launch_bounds__(1024) k_huge_scan(BinArgs<K> a, const uint32_t* __restrict__ hcount,
                                                    const uint32_t* __restrict__ hlist, uint32_t* __restrict__ rowcnt) {
  extern __shared__ __align__(16) uint32_t tot[];
  __shared__ uint32_t wsum[32];
  const uint32_t nbmax = 1u << a.s;
  const uint32_t H = *hcount;
  for (uint32_t k = blockIdx.x; k < H; k += gridDim.x) {
    const uint32_t b = hlist[3 * k], r0 = hlist[3 * k + 1], nr = hlist[3 * k + 2];
    const uint64_t bucket0 = (uint64_t)b << a.s;
    const uint32_t nb = (uint32_t)min((uint64_t)nbmax, a.V - bucket0);
    const uint32_t start = a.BS[b];
    for (uint32_t v = threadIdx.x; v < nb; v += blockDim.x) {
      uint32_t run = 0;
      for (uint32_t r = 0; r < nr; ++r) {
        uint32_t* p = rowcnt + (uint64_t)(r0 + r) * nbmax + v;
        const uint32_t c = *p;
        *p = run;
        run += c;
      }
      tot[v] = run;
    }
    __syncthreads();
    block_excl_scan_smem(tot, (int)nb, wsum);
    for (uint32_t v = threadIdx.x; v < nb; v += blockDim.x) {
      const uint32_t first = start + tot[v];
      a.offsets[bucket0 + v] = a.pos_base + first;
      for (uint32_t r = 0; r < nr; ++r) rowcnt[(uint64_t)(r0 + r) * nbmax + v] += first;
    }
    __syncthreads();
  }
}

// 3. every row streams its segment to its cursors, one CTA per row
template <typename K, typename Map>
__global__ void __launch_bounds__(kBinNW * 32, 1) k_huge_scatter(BinArgs<K> a, const uint32_t* __restrict__ rows,
                                                               const uint32_t* __restrict__ rowdesc,
                                                               const uint32_t* __restrict__ rowcnt, Map map) {
  extern __shared__ __align__(16) uint8_t smem[];
  map.init();
  const uint32_t nbmax = 1u << a.s;
  uint32_t* cur = (uint32_t*)smem;
  uint8_t* rest = smem + align_up((size_t)nbmax * 4, 16);
  const uint32_t R = *rows;
  for (uint32_t r = blockIdx.x; r < R; r += gridDim.x) {
    const uint32_t b = rowdesc[2 * r], sg = rowdesc[2 * r + 1];
    const uint32_t off = sg * kHugeSeg;
    const uint32_t len = min(kHugeSeg, a.T[b] - off);
    const uint64_t bucket0 = (uint64_t)b << a.s;
    const uint32_t nb = (uint32_t)min((uint64_t)nbmax, a.V - bucket0);
    for (uint32_t v = threadIdx.x; v < nb; v += blockDim.x) cur[v] = rowcnt[(uint64_t)r * nbmax + v];
    __syncthreads();
    stream_runs<K, Map, kBinNW>(a, map, a.BS[b] + off, len, bucket0, nb, cur, rest);
  }
}

// ===========================================================================
// V1 (Alg. 1): global histogram with atomics, prefix sum, atomic scatter.
// Atomics leave the order inside a bucket arbitrary; a fix-up then sorts
// every bucket by input position (the ids hold positions until the end).
// ===========================================================================
template <typename K, typename Map>
__global__ void k_v1_count(const K* __restrict__ keys, uint64_t n, uint32_t* __restrict__ counts, Map map) {
  map.init();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[map(keys[i])], 1u);
}

template <typename K, typename Map>
__global__ void k_v1_scatter(const K* __restrict__ keys, uint64_t n, const uint32_t* __restrict__ offsets,
                             uint32_t* __restrict__ cursor, K* __restrict__ csr_k,
                             uint32_t* __restrict__ csr_i, Map map) {
  map.init();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const K key = keys[i];
    const uint32_t b = map(key);
    const uint32_t pos = offsets[b] + atomicAdd(&cursor[b], 1u);
    csr_k[pos] = key;
    csr_i[pos] = (uint32_t)i;
  }
}

// Buckets of up to kV1Small edges: insertion sort by position, one thread per
// bucket.  Longer buckets go to a list for k_v1_fix_heavy.
template <typename K>
__global__ void k_v1_fix_small(const uint32_t* __restrict__ offsets, uint64_t V, K* csr_k, uint32_t* csr_i,
                               uint32_t* heavy_list, uint32_t* heavy_count) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = offsets[v], e = offsets[v + 1];
    const uint32_t c = e - s;
    if (c <= 1) continue;
    if (c > kV1Small) {
      heavy_list[atomicAdd(heavy_count, 1u)] = (uint32_t)v;
      continue;
    }
    for (uint32_t i = s + 1; i < e; ++i) {
      const uint32_t p = csr_i[i];
      const K k = csr_k[i];
      uint32_t j = i;
      while (j > s && csr_i[j - 1] > p) {
        csr_i[j] = csr_i[j - 1];
        csr_k[j] = csr_k[j - 1];
        --j;
      }
      csr_i[j] = p;
      csr_k[j] = k;
    }
  }
}

// Heavy buckets: one CTA per bucket, least-significant-digit radix sort of
// the (position, key) pairs by position, 8 bits per pass.  Segments that fit
// shared memory are sorted in place there; longer ones stream through a
// global temporary, one stable tile partition at a time.
template <typename K>
__global__ void __launch_bounds__(kV1HeavyNW * 32) k_v1_fix_heavy(const uint32_t* __restrict__ offsets,
                                                                 const uint32_t* heavy_list,
                                                                 const uint32_t* heavy_count, K* csr_k,
                                                                 uint32_t* csr_i, K* tmp_k, uint32_t* tmp_i,
                                                                 uint32_t nbits) {
  constexpr int NW = kV1HeavyNW, IPT = kV1HeavyIPT;
  constexpr uint32_t TILE = NW * 32 * IPT;
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* sp = smem;
  K* sk = (K*)sp; sp += TILE * sizeof(K);
  uint32_t* sv = (uint32_t*)sp; sp += TILE * 4;
  uint32_t* wc = (uint32_t*)sp; sp += rank_words<NW>() * 4;
  uint32_t* dstart = (uint32_t*)sp; sp += 256 * 4;
  uint32_t* cursor = (uint32_t*)sp; sp += 256 * 4;
  uint8_t* sd = sp; sp += TILE;
  sp = (uint8_t*)(((uintptr_t)sp + 15) & ~(uintptr_t)15);
  uint32_t* wsum = (uint32_t*)sp;
  const uint32_t seg0 = (threadIdx.x >> 5) * (32u * IPT), lane = lane_id();
  const uint32_t nh = *heavy_count;
  for (uint32_t h = blockIdx.x; h < nh; h += gridDim.x) {
    const uint32_t v = heavy_list[h];
    const uint32_t s = offsets[v], c = offsets[v + 1] - s;
    K* src_k = csr_k + s;
    uint32_t* src_i = csr_i + s;
    K* dst_k = tmp_k + s;
    uint32_t* dst_i = tmp_i + s;
    for (uint32_t shift = 0; shift < nbits; shift += 8) {
      // count digits of this pass
      for (int d = threadIdx.x; d < 256; d += blockDim.x) cursor[d] = 0;
      __syncthreads();
      for (uint32_t e = threadIdx.x; e < c; e += blockDim.x) atomicAdd(&cursor[(src_i[e] >> shift) & 255u], 1u);
      __syncthreads();
      block_excl_scan_smem(cursor, 256, wsum);
      for (uint32_t t0 = 0; t0 < c; t0 += TILE) {
        const uint32_t cnt = min(TILE, c - t0);
        K key[IPT];
        uint32_t val[IPT], dig[IPT];
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
          const uint32_t idx = seg0 + (uint32_t)r * 32u + lane;
          if (idx < cnt) {
            key[r] = src_k[t0 + idx];
            val[r] = src_i[t0 + idx];
            dig[r] = (val[r] >> shift) & 255u;
          } else {
            key[r] = 0; val[r] = 0; dig[r] = 0;
          }
        }
        tile_partition_out<K, IPT, NW>(key, val, dig, cnt, 256, sk, sv, sd, wc, dstart, cursor, wsum,
                                       dst_k, dst_i);
      }
      K* tk = src_k; src_k = dst_k; dst_k = tk;
      uint32_t* tv = src_i; src_i = dst_i; dst_i = tv;
    }
    if (src_k != csr_k + s) {  // odd number of passes: copy back
      for (uint32_t e = threadIdx.x; e < c; e += blockDim.x) {
        csr_k[s + e] = src_k[e];
        csr_i[s + e] = src_i[e];
      }
    }
    __syncthreads();
  }
}

__global__ void k_v1_ids(uint32_t* __restrict__ csr_i, const uint32_t* __restrict__ ids, uint64_t n) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x)
    csr_i[j] = ids[csr_i[j]];
}

// ===========================================================================
// Host drivers
// ===========================================================================
// The largest dynamic shared memory each kernel was asked for, per device.
static std::mutex g_smem_mu;
static std::unordered_map<const void*, size_t> g_smem_max[64];

template <typename F>
static void set_smem_once(F* kernel, size_t bytes) {
  // The attribute belongs to the kernel, process-wide, and a launch needs it
  // at least as large as its own request.  It is raised to the largest
  // request so far and never lowered, so a call on another host thread that
  // asked for more is not cut short; it is set on every call (cheap), so it
  // holds again after a device reset.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lk(g_smem_mu);
  size_t& top = g_smem_max[dev][(const void*)kernel];
  if (bytes > top) top = bytes;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)top);
}

template <typename K, typename Map>
hg_status build_v2(const Plan& p, const K* keys, const uint32_t* ids, uint32_t* offsets, K* csr_k,
                   uint32_t* csr_i, uint8_t* ws, cudaStream_t st, Map map, uint32_t pos_base,
                   bool positional_ids) {
  WsHeader* hdr = (WsHeader*)ws;
  uint32_t* status = &hdr->status;
  uint32_t* H = (uint32_t*)(ws + p.o_H);
  uint32_t* C = (uint32_t*)(ws + p.o_C);
  uint32_t* CT = (uint32_t*)(ws + p.o_CT);
  uint32_t* T = (uint32_t*)(ws + p.o_T);
  uint32_t* BS = (uint32_t*)(ws + p.o_BS);
  uint32_t* ovf = (uint32_t*)(ws + p.o_ovf);
  K* bk = (K*)(ws + p.o_bk);
  uint32_t* bi = (uint32_t*)(ws + p.o_bi);
  const DevInfo& di = dev_info();

  {
    const size_t sm = hist_stage_offset(p.nbins) + Map::kStageBytes;
    auto kern = k_hist<K, Map>;
    set_smem_once(kern, sm);
    {
      HG_TRACE("k_hist", st);
      kern<<<p.G, kHistThreads, sm, st>>>(keys, p.n, p.chunk, p.s, p.nbins, p.sshift, p.nsb, H, C, map,
                                          (uint32_t)Map::kStageBytes);
    }
  }
  {
    HG_TRACE("k_colscan", st);
    colscan_launch(H, p.G, p.nbins, T, st);
  }
  {
    HG_TRACE("k_colscan", st);
    colscan_launch(C, p.G, p.nsb, CT, st);
  }
  const bool two = p.sshift > 0;
  const BinCfg bc = bin_config(p, recompute_bucket<Map>::value);
  // Implicit ids are input positions, so the bin build can restore the
  // canonical order (ascending position in every bucket) from the ids
  // alone; then, unless k_scan_bins finds a bin too large for the
  // shared-memory bin build, the partitions may rank tiles in any order.
  // Both variants of each such kernel are launched; the one that does not
  // match the order mode returns at once.
  const bool any_order = ids == nullptr || positional_ids;
  // bins for the single-buffered bin-build launch, counted by k_scan_bins
  uint32_t* const wide_count = (uint32_t*)&hdr->counters[7];
  {
    HG_TRACE("k_scan_bins", st);
    HugeArgs h{};
    // below kHugeMinN keys every oversized bin goes to the one-CTA path (at
    // most a few million edges), which spares small builds three launches
    if (p.n >= kHugeMinN) h.list = (uint32_t*)(ws + p.o_hlist);
    h.count = (uint32_t*)&hdr->counters[0];
    h.rows = (uint32_t*)&hdr->counters[0] + 1;
    h.rowdesc = (uint32_t*)(ws + p.o_rowdesc);
    h.max_rows = p.max_rows;
    h.status = status;
    // bins above the largest the shared-memory bin build takes (the second,
    // single-buffered launch included) go to the oversized-bin kernels
    k_scan_bins<<<1, 1024, 0, st>>>(T, p.nbins, BS, std::max(bc.emax, bc.emax_wide), ovf, &hdr->ovf_count,
                                    offsets, p.V, pos_base + (uint32_t)p.n, h,
                                    any_order ? &hdr->order_mode : nullptr, bc.emax,
                                    bc.emax_wide > bc.emax ? wide_count : nullptr);
  }

  PartArgs<K> pa{};
  pa.in_k = keys;
  pa.in_i = ids;
  // With two partition passes, pass A's output lives in the caller's CSR
  // arrays until pass B has read it; with one pass it goes straight to the
  // workspace, so that no bin build reads and writes the same region.
  pa.out_k = two ? csr_k : bk;
  pa.out_i = two ? csr_i : bi;
  pa.n = p.n;
  pa.chunk = p.chunk;
  pa.G = p.G;
  pa.s = p.s;
  pa.sshift = p.sshift;
  pa.nbins = p.nbins;
  pa.nsb = p.nsb;
  pa.H = H;
  pa.C = C;
  pa.CT = CT;
  pa.BS = BS;
  pa.status = status;
  {
    pa.order = any_order ? &hdr->order_mode : nullptr;
    // the map's tables are staged only where they fit next to the tile
    auto launch = [&](auto kern, int ipt) {
      PartArgs<K> x = pa;
      const size_t own = part_smem_bytes(sizeof(K), ids != nullptr, ipt, false, kPartNW);
      x.stage_bytes = own + Map::kStageBytes <= (size_t)di.max_smem_optin ? (uint32_t)Map::kStageBytes : 0u;
      set_smem_once(kern, own + x.stage_bytes);
      kern<<<p.G, kPartNW * 32, own + x.stage_bytes, st>>>(x, map);
    };
    HG_TRACE("k_partition_A", st);
    // (a tile of carried ids takes the stable variant's tile size: the
    // larger one leaves no room for staging the ids)
    if (any_order && ids == nullptr)
      launch(k_partition<K, Map, false, part_ipt_keys<K, true>(), kPartNW, part_minb_keys<K, true>(), true>,
             part_ipt_keys<K, true>());
    else if (any_order)
      launch(k_partition<K, Map, false, part_ipt_keys<K, false>(), kPartNW, part_minb_keys<K, false>(), true>,
             part_ipt_keys<K, false>());
    launch(k_partition<K, Map, false, part_ipt_keys<K, false>(), kPartNW, part_minb_keys<K, false>(), false>,
           part_ipt_keys<K, false>());
  }
  if (two) {
    PartArgs<K> pb = pa;
    pb.in_k = csr_k;
    pb.in_i = csr_i;
    pb.out_k = bk;
    pb.out_i = bi;
    pb.stage_bytes = 0;  // (staging would cost pass B a resident CTA per SM)
    // ~32K edges per item: enough to amortise the per-item set-up
    const uint64_t per_chunk_sb = std::max<uint64_t>(1, p.n / ((uint64_t)p.G * p.nsb));
    pb.gg = (uint32_t)std::min<uint64_t>(p.G, std::max<uint64_t>(1, 32768 / per_chunk_sb));
    pb.ngroups = (p.G + pb.gg - 1) / pb.gg;
    const uint64_t items = (uint64_t)p.nsb * pb.ngroups;
    auto launch = [&](auto kern, int nw) {
      const size_t sm = part_smem_bytes(sizeof(K), true, kPartIPTB, true, nw);
      set_smem_once(kern, sm);
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nw * 32, sm);
      unsigned grid = (unsigned)std::min<uint64_t>(items, (uint64_t)std::max(1, per_sm) * di.sms);
      grid = (unsigned)std::max<uint64_t>(grid, (items + kMaxItemsPerCta - 1) / kMaxItemsPerCta);
      kern<<<grid, nw * 32, sm, st>>>(pb, map);
    };
    HG_TRACE("k_partition_B", st);
    if (any_order) launch(k_partition<K, Map, true, kPartIPTB, partb_nw<true>(), partb_minb<true>(), true>, partb_nw<true>());
    launch(k_partition<K, Map, true, kPartIPTB, partb_nw<false>(), partb_minb<false>(), false>, partb_nw<false>());
  }
  // A partition that could not be launched (say, a tile geometry built in at
  // compile time that needs more shared memory than a CTA may have) left the
  // bins unwritten: stop before the bin build reads them.
  if (cudaPeekAtLastError() != cudaSuccess) return last_launch_status();
  BinArgs<K> ba{};
  ba.in_k = bk;
  ba.in_i = bi;
  ba.csr_k = csr_k;
  ba.csr_i = csr_i;
  ba.offsets = offsets;
  ba.T = T;
  ba.BS = BS;
  ba.V = p.V;
  ba.nbins = p.nbins;
  ba.s = p.s;
  ba.emax = bc.emax;
  ba.pos_base = pos_base;
  ba.status = status;
  ba.nbuf = bc.nbuf;
  ba.order = any_order ? &hdr->order_mode : nullptr;
  {
    unsigned grid = (unsigned)std::min<uint64_t>(p.nbins, (uint64_t)di.sms * bc.per_sm);
    grid = std::max<unsigned>(grid, (p.nbins + kMaxBinsPerCta - 1) / kMaxBinsPerCta);
    HG_TRACE("k_binbuild", st);
    auto launch = [&](auto kern, auto kany, unsigned threads) {
      set_smem_once(kern, std::max(bc.smem, bc.smem_wide));
      set_smem_once(kany, std::max(bc.smem, bc.smem_wide));
      if (any_order) kany<<<grid, threads, bc.smem, st>>>(ba, map);
      kern<<<grid, threads, bc.smem, st>>>(ba, map);
      if (bc.emax_wide > bc.emax) {  // bins above emax, single-buffered
        BinArgs<K> bw = ba;
        bw.emin = bc.emax;
        bw.emax = bc.emax_wide;
        bw.nbuf = 1;
        bw.gate = wide_count;
        if (any_order) kany<<<grid, threads, bc.smem_wide, st>>>(bw, map);
        kern<<<grid, threads, bc.smem_wide, st>>>(bw, map);
      }
    };
    if (bc.per_sm == 2) {
      if (bc.lb)
        launch(k_binbuild<K, Map, 16, 2, true, false>, k_binbuild<K, Map, 16, 2, true, true>, 512);
      else
        launch(k_binbuild<K, Map, 16, 2, false, false>, k_binbuild<K, Map, 16, 2, false, true>, 512);
    } else if (bc.tpb == 512) {
      launch(k_binbuild<K, Map, 16, 1, true, false>, k_binbuild<K, Map, 16, 1, true, true>, 512);
    } else {
      launch(k_binbuild<K, Map, kBinNW, 1, true, false>, k_binbuild<K, Map, kBinNW, 1, true, true>, kBinNW * 32);
    }
  }
  {
    const size_t sm = big_smem_bytes(sizeof(K), 1u << p.s);
    auto kern = k_binbuild_big<K, Map>;
    set_smem_once(kern, sm);
    const unsigned grid = (unsigned)std::min<uint64_t>(p.nbins, (uint64_t)di.sms);
    {
      HG_TRACE("k_binbuild_big", st);
      kern<<<grid, kBinNW * 32, sm, st>>>(ba, ovf, &hdr->ovf_count, map);
    }
  }
  if (p.n >= kHugeMinN) {
    // bins above kHugeSeg edges (duplicates): several CTAs per bin
    const uint32_t nbmax = 1u << p.s;
    uint32_t* hcount = (uint32_t*)&hdr->counters[0];
    uint32_t* hrows = hcount + 1;
    const uint32_t* hlist = (const uint32_t*)(ws + p.o_hlist);
    const uint32_t* rowdesc = (const uint32_t*)(ws + p.o_rowdesc);
    uint32_t* rowcnt = (uint32_t*)(ws + p.o_rowcnt);
    const unsigned grid = (unsigned)std::min<uint64_t>(p.max_rows, (uint64_t)di.sms);
    const unsigned hgrid = (unsigned)std::min<uint64_t>(p.n / kHugeSeg + 1, (uint64_t)di.sms);
    HG_TRACE("k_binbuild_huge", st);
    auto kc = k_huge_count<K, Map>;
    set_smem_once(kc, (size_t)nbmax * 4);
    kc<<<grid, kBinNW * 32, (size_t)nbmax * 4, st>>>(ba, hrows, rowdesc, rowcnt, map);
    auto ks = k_huge_scan<K>;
    set_smem_once(ks, (size_t)nbmax * 4);
    ks<<<hgrid, 1024, (size_t)nbmax * 4, st>>>(ba, hcount, hlist, rowcnt);
    const size_t sm = big_smem_bytes(sizeof(K), nbmax);
    auto kx = k_huge_scatter<K, Map>;
    set_smem_once(kx, sm);
    kx<<<grid, kBinNW * 32, sm, st>>>(ba, hrows, rowdesc, rowcnt, map);
  }
  return last_launch_status();
}

bool v2_plan_fits(const Plan& p) {
  if (p.n == 0) return true;
  const double mean = (double)p.n * (double)(1ull << p.s) / (double)p.V;
  return mean + 5.0 * std::sqrt(mean) + 16.0 <= (double)p.emax;
}

bool make_slab_plan(const hg_config* cfg, uint64_t n, SlabPlan* p) {
  if (cfg->bin_shift != 0 || n == 0) return false;  // an explicit bin size asks for one two-level plan
  const DevInfo& di = dev_info();
  p->kb = cfg->key_type == HG_KEY_U64 ? 8 : 4;
  p->n = n;
  p->V = cfg->num_buckets;
  const double emax = p->kb == 4 ? kBinEmaxU32 : kBinEmaxU64;
  const double alpha = (double)n / (double)p->V;
  // largest bins (2^s buckets) that still fit shared memory at this load
  int s_fit = -1;
  for (int s = 0; s <= (int)kMaxBinShift; ++s) {
    const double mean = alpha * (double)(1ull << s);
    if (mean + 5.0 * std::sqrt(mean) + 16.0 <= emax) s_fit = s;
  }
  if (s_fit < 0) return false;  // a bin of one bucket would overflow: no relabeling helps
  p->Ls = (uint32_t)s_fit + kMaxBinsLog2;
  const uint64_t S = (p->V + (1ull << p->Ls) - 1) >> p->Ls;
  if (S < 2 || S > 256) return false;
  p->S = (uint32_t)S;
  const int sms = std::max(di.sms, 1);
  uint64_t chunk = std::max<uint64_t>(kPartTile, (n + 2 * sms - 1) / (2 * sms));
  chunk = (chunk + 15) / 16 * 16;
  p->chunk = chunk;
  p->G = (uint32_t)std::max<uint64_t>(1, (n + chunk - 1) / chunk);
  hg_config cs = *cfg;
  cs.num_buckets = std::min<uint64_t>(1ull << p->Ls, p->V);
  cs.bin_shift = 0;
  if (!make_plan_v2(&cs, n, &p->sub)) return false;
  size_t o = sizeof(WsHeader);
  p->o_H = o;   o = align_up(o + (size_t)p->G * p->S * 4);
  p->o_C = o;   o = align_up(o + (size_t)p->G * p->S * 4);
  p->o_CT = o;  o = align_up(o + (size_t)p->S * 4);
  p->o_T = o;   o = align_up(o + (size_t)p->S * 4);
  p->o_BS = o;  o = align_up(o + ((size_t)p->S + 1) * 4);
  p->o_ovf = o; o = align_up(o + (size_t)p->S * 4 + 16);
  p->o_k = o;   o = align_up(o + ((size_t)n + 16) * p->kb);
  p->o_i = o;   o = align_up(o + ((size_t)n + 16) * 4);
  p->o_sub = o; o = align_up(o + p->sub.total);
  p->total = o;
  return true;
}

__global__ void k_fill_u32(uint32_t* __restrict__ a, uint64_t n, uint32_t v) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// A slab build records its device errors in its own workspace header; they
// are carried over to the caller's.
__global__ void k_carry_status(const uint32_t* __restrict__ from, uint32_t* to) {
  if (*from) set_status(to, *from);
}

template <typename K, typename Map>
hg_status build_slabs(const hg_config* cfg, const SlabPlan& p, const K* keys, const uint32_t* ids,
                      uint32_t* offsets, K* csr_k, uint32_t* csr_i, uint8_t* ws, cudaStream_t st, Map map) {
  WsHeader* hdr = (WsHeader*)ws;
  uint32_t* H = (uint32_t*)(ws + p.o_H);
  uint32_t* C = (uint32_t*)(ws + p.o_C);
  uint32_t* CT = (uint32_t*)(ws + p.o_CT);
  uint32_t* T = (uint32_t*)(ws + p.o_T);
  uint32_t* BS = (uint32_t*)(ws + p.o_BS);
  uint32_t* ovf = (uint32_t*)(ws + p.o_ovf);
  K* lk = (K*)(ws + p.o_k);
  uint32_t* li = (uint32_t*)(ws + p.o_i);
  uint8_t* sub = ws + p.o_sub;
  const DevInfo& di = dev_info();
  // 1. slab of every key (bucket >> Ls), counted per input chunk
  {
    const size_t sm = hist_stage_offset(p.S) + Map::kStageBytes;
    auto kern = k_hist<K, Map>;
    set_smem_once(kern, sm);
    HG_TRACE("k_hist_slab", st);
    kern<<<p.G, kHistThreads, sm, st>>>(keys, p.n, p.chunk, p.Ls, p.S, 0, p.S, H, C, map,
                                        (uint32_t)Map::kStageBytes);
    colscan_launch(H, p.G, p.S, T, st);
    colscan_launch(C, p.G, p.S, CT, st);
    k_scan_bins<<<1, 1024, 0, st>>>(T, p.S, BS, 0xffffffffu, ovf, &hdr->ovf_count, ovf + p.S, 0, (uint32_t)p.n,
                                    HugeArgs{}, nullptr);
  }
  // 2. stable partition by slab: each slab keeps its keys in input order,
  //    with their ids (the input positions when none are given)
  {
    PartArgs<K> pa{};
    pa.in_k = keys;
    pa.in_i = ids;
    pa.out_k = lk;
    pa.out_i = li;
    pa.n = p.n;
    pa.chunk = p.chunk;
    pa.G = p.G;
    pa.s = p.Ls;
    pa.sshift = 0;
    pa.nbins = p.S;
    pa.nsb = p.S;
    pa.H = H;
    pa.C = C;
    pa.CT = CT;
    pa.BS = BS;
    pa.status = &hdr->status;
    pa.order = nullptr;
    constexpr int ipt = part_ipt_keys<K, false>();
    auto kern = k_partition<K, Map, false, ipt, kPartNW, part_minb_keys<K, false>(), false>;
    const size_t own = part_smem_bytes(sizeof(K), ids != nullptr, ipt, false, kPartNW);
    pa.stage_bytes = own + Map::kStageBytes <= (size_t)di.max_smem_optin ? (uint32_t)Map::kStageBytes : 0u;
    set_smem_once(kern, own + pa.stage_bytes);
    HG_TRACE("k_partition_slab", st);
    kern<<<p.G, kPartNW * 32, own + pa.stage_bytes, st>>>(pa, map);
  }
  if (cudaPeekAtLastError() != cudaSuccess) return last_launch_status();  // partition not launched
  // 3. slab sizes to the host, then one two-level build per slab
  uint32_t hT[256];
  if (cudaMemcpyAsync(hT, T, (size_t)p.S * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HG_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HG_ERR_CUDA;
  uint64_t start = 0;
  for (uint32_t sl = 0; sl < p.S; ++sl) {
    const uint64_t b0 = (uint64_t)sl << p.Ls;
    const uint64_t Vs = std::min<uint64_t>(1ull << p.Ls, p.V - b0);
    const uint64_t ns = hT[sl];
    if (ns == 0) {
      k_fill_u32<<<(unsigned)std::min<uint64_t>((Vs + 256) / 256, (uint64_t)di.sms * 8), 256, 0, st>>>(
          offsets + b0, Vs + 1, (uint32_t)start);
      continue;
    }
    hg_config cs = *cfg;
    cs.num_buckets = Vs;
    cs.bin_shift = 0;
    Plan ps{};
    if (!make_plan_v2(&cs, ns, &ps) || ps.total > p.sub.total) return HG_ERR_UNSUPPORTED;
    Map ms = map;
    ms.slab_base = (uint32_t)b0;
    if (cudaMemsetAsync(sub, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
    hg_status rc = build_v2<K, Map>(ps, lk + start, li + start, offsets + b0, csr_k + start, csr_i + start, sub, st,
                                    ms, (uint32_t)start, ids == nullptr);
    if (rc != HG_OK) return rc;
    k_carry_status<<<1, 1, 0, st>>>(&((WsHeader*)sub)->status, &hdr->status);
    start += ns;
  }
  return last_launch_status();
}

size_t v1_workspace_bytes(int kb, uint64_t n, uint64_t V) {
  size_t o = sizeof(WsHeader);
  o = align_up(o + (size_t)V * 4);                  // cursors
  o = align_up(o + scan_workspace_bytes<uint32_t>(V + 1));    // scan partials
  o = align_up(o + (size_t)V * 4);                  // heavy list
  o = align_up(o + ((size_t)n + 16) * kb);          // temp keys
  o = align_up(o + ((size_t)n + 16) * 4);           // temp positions
  return o;
}

template <typename K, typename Map>
hg_status build_v1(uint64_t n, uint64_t V, const K* keys, const uint32_t* ids, uint32_t* offsets, K* csr_k,
                   uint32_t* csr_i, uint8_t* ws, cudaStream_t st, Map map) {
  WsHeader* hdr = (WsHeader*)ws;
  size_t o = sizeof(WsHeader);
  uint32_t* cursor = (uint32_t*)(ws + o); o = align_up(o + (size_t)V * 4);
  uint32_t* part = (uint32_t*)(ws + o);   o = align_up(o + scan_workspace_bytes<uint32_t>(V + 1));
  uint32_t* heavy = (uint32_t*)(ws + o);  o = align_up(o + (size_t)V * 4);
  K* tk = (K*)(ws + o);                   o = align_up(o + ((size_t)n + 16) * sizeof(K));
  uint32_t* ti = (uint32_t*)(ws + o);
  const int sms = dev_info().sms;
  const unsigned grid = (unsigned)std::max(1, sms * 8);
  cudaMemsetAsync(offsets, 0, (size_t)(V + 1) * 4, st);
  cudaMemsetAsync(cursor, 0, (size_t)V * 4, st);
  {
    HG_TRACE("k_v1_count", st);
    k_v1_count<K, Map><<<grid, 256, 0, st>>>(keys, n, offsets, map);
  }
  hg_status rc = device_excl_scan<uint32_t>(offsets, V + 1, part, st);
  if (rc != HG_OK) return rc;
  {
    HG_TRACE("k_v1_scatter", st);
    k_v1_scatter<K, Map><<<grid, 256, 0, st>>>(keys, n, offsets, cursor, csr_k, csr_i, map);
  }
  {
    HG_TRACE("k_v1_fix_small", st);
    k_v1_fix_small<K><<<grid, 256, 0, st>>>(offsets, V, csr_k, csr_i, heavy, &hdr->heavy_count);
  }
  uint32_t nbits = 8;
  while (nbits < 32 && (n - 1) >> nbits) nbits += 8;
  {
    const size_t sm = align_up((size_t)kV1HeavyNW * 32 * kV1HeavyIPT * (sizeof(K) + 5) +
                               (size_t)rank_words<kV1HeavyNW>() * 4 + 2 * 256 * 4, 16) + 32 * 4 + 64;
    auto kern = k_v1_fix_heavy<K>;
    set_smem_once(kern, sm);
    {
      HG_TRACE("k_v1_fix_heavy", st);
      kern<<<(unsigned)std::max(1, sms), kV1HeavyNW * 32, sm, st>>>(offsets, heavy, &hdr->heavy_count, csr_k,
                                                                    csr_i, tk, ti, nbits);
    }
  }
  if (ids) {
    HG_TRACE("k_v1_ids", st);
    k_v1_ids<<<grid, 256, 0, st>>>(csr_i, ids, n);
  }
  return last_launch_status();
}

// ===========================================================================
// Binned probe.  HashGraph-Probe-Standard answers each query with random
// reads into the table; on HBM every random 4-byte read costs a whole DRAM
// burst.  Here the queries are first partitioned by bucket range into ng
// groups (the build's histogram and partition kernels, applied to the
// queries), so that the group being probed touches one table slice small
// enough to stay in L2; the per-query counts are then put back in query
// order by a merge over the groups (inside a group the query positions
// ascend from one block of kQueryBlock positions to the next).
// ===========================================================================
// Counts back to query order when the positions inside every group come in
// long ascending runs (batched tables: a table's queries fall into one or two
// groups): a plain in-order scatter, coalesced along each run.
__global__ void k_scatter_counts(const uint32_t* __restrict__ Qi, const uint32_t* __restrict__ Qc, uint64_t Q,
                                 uint32_t* __restrict__ counts) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < Q; j += (uint64_t)gridDim.x * blockDim.x)
    counts[__ldcs(Qi + j)] = __ldcs(Qc + j);
}

#ifndef HG_UNPERMUTE_TILE
#define HG_UNPERMUTE_TILE 32768
#endif
constexpr int kUnpermuteThreads = 1024;
constexpr uint32_t kUnpermuteTile = HG_UNPERMUTE_TILE;  // outputs per merge tile (shared memory: 4 B each)

// Every warp merges the groups warp, warp + 32, ... (GPW of them); per round
// it loads UNR runs of 32 (position, count) pairs of each of its groups, so
// GPW * UNR pairs per lane are in flight (eight for any number of groups).
template <int GPW, int UNR>
__global__ void __launch_bounds__(kUnpermuteThreads) k_unpermute(const uint32_t* __restrict__ Qi,
                                                                 const uint32_t* __restrict__ Qc,
                                                                 const uint32_t* __restrict__ GS, uint32_t ng,
                                                                 uint64_t Q, uint64_t span,
                                                                 uint32_t* __restrict__ counts) {
  __shared__ uint32_t cur[256], gend[256];
  extern __shared__ uint32_t out_s[];  // kUnpermuteTile entries
  const uint64_t ob = (uint64_t)blockIdx.x * span;
  if (ob >= Q) return;
  const uint64_t oe = min(ob + span, Q);
  if (threadIdx.x < ng) {  // first query of each group at or after ob
    uint32_t lo = GS[threadIdx.x], hi = GS[threadIdx.x + 1];
    gend[threadIdx.x] = hi;
    while (lo < hi) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      if (Qi[mid] < ob) lo = mid + 1; else hi = mid;
    }
    cur[threadIdx.x] = lo;
  }
  __syncthreads();
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint64_t o0 = ob; o0 < oe; o0 += kUnpermuteTile) {
    const uint64_t o1 = min(o0 + (uint64_t)kUnpermuteTile, oe);
    uint32_t c[GPW], e[GPW];
    bool act[GPW];
#pragma unroll
    for (int k = 0; k < GPW; ++k) {
      const uint32_t g = warp + k * nw;
      act[k] = g < ng;
      c[k] = act[k] ? cur[g] : 0u;
      e[k] = act[k] ? gend[g] : 0u;
    }
    bool any = true;
    while (any) {
      uint32_t v[GPW][UNR], x[GPW][UNR];
#pragma unroll
      for (int k = 0; k < GPW; ++k) {
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          v[k][u] = 0xffffffffu;
          x[k][u] = 0u;
          const uint32_t j = c[k] + 32u * u + lane;
          if (act[k] && j < e[k]) {
            v[k][u] = __ldcs(Qi + j);
            x[k][u] = __ldcs(Qc + j);
          }
        }
      }
      any = false;
#pragma unroll
      for (int k = 0; k < GPW; ++k) {
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          if (!act[k]) break;  // warp-uniform
          const bool in = (uint64_t)v[k][u] < o1;
          if (in) out_s[v[k][u] - (uint32_t)o0] = x[k][u];
          const uint32_t n = __popc(__ballot_sync(kFull, in));
          c[k] += n;
          act[k] = n == 32;
        }
        any |= act[k];
      }
    }
#pragma unroll
    for (int k = 0; k < GPW; ++k) {
      const uint32_t g = warp + k * nw;
      if (g < ng && lane == 0) cur[g] = c[k];
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < (uint32_t)(o1 - o0); t += blockDim.x) __stcs(counts + o0 + t, out_s[t]);
    __syncthreads();
  }
}

// Counts back to query order, balanced over the warps whatever the group
// sizes (a skewed bucket map can put half of the queries into one group).
// For every output tile [o0, o1) the run of each group (its elements with
// positions in the tile, contiguous in its arrays) has the length the query
// partition recorded for the partition tiles that make up the output tile
// (TC: ng 16-bit counts per partition tile of ptile queries).  The runs,
// back to back, are split evenly over the warps; each lane keeps
// kUnpermuteUNR (position, count) pairs in flight and scatters them into the
// tile in shared memory, which is then written out coalesced.
constexpr int kUnpermuteUNR = 8;
__global__ void __launch_bounds__(kUnpermuteThreads) k_unpermute_bal(
    const uint32_t* __restrict__ Qi, const uint32_t* __restrict__ Qc, const uint32_t* __restrict__ GS, uint32_t ng,
    const uint16_t* __restrict__ TC, uint32_t ptile, uint64_t Q, uint64_t span, uint32_t* __restrict__ counts) {
  __shared__ uint32_t cur[256], run[256], rstart[257], wsum[32];
  extern __shared__ uint32_t out_s[];  // kUnpermuteTile entries
  const uint64_t ob = (uint64_t)blockIdx.x * span;
  if (ob >= Q) return;
  const uint64_t oe = min(ob + span, Q);
  if (threadIdx.x < ng) {  // first query of each group at or after ob
    uint32_t lo = GS[threadIdx.x], hi = GS[threadIdx.x + 1];
    while (lo < hi) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      if (Qi[mid] < ob) lo = mid + 1; else hi = mid;
    }
    cur[threadIdx.x] = lo;
  }
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint64_t o0 = ob; o0 < oe; o0 += kUnpermuteTile) {
    const uint64_t o1 = min(o0 + (uint64_t)kUnpermuteTile, oe);
    const uint32_t total = (uint32_t)(o1 - o0);
    // 1. every group's run in this tile, and where it starts among all runs
    uint32_t r = 0;
    if (threadIdx.x < ng)
      for (uint64_t t = o0 / ptile; t * ptile < o1; ++t) r += TC[t * ng + threadIdx.x];
    const uint32_t st = block_excl_scan<uint32_t>(r, wsum, (uint32_t*)nullptr);
    if (threadIdx.x < ng) {
      run[threadIdx.x] = r;
      rstart[threadIdx.x] = st;
    }
    if (threadIdx.x == 0) rstart[ng] = total;
    __syncthreads();
    // 2. the runs back to back, an equal slice per warp
    const uint32_t per = (total + nw - 1) / nw;
    const uint32_t x0 = min(warp * per, total), x1 = min(x0 + per, total);
    uint32_t g = 0;  // last group whose run starts at or before x0
    {
      uint32_t lo = 0, hi = ng;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (rstart[mid] <= x0) lo = mid; else hi = mid;
      }
      g = lo;
    }
    for (uint32_t xb = x0; xb < x1; xb += 32u * kUnpermuteUNR) {
      uint32_t v[kUnpermuteUNR], c[kUnpermuteUNR];
#pragma unroll
      for (int u = 0; u < kUnpermuteUNR; ++u) {
        const uint32_t x = xb + 32u * u + lane;
        v[u] = 0xffffffffu;
        c[u] = 0u;
        if (x < x1) {
          while (rstart[g + 1] <= x) ++g;
          const uint32_t j = cur[g] + (x - rstart[g]);
          v[u] = __ldcs(Qi + j);
          c[u] = __ldcs(Qc + j);
        }
      }
#pragma unroll
      for (int u = 0; u < kUnpermuteUNR; ++u)
        if (v[u] != 0xffffffffu) out_s[v[u] - (uint32_t)o0] = c[u];
    }
    __syncthreads();
    if (threadIdx.x < ng) cur[threadIdx.x] += run[threadIdx.x];
    for (uint32_t t = threadIdx.x; t < total; t += blockDim.x) __stcs(counts + o0 + t, out_s[t]);
    __syncthreads();
  }
}

// Queries are grouped by a partition that ranks each tile in any order (its
// tiles are whole blocks of kQueryBlock positions or the end of the
// queries).  A group's positions are therefore ascending from block to
// block, though not inside a block's run, and the merge works in output
// tiles made of whole blocks: within a group, every query of an earlier
// output tile precedes every query of a later one, which is all its
// cursors need.
constexpr uint64_t kQueryBlock = 4096;
static_assert(kQueryBlock % (kPartNW * 32 * part_ipt_queries<uint32_t>()) == 0 &&
                  kQueryBlock % (kPartNW * 32 * part_ipt_queries<uint64_t>()) == 0 && kUnpermuteTile % kQueryBlock == 0,
              "query blocks are whole partition tiles; merge tiles are whole blocks");

// Elements per tile of the query partition (whole tiles per query block).
static uint32_t query_tile(int kb) {
  return kb == 8 ? (uint32_t)(kPartNW * 32 * part_ipt_queries<uint64_t>())
                 : (uint32_t)(kPartNW * 32 * part_ipt_queries<uint32_t>());
}

#ifndef HG_PROBE_GROUP_BITS
#define HG_PROBE_GROUP_BITS 7  // log2 of the query groups (at most 8; 7 measured best at 2^28)
#endif
bool make_probe_plan(const hg_config* cfg, uint64_t table_n, uint64_t q, ProbePlan* p) {
  const DevInfo& di = dev_info();
  const int kb = cfg->key_type == HG_KEY_U64 ? 8 : 4;
  const uint64_t V = cfg->num_buckets;
  // 256 groups (fewer only for V < 256): a group's slice of the table stays
  // well below L2 up to 4 GB tables (a 2^28-key table gives 8 MB slices), and
  // with many groups every output tile of the merge draws on many of them,
  // which keeps its warps evenly loaded.
  (void)table_n;
  int sg = ceil_log2_u64(V) - HG_PROBE_GROUP_BITS;
  if (sg < 0) sg = 0;
  p->sg = (uint32_t)sg;
  p->ng = (uint32_t)(((V - 1) >> sg) + 1);
  if (p->ng > 256) return false;
  const int sms = std::max(di.sms, 1);
  // chunks are whole 4096-query blocks, so every partition tile lies in one
  // block (the merge below relies on it)
  uint64_t chunk = std::max<uint64_t>(kPartTile, (q + 2 * sms - 1) / (2 * sms));
  chunk = (chunk + kQueryBlock - 1) / kQueryBlock * kQueryBlock;
  p->chunk = chunk;
  p->G = (uint32_t)std::max<uint64_t>(1, (q + chunk - 1) / chunk);
  size_t o = sizeof(WsHeader);
  p->o_H = o;   o = align_up(o + (size_t)p->G * p->ng * 4);
  p->o_C = o;   o = align_up(o + (size_t)p->G * p->ng * 4);
  p->o_CT = o;  o = align_up(o + (size_t)p->ng * 4);
  p->o_GS = o;  o = align_up(o + ((size_t)p->ng + 1) * 4);
  p->o_ovf = o; o = align_up(o + (size_t)p->ng * 4 + 16);
  p->o_qk = o;  o = align_up(o + ((size_t)q + 16) * kb);
  p->o_qi = o;  o = align_up(o + ((size_t)q + 16) * 4);
  p->o_qc = o;  o = align_up(o + ((size_t)q + 16) * 4);
  p->ptile = query_tile(kb);
  p->o_tc = o;  o = align_up(o + ((size_t)(q + p->ptile - 1) / p->ptile) * p->ng * 2);
  p->total = o;
  return true;
}

template <typename K, typename Map>
hg_status probe_binned_impl(const ProbePlan& p, uint64_t V, const hg_table* t, const K* queries, uint64_t q,
                            uint32_t* counts, uint8_t* ws, cudaStream_t st, Map map) {
  WsHeader* hdr = (WsHeader*)ws;
  uint32_t* H = (uint32_t*)(ws + p.o_H);
  uint32_t* C = (uint32_t*)(ws + p.o_C);
  uint32_t* CT = (uint32_t*)(ws + p.o_CT);
  uint32_t* GS = (uint32_t*)(ws + p.o_GS);
  uint32_t* ovf = (uint32_t*)(ws + p.o_ovf);
  K* qk = (K*)(ws + p.o_qk);
  uint32_t* qi = (uint32_t*)(ws + p.o_qi);
  uint32_t* qc = (uint32_t*)(ws + p.o_qc);
  const DevInfo& di = dev_info();
  {
    const size_t sm = hist_stage_offset(p.ng) + Map::kStageBytes;
    auto kern = k_hist<K, Map>;
    set_smem_once(kern, sm);
    HG_TRACE("k_hist_Q", st);
    kern<<<p.G, kHistThreads, sm, st>>>(queries, q, p.chunk, p.sg, p.ng, 0, p.ng, H, C, map,
                                        (uint32_t)Map::kStageBytes);
  }
  {
    HG_TRACE("k_colscan_Q", st);
    colscan_launch(C, p.G, p.ng, CT, st);
  }
  {
    HG_TRACE("k_scan_Q", st);
    // no bin is "oversized" here; the closing-offset store goes to scratch
    k_scan_bins<<<1, 1024, 0, st>>>(CT, p.ng, GS, 0xffffffffu, ovf, &hdr->ovf_count, ovf + p.ng, 0,
                                    (uint32_t)q, HugeArgs{}, nullptr);
  }
  PartArgs<K> pa{};
  pa.in_k = queries;
  pa.in_i = nullptr;  // ids = query positions
  pa.out_k = qk;
  pa.out_i = qi;
  pa.n = q;
  pa.chunk = p.chunk;
  pa.G = p.G;
  pa.s = p.sg;
  pa.sshift = 0;
  pa.nbins = p.ng;
  pa.nsb = p.ng;
  pa.H = H;
  pa.C = C;
  pa.CT = CT;
  pa.BS = GS;
  pa.status = &hdr->status;
  pa.tile_counts = Map::kSkewed ? (uint16_t*)(ws + p.o_tc) : nullptr;
  {
    const size_t own = part_smem_bytes(sizeof(K), false, part_ipt_queries<K>(), false, kPartNW);
    pa.stage_bytes = own + Map::kStageBytes <= (size_t)di.max_smem_optin ? (uint32_t)Map::kStageBytes : 0u;
    const size_t sm = own + pa.stage_bytes;
    auto kern = k_partition<K, Map, false, part_ipt_queries<K>(), kPartNW, kPartMinBlocksQ, true>;
    set_smem_once(kern, sm);
    HG_TRACE("k_partition_Q", st);
    kern<<<p.G, kPartNW * 32, sm, st>>>(pa, map);
  }
  // the probe and the merge index by the grouped positions: none may run on
  // a query partition that was not launched
  if (cudaPeekAtLastError() != cudaSuccess) return last_launch_status();
  hg_status rc = probe_launch<K, Map>(qk, q, t->d_offsets, (const K*)t->d_keys, qc, V, st, map,
                                      Map::kNeedsPos ? qi : nullptr);
  if (rc != HG_OK) return rc;
  {
    // every CTA merges a span of at least 4096 outputs (in tiles of up to
    // kUnpermuteTile), so small batches still spread over the SMs
    const uint64_t blocks = (q + kQueryBlock - 1) / kQueryBlock;
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(blocks, (uint64_t)2 * di.sms));
    const uint64_t span = (blocks + grid - 1) / grid * kQueryBlock;  // whole blocks
    HG_TRACE("k_unpermute", st);
    if (Map::kNeedsPos)
      k_scatter_counts<<<(unsigned)std::min<uint64_t>((q + 255) / 256, (uint64_t)di.sms * 16), 256, 0, st>>>(
          qi, qc, q, counts);
    else {
      if (Map::kSkewed) {
        set_smem_once(k_unpermute_bal, (size_t)kUnpermuteTile * 4);
        k_unpermute_bal<<<(unsigned)grid, kUnpermuteThreads, (size_t)kUnpermuteTile * 4, st>>>(
            qi, qc, GS, p.ng, (const uint16_t*)(ws + p.o_tc), p.ptile, q, span, counts);
      } else {  // even groups: one warp per group merges faster
        auto launch = [&](auto kern) {
          set_smem_once(kern, (size_t)kUnpermuteTile * 4);
          kern<<<(unsigned)grid, kUnpermuteThreads, (size_t)kUnpermuteTile * 4, st>>>(qi, qc, GS, p.ng, q, span,
                                                                                      counts);
        };
        if (p.ng <= 32) launch(k_unpermute<1, 8>);
        else if (p.ng <= 64) launch(k_unpermute<2, 4>);
        else if (p.ng <= 128) launch(k_unpermute<4, 2>);
        else launch(k_unpermute<8, 1>);
      }
    }
  }
  return last_launch_status();
}

bool make_slab_probe_plan(const hg_config* cfg, uint64_t table_n, uint64_t q, SlabProbePlan* p) {
  const uint64_t V = cfg->num_buckets;
  if (V <= (1ull << kSlabProbeLog2) || q == 0) return false;
  const DevInfo& di = dev_info();
  const int kb = cfg->key_type == HG_KEY_U64 ? 8 : 4;
  p->V = V;
  p->q = q;
  p->Ls = kSlabProbeLog2;
  p->S = (uint32_t)((V + (1ull << p->Ls) - 1) >> p->Ls);
  const int sms = std::max(di.sms, 1);
  // chunks are whole blocks of queries, as in the binned probe (its merge
  // relies on it)
  uint64_t chunk = std::max<uint64_t>(kPartTile, (q + 2 * sms - 1) / (2 * sms));
  chunk = (chunk + kQueryBlock - 1) / kQueryBlock * kQueryBlock;
  p->chunk = chunk;
  p->G = (uint32_t)std::max<uint64_t>(1, (q + chunk - 1) / chunk);
  hg_config cs = *cfg;
  cs.num_buckets = 1ull << p->Ls;
  if (!make_probe_plan(&cs, table_n, q, &p->sub)) return false;
  size_t o = sizeof(WsHeader);
  p->o_H = o;   o = align_up(o + (size_t)p->G * p->S * 4);
  p->o_C = o;   o = align_up(o + (size_t)p->G * p->S * 4);
  p->o_CT = o;  o = align_up(o + (size_t)p->S * 4);
  p->o_GS = o;  o = align_up(o + ((size_t)p->S + 1) * 4);
  p->o_ovf = o; o = align_up(o + (size_t)p->S * 4 + 16);
  p->o_qk = o;  o = align_up(o + ((size_t)q + 16) * kb);
  p->o_qi = o;  o = align_up(o + ((size_t)q + 16) * 4);
  p->o_qc = o;  o = align_up(o + ((size_t)q + 16) * 4);
  p->ptile = query_tile(kb);
  p->o_tc = o;  o = align_up(o + ((size_t)(q + p->ptile - 1) / p->ptile) * p->S * 2);
  p->o_sub = o; o = align_up(o + p->sub.total);
  p->total = o;
  return true;
}

template <typename K, typename Map>
hg_status probe_slabs(const hg_config* cfg, const SlabProbePlan& p, const hg_table* t, const K* queries,
                      uint64_t q, uint32_t* counts, uint8_t* ws, cudaStream_t st, Map map) {
  WsHeader* hdr = (WsHeader*)ws;
  uint32_t* H = (uint32_t*)(ws + p.o_H);
  uint32_t* C = (uint32_t*)(ws + p.o_C);
  uint32_t* CT = (uint32_t*)(ws + p.o_CT);
  uint32_t* GS = (uint32_t*)(ws + p.o_GS);
  uint32_t* ovf = (uint32_t*)(ws + p.o_ovf);
  K* qk = (K*)(ws + p.o_qk);
  uint32_t* qi = (uint32_t*)(ws + p.o_qi);
  uint32_t* qc = (uint32_t*)(ws + p.o_qc);
  uint8_t* sub = ws + p.o_sub;
  const DevInfo& di = dev_info();
  // 1. queries grouped by slab (bucket >> Ls), in whole query blocks
  {
    const size_t sm = hist_stage_offset(p.S) + Map::kStageBytes;
    auto kern = k_hist<K, Map>;
    set_smem_once(kern, sm);
    HG_TRACE("k_hist_Q", st);
    kern<<<p.G, kHistThreads, sm, st>>>(queries, q, p.chunk, p.Ls, p.S, 0, p.S, H, C, map,
                                        (uint32_t)Map::kStageBytes);
    colscan_launch(C, p.G, p.S, CT, st);
    k_scan_bins<<<1, 1024, 0, st>>>(CT, p.S, GS, 0xffffffffu, ovf, &hdr->ovf_count, ovf + p.S, 0, (uint32_t)q,
                                    HugeArgs{}, nullptr);
  }
  {
    PartArgs<K> pa{};
    pa.in_k = queries;
    pa.in_i = nullptr;  // ids = query positions
    pa.out_k = qk;
    pa.out_i = qi;
    pa.n = q;
    pa.chunk = p.chunk;
    pa.G = p.G;
    pa.s = p.Ls;
    pa.sshift = 0;
    pa.nbins = p.S;
    pa.nsb = p.S;
    pa.H = H;
    pa.C = C;
    pa.CT = CT;
    pa.BS = GS;
    pa.status = &hdr->status;
    pa.tile_counts = Map::kSkewed ? (uint16_t*)(ws + p.o_tc) : nullptr;
    const size_t own = part_smem_bytes(sizeof(K), false, part_ipt_queries<K>(), false, kPartNW);
    pa.stage_bytes = own + Map::kStageBytes <= (size_t)di.max_smem_optin ? (uint32_t)Map::kStageBytes : 0u;
    auto kern = k_partition<K, Map, false, part_ipt_queries<K>(), kPartNW, kPartMinBlocksQ, true>;
    set_smem_once(kern, own + pa.stage_bytes);
    HG_TRACE("k_partition_Q", st);
    kern<<<p.G, kPartNW * 32, own + pa.stage_bytes, st>>>(pa, map);
  }
  if (cudaPeekAtLastError() != cudaSuccess) return last_launch_status();  // partition not launched
  // 2. slab query counts to the host, then the binned probe of every slab
  uint32_t hGS[257];
  if (cudaMemcpyAsync(hGS, GS, ((size_t)p.S + 1) * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HG_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HG_ERR_CUDA;
  for (uint32_t sl = 0; sl < p.S; ++sl) {
    const uint64_t qs = hGS[sl + 1] - hGS[sl];
    if (qs == 0) continue;
    const uint64_t b0 = (uint64_t)sl << p.Ls;
    hg_config cs = *cfg;
    cs.num_buckets = std::min<uint64_t>(1ull << p.Ls, p.V - b0);
    ProbePlan ps{};
    if (!make_probe_plan(&cs, t->n, qs, &ps) || ps.total > p.sub.total) return HG_ERR_UNSUPPORTED;
    hg_table ts = *t;
    ts.d_offsets = t->d_offsets + b0;  // offsets are positions in the whole table's key array
    Map ms = map;
    ms.slab_base = (uint32_t)b0;
    if (cudaMemsetAsync(sub, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
    hg_status rc = probe_binned_impl<K, Map>(ps, cs.num_buckets, &ts, qk + hGS[sl], qs, qc + hGS[sl], sub, st, ms);
    if (rc != HG_OK) return rc;
    k_carry_status<<<1, 1, 0, st>>>(&((WsHeader*)sub)->status, &hdr->status);
  }
  // 3. counts back to query order
  {
    const uint64_t blocks = (q + kQueryBlock - 1) / kQueryBlock;
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(blocks, (uint64_t)2 * di.sms));
    const uint64_t span = (blocks + grid - 1) / grid * kQueryBlock;
    HG_TRACE("k_unpermute", st);
    if (Map::kSkewed) {
      set_smem_once(k_unpermute_bal, (size_t)kUnpermuteTile * 4);
      k_unpermute_bal<<<(unsigned)grid, kUnpermuteThreads, (size_t)kUnpermuteTile * 4, st>>>(
          qi, qc, GS, p.S, (const uint16_t*)(ws + p.o_tc), p.ptile, q, span, counts);
    } else {
      auto kern = k_unpermute<1, 8>;
      set_smem_once(kern, (size_t)kUnpermuteTile * 4);
      kern<<<(unsigned)grid, kUnpermuteThreads, (size_t)kUnpermuteTile * 4, st>>>(qi, qc, GS, p.S, q, span, counts);
    }
  }
  return last_launch_status();
}

// ===========================================================================
// LSD radix sort of uint64 keys (used for the learned map's key sample):
// eight stable passes of the same histogram -> scan -> stable tile partition
// pipeline, with the "bucket" of a key being one of its bytes.
// ===========================================================================
struct RadixByteMap {
  static constexpr bool kNeedsPos = false;
  static constexpr bool kSkewed = false;
  static constexpr size_t kStageBytes = 0;
  uint32_t shift;
  __device__ __forceinline__ void init() {}
  __device__ __forceinline__ void stage(uint8_t*, size_t) {}
  template <typename K>
  __device__ __forceinline__ uint32_t operator()(K key, uint32_t /*pos*/ = 0) const {
    return (uint32_t)(((uint64_t)key >> shift) & 255u);
  }
  __device__ __forceinline__ uint32_t out_id(uint32_t id) const { return id; }
};

static void radix_layout(uint64_t n, uint64_t* chunk, uint32_t* G, size_t* o) {
  const int sms = std::max(dev_info().sms, 1);
  uint64_t c = std::max<uint64_t>(kPartTile, (n + 2 * sms - 1) / (2 * sms));
  c = (c + 15) / 16 * 16;
  *chunk = c;
  *G = (uint32_t)std::max<uint64_t>(1, (n + c - 1) / c);
  size_t off = sizeof(WsHeader);
  o[0] = off; off = align_up(off + (size_t)*G * 256 * 4);  // H
  o[1] = off; off = align_up(off + (size_t)*G * 256 * 4);  // C
  o[2] = off; off = align_up(off + 256 * 4);               // column totals
  o[3] = off; off = align_up(off + 257 * 4);               // digit starts
  o[4] = off; off = align_up(off + 256 * 4 + 16);          // unused list + scratch word
  o[5] = off; off = align_up(off + (n + 16) * 8);          // ping-pong keys
  o[6] = off; off = align_up(off + (n + 16) * 4);          // payload (positions, unused)
  o[7] = off;
}

size_t radix_sort_workspace_bytes(uint64_t n) {
  uint64_t chunk;
  uint32_t G;
  size_t o[8];
  radix_layout(n, &chunk, &G, o);
  return o[7];
}

hg_status radix_sort_u64(uint64_t* keys, uint64_t n, uint8_t* ws, cudaStream_t st) {
  if (n <= 1) return HG_OK;
  uint64_t chunk;
  uint32_t G;
  size_t o[8];
  radix_layout(n, &chunk, &G, o);
  WsHeader* hdr = (WsHeader*)ws;
  uint32_t* H = (uint32_t*)(ws + o[0]);
  uint32_t* C = (uint32_t*)(ws + o[1]);
  uint32_t* CT = (uint32_t*)(ws + o[2]);
  uint32_t* BS = (uint32_t*)(ws + o[3]);
  uint32_t* ovf = (uint32_t*)(ws + o[4]);
  uint64_t* tmp = (uint64_t*)(ws + o[5]);
  uint32_t* ids = (uint32_t*)(ws + o[6]);
  uint64_t* src = keys;
  uint64_t* dst = tmp;
  const size_t psm = part_smem_bytes(8, false, part_ipt_queries<uint64_t>(), false, kPartNW);
  auto kp = k_partition<uint64_t, RadixByteMap, false, part_ipt_queries<uint64_t>(), kPartNW, kPartMinBlocksQ, false>;
  set_smem_once(kp, psm);
  auto kh = k_hist<uint64_t, RadixByteMap>;
  const size_t hsm = hist_stage_offset(256);
  set_smem_once(kh, hsm);
  for (uint32_t pass = 0; pass < 8; ++pass) {
    RadixByteMap map{8 * pass};
    {
      HG_TRACE("k_radix_hist", st);
      kh<<<G, kHistThreads, hsm, st>>>(src, n, chunk, 0, 256, 0, 256, H, C, map, 0u);
    }
    {
      HG_TRACE("k_radix_scan", st);
      colscan_launch(C, G, 256, CT, st);
      k_scan_bins<<<1, 1024, 0, st>>>(CT, 256, BS, 0xffffffffu, ovf, &hdr->ovf_count, ovf + 256, 0, (uint32_t)n,
                                      HugeArgs{}, nullptr);
    }
    PartArgs<uint64_t> pa{};
    pa.in_k = src;
    pa.in_i = nullptr;
    pa.out_k = dst;
    pa.out_i = ids;
    pa.n = n;
    pa.chunk = chunk;
    pa.G = G;
    pa.s = 0;
    pa.sshift = 0;
    pa.nbins = 256;
    pa.nsb = 256;
    pa.H = H;
    pa.C = C;
    pa.CT = CT;
    pa.BS = BS;
    pa.status = &hdr->status;
    {
      HG_TRACE("k_radix_partition", st);
      kp<<<G, kPartNW * 32, psm, st>>>(pa, map);
    }
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  return last_launch_status();  // eight passes: the result is back in keys
}

// Explicit instantiations used by hg_api.cu (build entry point).
#define HG_INST(K, M)                                                                                   \
  template hg_status build_v2<K, M>(const Plan&, const K*, const uint32_t*, uint32_t*, K*, uint32_t*, \
                                    uint8_t*, cudaStream_t, M, uint32_t, bool);                         \
  template hg_status build_slabs<K, M>(const hg_config*, const SlabPlan&, const K*, const uint32_t*,  \
                                       uint32_t*, K*, uint32_t*, uint8_t*, cudaStream_t, M);            \
  template hg_status build_v1<K, M>(uint64_t, uint64_t, const K*, const uint32_t*, uint32_t*, K*,       \
                                    uint32_t*, uint8_t*, cudaStream_t, M);                              \
  template hg_status probe_slabs<K, M>(const hg_config*, const SlabProbePlan&, const hg_table*, const K*,  \
                                       uint64_t, uint32_t*, uint8_t*, cudaStream_t, M);                   \
  template hg_status probe_binned_impl<K, M>(const ProbePlan&, uint64_t, const hg_table*, const K*,     \
                                             uint64_t, uint32_t*, uint8_t*, cudaStream_t, M);
HG_INST(uint32_t, MurmurMap)
HG_INST(uint64_t, MurmurMap)
HG_INST(uint32_t, LearnedMap)
HG_INST(uint64_t, LearnedMap)
#undef HG_INST
// batched tables: V2 build and binned probe only (the map needs positions)
template hg_status build_v2<uint32_t, BatchedMap>(const Plan&, const uint32_t*, const uint32_t*, uint32_t*,
                                                  uint32_t*, uint32_t*, uint8_t*, cudaStream_t, BatchedMap,
                                                  uint32_t, bool);
template hg_status probe_binned_impl<uint32_t, BatchedMap>(const ProbePlan&, uint64_t, const hg_table*,
                                                           const uint32_t*, uint64_t, uint32_t*, uint8_t*,
                                                           cudaStream_t, BatchedMap);

}  // namespace hg
