// Declarations shared between the build translation unit and the API layer.
#pragma once

#include "hg_device.cuh"

namespace hg {

constexpr int kHistThreads = 1024;
constexpr uint32_t kMaxBinsLog2 = 15;  // bins counted in one shared-memory histogram
constexpr uint32_t kMaxBinShift = 15;  // buckets per bin <= 2^15 (u16 local index, 128 KB cursors)
// Partition geometry (compile-time; the defaults are the tuned values).
// Pass A (keys) and the query partition share a kernel but not their tiles:
// the query tiles must be powers of two (whole blocks of the probe's merge).
// The tile ranking in any order (k_partition ANY) and the stable ranking
// are tuned separately: they cost different registers and instructions.
#ifndef HG_PART_NW
#define HG_PART_NW 16
#endif
#ifndef HG_PART_IPT
#define HG_PART_IPT 20  // pass A, 4-byte keys, any order: tiles of 10240, one CTA per SM
#endif
#ifndef HG_PART_MINB
#define HG_PART_MINB 1
#endif
#ifndef HG_PART_IPTS
#define HG_PART_IPTS 16  // pass A, 4-byte keys, stable: tiles of 8192, one CTA per SM
#endif
#ifndef HG_PART_MINBS
#define HG_PART_MINBS 1
#endif
#ifndef HG_PART_IPTQ
#define HG_PART_IPTQ 8  // query partition (and the sample sort), 4-byte keys: tiles of 4096
#endif
#ifndef HG_PART_MINBQ
#define HG_PART_MINBQ 2
#endif
#ifndef HG_PART_IPT64
#define HG_PART_IPT64 4  // 8-byte keys, everywhere: tiles of 2048, two CTAs per SM
#endif
#ifndef HG_PART_IPTB
#define HG_PART_IPTB 6  // pass B items per thread
#endif
#ifndef HG_PARTB_NW
#define HG_PARTB_NW 16  // pass B, any order: 512-thread CTAs, two per SM
#endif
#ifndef HG_PARTB_MINB
#define HG_PARTB_MINB 2
#endif
#ifndef HG_PARTB_NWS
#define HG_PARTB_NWS 8  // pass B, stable: 256-thread CTAs, up to four per SM
#endif
#ifndef HG_PARTB_MINBS
#define HG_PARTB_MINBS 4
#endif
constexpr int kPartNW = HG_PART_NW;  // warps of the pass A / query partition CTAs
template <typename K, bool ANY>
constexpr int part_ipt_keys() {  // pass A items per thread
  return sizeof(K) == 8 ? HG_PART_IPT64 : ANY ? HG_PART_IPT : HG_PART_IPTS;
}
template <typename K, bool ANY>
constexpr int part_minb_keys() {
  return sizeof(K) == 8 ? 2 : ANY ? HG_PART_MINB : HG_PART_MINBS;
}
template <typename K>
constexpr int part_ipt_queries() {  // query partition items per thread
  return sizeof(K) == 8 ? HG_PART_IPT64 : HG_PART_IPTQ;
}
constexpr int kPartMinBlocksQ = HG_PART_MINBQ;
constexpr int kPartIPTB = HG_PART_IPTB;
template <bool ANY>
constexpr int partb_nw() {
  return ANY ? HG_PARTB_NW : HG_PARTB_NWS;
}
template <bool ANY>
constexpr int partb_minb() {
  return ANY ? HG_PARTB_MINB : HG_PARTB_MINBS;
}
constexpr uint32_t kMaxItemsPerCta = 128;  // pass B work items one CTA may own
constexpr uint32_t kMaxBinsPerCta = 256;   // bins one bin-build CTA may own
constexpr int kPartTile = kPartNW * 32 * HG_PART_IPTQ;  // query tile: 4096 elements (smallest chunk)
#ifndef HG_BIN_NW
#define HG_BIN_NW 32
#endif
constexpr int kBinNW = HG_BIN_NW;      // warps of the bin-build kernels (1024 threads)
constexpr int kBigTile = 2048;         // tile of the oversized-bin kernel
constexpr uint32_t kBinEmaxU32 = 9216;  // largest bin built in shared memory (uint32 keys)
constexpr uint32_t kBinEmaxU64 = 7168;  // same for uint64 keys
constexpr uint32_t kBinSmallBucket = 32; // bucket length sorted by one thread in the bin build
constexpr uint32_t kHugeSeg = 1u << 17;  // bins above this many edges are built by several CTAs, one per segment
constexpr uint64_t kHugeMinN = 1ull << 22;  // ... in builds of at least this many keys
constexpr uint32_t kBinRankBucket = 256; // longest bucket a warp ranks in registers in the bin build
constexpr uint32_t kBinBitmapWarps = 4;  // warps sorting longer buckets with position bitmaps
constexpr uint32_t kV1Small = 32;      // V1 fix-up: longest bucket sorted by one thread
constexpr int kV1HeavyNW = 16;
constexpr int kV1HeavyIPT = 8;  // V1 fix-up of long buckets: tiles of 4096

// V2 launch plan and workspace layout.
struct Plan {
  int kb;            // key bytes
  uint64_t n, V;
  uint32_t s;        // log2(buckets per bin)
  uint32_t sshift;   // log2(bins per super-bin)
  uint32_t nbins, nsb;
  uint32_t G;        // input chunks of pass A
  uint64_t chunk;    // elements per chunk (multiple of 16)
  uint32_t emax;     // largest bin built in shared memory
  uint32_t tpb;      // threads per bin-build CTA asked for (512 or 1024; 0 = automatic)
  uint32_t max_rows; // segments of huge bins (bins above kHugeSeg edges), upper bound
  size_t o_H, o_C, o_CT, o_T, o_BS, o_ovf, o_hlist, o_rowdesc, o_rowcnt, o_bk, o_bi, total;
};

bool make_plan_v2(const hg_config* cfg, uint64_t n, Plan* p);
// Whether every bin of a uniform spread of the keys is expected to fit the
// shared-memory bin build (mean + 5 standard deviations of a Poisson count).
bool v2_plan_fits(const Plan& p);

// Builds whose buckets need more than 2^15 bins of shared-memory size relabel
// once more (Section 3.3, "Larger Inputs"): a stable partition of the keys by
// slab of 2^Ls buckets, then one two-level build (Alg. 2) per slab into its
// slice of the table.  The slab sizes are read back to the host between the
// two steps (one stream synchronisation).
struct SlabPlan {
  int kb;
  uint64_t n, V;
  uint32_t Ls, S, G;
  uint64_t chunk;
  Plan sub;  // plan of a slab holding all n keys: the bound of every slab build's workspace
  size_t o_H, o_C, o_CT, o_T, o_BS, o_ovf, o_k, o_i, o_sub, total;
};
bool make_slab_plan(const hg_config* cfg, uint64_t n, SlabPlan* p);
template <typename K, typename Map>
hg_status build_slabs(const hg_config* cfg, const SlabPlan& p, const K* keys, const uint32_t* ids,
                      uint32_t* offsets, K* csr_k, uint32_t* csr_i, uint8_t* ws, cudaStream_t st, Map map);

// Binned probe: query groups by bucket range, workspace layout.
struct ProbePlan {
  uint32_t sg;   // group = bucket >> sg
  uint32_t ng;   // groups (<= 256)
  uint32_t G;    // query chunks
  uint64_t chunk;
  uint32_t ptile;  // queries per tile of the query partition
  size_t o_H, o_C, o_CT, o_GS, o_ovf, o_qk, o_qi, o_qc, o_tc, total;
};
bool make_probe_plan(const hg_config* cfg, uint64_t table_n, uint64_t q, ProbePlan* p);
// Binned probe of a table of more than 2^kSlabProbeLog2 buckets: 128 query
// groups would leave each group a table slice too large for L2, so the
// queries are first grouped by slab of 2^kSlabProbeLog2 buckets (the slabs a
// large build relabels by), each slab's queries take the binned probe
// against the slab's part of the table, and the counts are merged back to
// query order.  The slab query counts are read back to the host between the
// two steps (one stream synchronisation).
constexpr uint32_t kSlabProbeLog2 = 28;
struct SlabProbePlan {
  uint64_t V, q;
  uint32_t Ls, S, G;
  uint64_t chunk;
  uint32_t ptile;
  ProbePlan sub;  // plan of a slab holding all q queries: the bound of every slab probe's workspace
  size_t o_H, o_C, o_CT, o_GS, o_ovf, o_qk, o_qi, o_qc, o_tc, o_sub, total;
};
bool make_slab_probe_plan(const hg_config* cfg, uint64_t table_n, uint64_t q, SlabProbePlan* p);
template <typename K, typename Map>
hg_status probe_slabs(const hg_config* cfg, const SlabProbePlan& p, const hg_table* t, const K* queries,
                      uint64_t q, uint32_t* counts, uint8_t* ws, cudaStream_t st, Map map);
size_t radix_sort_workspace_bytes(uint64_t n);
hg_status radix_sort_u64(uint64_t* keys, uint64_t n, uint8_t* ws, cudaStream_t st);
template <typename K, typename Map>
hg_status probe_binned_impl(const ProbePlan& p, uint64_t V, const hg_table* t, const K* queries, uint64_t q,
                            uint32_t* counts, uint8_t* ws, cudaStream_t st, Map map);
size_t v1_workspace_bytes(int kb, uint64_t n, uint64_t V);

// pos_base is added to every CSR offset written (the position of element 0
// of these CSR arrays inside larger ones; 0 for a standalone table).
// positional_ids: the ids carried are distinct input positions, in input
// order (a slab of a larger build), so the partitions may rank tiles in any
// order, as with implicit ids.
template <typename K, typename Map>
hg_status build_v2(const Plan& p, const K* keys, const uint32_t* ids, uint32_t* offsets, K* csr_k,
                   uint32_t* csr_i, uint8_t* ws, cudaStream_t st, Map map, uint32_t pos_base = 0,
                   bool positional_ids = false);
template <typename K, typename Map>
hg_status build_v1(uint64_t n, uint64_t V, const K* keys, const uint32_t* ids, uint32_t* offsets,
                   K* csr_k, uint32_t* csr_i, uint8_t* ws, cudaStream_t st, Map map);

// Bucket-map construction on the host.
inline MurmurMap make_murmur(uint32_t seed, uint64_t V) {
  MurmurMap m{};
  m.seed = seed;
  if ((V & (V - 1)) == 0) {  // powers of two up to 2^32
    m.mod.pow2 = 1;
    m.mod.mask = (uint32_t)(V - 1);
  } else {                   // V < 2^32
    m.mod.pow2 = 0;
    m.mod.d = (uint32_t)V;
    fastmod_params((uint32_t)V, &m.mod.m, &m.mod.sh1, &m.mod.sh2);
  }
  return m;
}
inline LearnedMap make_learned(const void* blob, uint64_t V) {
  LearnedMap m{};
  m.blob = (const uint8_t*)blob;
  m.Vcap = V;
  return m;
}

// Calls f(K{}, map) with the key type and map the config names.
template <typename F>
hg_status dispatch_key_map(const hg_config* cfg, F&& f) {
  if (cfg->map == HG_MAP_LEARNED) {
    LearnedMap m = make_learned(cfg->d_model, cfg->num_buckets);
    return cfg->key_type == HG_KEY_U64 ? f(uint64_t{}, m) : f(uint32_t{}, m);
  }
  MurmurMap m = make_murmur(cfg->seed, cfg->num_buckets);
  return cfg->key_type == HG_KEY_U64 ? f(uint64_t{}, m) : f(uint32_t{}, m);
}

}  // namespace hg

namespace hg {
size_t join_workspace_bytes(uint64_t nA, uint64_t V);
template <typename K, typename Map>
hg_status join_count_impl(const hg_config* cfg, const hg_table* A, const hg_table* B, int64_t* d_total,
                          int64_t* d_bucket_counts, uint8_t* ws, cudaStream_t st, Map map);
template <typename K, typename Map>
hg_status join_materialize_impl(const hg_config* cfg, const hg_table* A, const hg_table* B, int64_t* outA,
                                int64_t* outB, uint64_t cap, int64_t* d_total, uint8_t* ws, cudaStream_t st,
                                Map map, bool after_count);
}  // namespace hg
