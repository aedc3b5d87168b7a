// Internal declarations shared by the translation units of libhg.so.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/hg.h"

namespace hg {

// Every workspace starts with this header (256 bytes, device memory).
struct WsHeader {
  uint32_t status;      // hg_status recorded by device code (0 = OK)
  uint32_t ovf_count;   // number of oversized bins (build)
  uint32_t heavy_count; // number of heavy buckets (V1 fix-up, join)
  uint32_t order_mode;  // V2 build with implicit ids: 0 = partitions may rank tiles in any
                        // order (every bin fits shared memory), 1 = stable partitions needed
  uint64_t counters[8]; // scratch counters for kernels
  uint64_t join_stamp[8];  // hg_join_count: the tables whose per-edge match counts the workspace holds
  uint32_t join_abort;     // hg_join_materialize_after_count: the stamp did not match, write nothing
  uint8_t reserved[256 - 16 - 64 - 64 - 4];
};
static_assert(sizeof(WsHeader) == 256, "workspace header");

constexpr size_t kAlign = 256;
#ifdef __CUDACC__
__host__ __device__
#endif
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// Device properties cached per device.
struct DevInfo {
  int sms = 0;
  int max_smem_optin = 0;
  int smem_per_sm = 0;    // shared memory of one SM (all resident CTAs together)
  int smem_reserved = 0;  // shared memory the system reserves per CTA
};
const DevInfo& dev_info();

// Map descriptor as resolved on the host.
struct MapDesc {
  int kind;           // hg_map_kind
  uint32_t seed;
  uint64_t V;
  const void* model;  // device pointer (learned)
};

hg_status validate_config(const hg_config* cfg);
hg_status last_launch_status();

}  // namespace hg

#define HG_RETURN_IF(cond, code) \
  do {                           \
    if (cond) return (code);     \
  } while (0)
