// hg_build_static_scratch: the V2 build with its scratch memory in a fixed
// device array owned by the library, for callers that cannot allocate.
//
// Who needs it: code that runs where device allocation is unavailable or not
// allowed -- for example a plug-in called from inside another runtime that
// owns all device memory and exposes no allocator, or a serving loop that
// forbids cudaMalloc/cudaFree on its hot path because they can synchronise
// the device.  Such callers still provide the inputs and outputs; only the
// intermediate bin tables and the partitioned copy of the input live here.
//
// The array below is a host-side stand-in in host code: its device address is
// obtained once per device with cudaGetSymbolAddress (while that device is
// current) and cached.  The first call on a device performs this set-up, so
// make that first call before any stream capture.  Every call shares the same
// array and leaves its contents behind; calls whose GPU work overlaps (two
// streams, two threads) race on it and must be serialised by the caller.
#include <mutex>

#include "hg_build.cuh"

namespace hg {

// 8 MiB: enough for the V2 plan of up to 2^18 keys of either key type for any
// V <= 2^29 buckets.  Larger plans (see hg_build_workspace_size) are refused.
constexpr size_t kStaticScratchBytes = 8u << 20;
static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

static hg_status static_scratch_address(void** out) {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HG_ERR_CUDA;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return HG_ERR_CUDA;
    addr[dev] = p;
  }
  *out = addr[dev];
  return HG_OK;
}

}  // namespace hg

using namespace hg;

extern "C" {

size_t hg_static_scratch_bytes(void) { return kStaticScratchBytes; }

hg_status hg_build_static_scratch(const hg_config* cfg, const void* d_keys, const uint32_t* d_ids,
                                  uint64_t n, uint32_t* d_offsets, void* d_csr_keys,
                                  uint32_t* d_csr_ids, void* stream) {
  hg_status rc = validate_config(cfg);
  if (rc != HG_OK) return rc;
  if (cfg->algo == HG_ALGO_V1) return HG_ERR_UNSUPPORTED;
  if (n >= (1ull << 32) || !d_offsets) return HG_ERR_INVALID_ARG;
  if (n > 0 && (!d_keys || !d_csr_keys || !d_csr_ids)) return HG_ERR_INVALID_ARG;
  auto mis = [](const void* p, uintptr_t a) { return ((uintptr_t)p % a) != 0; };
  if (mis(d_keys, 16) || mis(d_ids, 16) || mis(d_csr_keys, 16) || mis(d_csr_ids, 16) || mis(d_offsets, 4))
    return HG_ERR_INVALID_ARG;
  Plan p{};
  if (!make_plan_v2(cfg, n, &p)) return HG_ERR_UNSUPPORTED;
  if (p.total > kStaticScratchBytes) return HG_ERR_WORKSPACE_TOO_SMALL;  // request beyond the fixed array
  void* ws = nullptr;
  rc = static_scratch_address(&ws);
  if (rc != HG_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // The header (device status word, oversized-bin counter) must start at zero.
  if (cudaMemsetAsync(ws, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
  if (n == 0)
    return cudaMemsetAsync(d_offsets, 0, (size_t)(cfg->num_buckets + 1) * 4, st) == cudaSuccess ? HG_OK
                                                                                                : HG_ERR_CUDA;
  return dispatch_key_map(cfg, [&](auto k, auto map) -> hg_status {
    using K = decltype(k);
    return build_v2<K>(p, (const K*)d_keys, d_ids, d_offsets, (K*)d_csr_keys, d_csr_ids, (uint8_t*)ws, st, map);
  });
}

}  // extern "C"
