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
// In host code, g_static_scratch names only a handle to the array; the
// array itself lives in device memory.  Its device address is looked up with
// cudaGetSymbolAddress, with the device current, and cached per device.  The
// first call on a device does this set-up, so make it before any stream
// capture.  Later calls look the address up again whenever their stream is
// not capturing (a device reset reloads the module at a new address); a call
// made during a capture uses the cached one.  Every call shares the same
// array and leaves its contents behind; calls whose GPU work overlaps (two
// streams, two threads) race on it and must be serialised by the caller.
#include <mutex>

#include "hg_build.cuh"

namespace hg {

// 8 MiB: with the automatic bin size, enough for the V2 plan of up to 2^18
// keys into V <= 2^29 buckets with uint32 keys (7.0 MiB at the edge) and
// V <= 2^28 with uint64 keys (6.0 MiB; 2^29 buckets would need 8.002 MiB).
// Larger plans (see hg_build_workspace_size) are refused.
constexpr size_t kStaticScratchBytes = 8u << 20;
static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

static hg_status static_scratch_address(cudaStream_t st, void** out) {
  static std::mutex mu;
  static void* addr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HG_ERR_CUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return HG_ERR_CUDA;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev] || cs == cudaStreamCaptureStatusNone) {
    if (cs != cudaStreamCaptureStatusNone) return HG_ERR_UNSUPPORTED;  // first call inside a capture
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
  cudaStream_t st = (cudaStream_t)stream;
  void* ws = nullptr;
  rc = static_scratch_address(st, &ws);
  if (rc != HG_OK) return rc;
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

// The device status word of the last build in the fixed array (a bounded
// wait that gave up, a bin-size bound exceeded).  Synchronises the stream and
// reads the word; nothing is allocated.
hg_status hg_static_scratch_status(void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  void* ws = nullptr;
  hg_status rc = static_scratch_address(st, &ws);
  if (rc != HG_OK) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HG_ERR_CUDA;
  uint32_t s = 0;
  if (cudaMemcpy(&s, ws, sizeof(s), cudaMemcpyDeviceToHost) != cudaSuccess) return HG_ERR_CUDA;
  return (hg_status)s;
}

}  // extern "C"
