// C ABI entry points of libhg.so: argument checks, workspace layout and
// dispatch to the kernels.  See include/hg.h for the contract.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "hg_build.cuh"
#include "hg_probe.cuh"

namespace hg {

const DevInfo& dev_info() {
  static DevInfo cache[64];
  static bool init[64] = {};
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (!init[dev]) {
    cudaDeviceGetAttribute(&cache[dev].sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&cache[dev].max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&cache[dev].smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&cache[dev].smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (cache[dev].sms <= 0) cache[dev].sms = 152;
    init[dev] = true;
  }
  return cache[dev];
}

hg_status last_launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HG_OK : HG_ERR_CUDA;
}

hg_status validate_config(const hg_config* cfg) {
  if (!cfg) return HG_ERR_INVALID_ARG;
  if (cfg->key_type != HG_KEY_U32 && cfg->key_type != HG_KEY_U64) return HG_ERR_INVALID_ARG;
  if (cfg->map != HG_MAP_MURMUR3 && cfg->map != HG_MAP_LEARNED) return HG_ERR_INVALID_ARG;
  if (cfg->num_buckets == 0 || cfg->num_buckets > (1ull << 32)) return HG_ERR_INVALID_ARG;
  if (cfg->algo < HG_ALGO_AUTO || cfg->algo > HG_ALGO_V2) return HG_ERR_INVALID_ARG;
  if (cfg->map == HG_MAP_LEARNED && !cfg->d_model) return HG_ERR_MODEL;
  if (cfg->bin_shift > kMaxBinShift) return HG_ERR_INVALID_ARG;
  if (cfg->threads_per_bin != 0 && cfg->threads_per_bin != 512 && cfg->threads_per_bin != 1024)
    return HG_ERR_UNSUPPORTED;
  return HG_OK;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Which algorithm a build uses: V1 (Alg. 1), V2 (Alg. 2, one two-level
// plan) or V2 with one more relabeling level (slabs, when one two-level plan
// would leave its bins larger than shared memory); and the plan.
enum BuildKind { kBuildV1, kBuildV2, kBuildSlabs };
static hg_status choose_algo(const hg_config* cfg, uint64_t n, BuildKind* kind, Plan* plan, SlabPlan* slabs) {
  if (cfg->algo == HG_ALGO_V1) {
    *kind = kBuildV1;
    return HG_OK;
  }
  const bool v2ok = make_plan_v2(cfg, n, plan);
  if (v2ok && (cfg->bin_shift != 0 || v2_plan_fits(*plan))) {
    *kind = kBuildV2;
  } else if (make_slab_plan(cfg, n, slabs)) {
    *kind = kBuildSlabs;
  } else if (v2ok) {
    *kind = kBuildV2;  // bins larger than shared memory go to the oversized-bin kernels
  } else if (cfg->algo == HG_ALGO_V2) {
    return HG_ERR_UNSUPPORTED;
  } else {
    *kind = kBuildV1;
  }
  return HG_OK;
}

static size_t build_ws_bytes_of(const hg_config* cfg, uint64_t n, BuildKind kind, const Plan& p, const SlabPlan& sp) {
  if (kind == kBuildV2) return p.total;
  if (kind == kBuildSlabs) return sp.total;
  return v1_workspace_bytes(cfg->key_type == HG_KEY_U64 ? 8 : 4, n, cfg->num_buckets);
}

}  // namespace hg

using namespace hg;

extern "C" {

const char* hg_version(void) { return "hashgraph-gb300 0.1 (sm_103a)"; }

const char* hg_status_string(hg_status s) {
  switch (s) {
    case HG_OK: return "ok";
    case HG_ERR_INVALID_ARG: return "invalid argument";
    case HG_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case HG_ERR_OVERFLOW: return "output capacity exceeded";
    case HG_ERR_CUDA: return "CUDA error";
    case HG_ERR_TIMEOUT: return "device-side wait timed out";
    case HG_ERR_MODEL: return "invalid learned-map model";
    case HG_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

size_t hg_build_workspace_size(const hg_config* cfg, uint64_t n) {
  if (validate_config(cfg) != HG_OK) return 0;
  BuildKind kind = kBuildV1;
  Plan p{};
  SlabPlan sp{};
  if (choose_algo(cfg, n, &kind, &p, &sp) != HG_OK) return 0;
  return build_ws_bytes_of(cfg, n, kind, p, sp);
}

hg_status hg_build(const hg_config* cfg, const void* d_keys, const uint32_t* d_ids, uint64_t n,
                   uint32_t* d_offsets, void* d_csr_keys, uint32_t* d_csr_ids, void* d_ws,
                   size_t ws_bytes, void* stream) {
  hg_status rc = validate_config(cfg);
  if (rc != HG_OK) return rc;
  if (n >= (1ull << 32)) return HG_ERR_INVALID_ARG;
  if (!d_offsets || !d_ws) return HG_ERR_INVALID_ARG;
  if (n > 0 && (!d_keys || !d_csr_keys || !d_csr_ids)) return HG_ERR_INVALID_ARG;
  if (!aligned(d_keys, 16) || !aligned(d_ids, 16) || !aligned(d_csr_keys, 16) || !aligned(d_csr_ids, 16) ||
      !aligned(d_offsets, 4) || !aligned(d_ws, 256))
    return HG_ERR_INVALID_ARG;
  BuildKind kind = kBuildV1;
  Plan p{};
  SlabPlan sp{};
  rc = choose_algo(cfg, n, &kind, &p, &sp);
  if (rc != HG_OK) return rc;
  if (ws_bytes < build_ws_bytes_of(cfg, n, kind, p, sp)) return HG_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_ws, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
  if (n == 0) {
    if (cudaMemsetAsync(d_offsets, 0, (size_t)(cfg->num_buckets + 1) * 4, st) != cudaSuccess) return HG_ERR_CUDA;
    return HG_OK;
  }
  return dispatch_key_map(cfg, [&](auto k, auto map) -> hg_status {
    using K = decltype(k);
    if (kind == kBuildV2)
      return build_v2<K>(p, (const K*)d_keys, d_ids, d_offsets, (K*)d_csr_keys, d_csr_ids, (uint8_t*)d_ws, st, map);
    if (kind == kBuildSlabs)
      return build_slabs<K>(cfg, sp, (const K*)d_keys, d_ids, d_offsets, (K*)d_csr_keys, d_csr_ids, (uint8_t*)d_ws,
                            st, map);
    return build_v1<K>(n, cfg->num_buckets, (const K*)d_keys, d_ids, d_offsets, (K*)d_csr_keys, d_csr_ids,
                       (uint8_t*)d_ws, st, map);
  });
}

hg_status hg_probe(const hg_config* cfg, const hg_table* table, const void* d_queries, uint64_t q,
                   uint32_t* d_counts, void* stream) {
  hg_status rc = validate_config(cfg);
  if (rc != HG_OK) return rc;
  if (!table || !table->d_offsets) return HG_ERR_INVALID_ARG;
  if (q > 0 && (!d_queries || !d_counts)) return HG_ERR_INVALID_ARG;
  if (table->n > 0 && !table->d_keys) return HG_ERR_INVALID_ARG;
  const size_t kb = cfg->key_type == HG_KEY_U64 ? 8 : 4;
  if (!aligned(d_queries, kb) || !aligned(table->d_keys, kb) || !aligned(d_counts, 4)) return HG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  return dispatch_key_map(cfg, [&](auto k, auto map) -> hg_status {
    using K = decltype(k);
    return probe_launch<K>((const K*)d_queries, q, table->d_offsets, (const K*)table->d_keys, d_counts,
                           cfg->num_buckets, st, map);
  });
}

size_t hg_probe_workspace_size(const hg_config* cfg, uint64_t table_n, uint64_t q) {
  if (validate_config(cfg) != HG_OK) return 0;
  SlabProbePlan sp{};
  if (make_slab_probe_plan(cfg, table_n, q, &sp)) return sp.total;
  ProbePlan p{};
  if (!make_probe_plan(cfg, table_n, q, &p)) return 0;
  return p.total;
}

hg_status hg_probe_binned(const hg_config* cfg, const hg_table* table, const void* d_queries, uint64_t q,
                          uint32_t* d_counts, void* d_ws, size_t ws_bytes, void* stream) {
  hg_status rc = validate_config(cfg);
  if (rc != HG_OK) return rc;
  if (!table || !table->d_offsets || !d_ws) return HG_ERR_INVALID_ARG;
  if (q >= (1ull << 32)) return HG_ERR_INVALID_ARG;
  if (q > 0 && (!d_queries || !d_counts)) return HG_ERR_INVALID_ARG;
  if (table->n > 0 && !table->d_keys) return HG_ERR_INVALID_ARG;
  const size_t kb = cfg->key_type == HG_KEY_U64 ? 8 : 4;
  if (!aligned(d_queries, 16) || !aligned(table->d_keys, kb) || !aligned(d_counts, 4) || !aligned(d_ws, 256))
    return HG_ERR_INVALID_ARG;
  SlabProbePlan sp{};
  const bool slabs = make_slab_probe_plan(cfg, table->n, q, &sp);
  ProbePlan p{};
  if (!slabs && !make_probe_plan(cfg, table->n, q, &p)) return HG_ERR_UNSUPPORTED;
  if (ws_bytes < (slabs ? sp.total : p.total)) return HG_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_ws, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
  if (q == 0) return HG_OK;
  return dispatch_key_map(cfg, [&](auto k, auto map) -> hg_status {
    using K = decltype(k);
    if (slabs)
      return probe_slabs<K>(cfg, sp, table, (const K*)d_queries, q, d_counts, (uint8_t*)d_ws, st, map);
    return probe_binned_impl<K>(p, cfg->num_buckets, table, (const K*)d_queries, q, d_counts, (uint8_t*)d_ws, st,
                                map);
  });
}

// Per-device state of hg_build_probe_host (created on first use, kept until
// exit): the upload stream, on which the host -> device copies of all calls
// queue in call order, and an event marking the end of the last call's
// kernels, after which the next call's kernels start.
struct HostPipe {
  cudaStream_t up = nullptr;
  cudaEvent_t done = nullptr;
  bool recorded = false;
};
static std::mutex g_pipe_mu;
static HostPipe* host_pipe() {
  static HostPipe pipes[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  HostPipe& p = pipes[dev];
  if (!p.up && cudaStreamCreateWithFlags(&p.up, cudaStreamNonBlocking) != cudaSuccess) p.up = nullptr;
  if (!p.done && cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming) != cudaSuccess) p.done = nullptr;
  return p.up && p.done ? &p : nullptr;
}

// Records an event on `from` and makes `to` wait for it.
static bool join(cudaStream_t from, cudaStream_t to) {
  cudaEvent_t e;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
  const bool ok = cudaEventRecord(e, from) == cudaSuccess && cudaStreamWaitEvent(to, e, 0) == cudaSuccess;
  cudaEventDestroy(e);  // released once it has completed
  return ok;
}

hg_status hg_build_probe_host(const hg_config* cfg, const void* h_keys, uint64_t n, const void* h_queries,
                              uint64_t q, uint32_t* h_counts, void* d_keys, void* d_queries, uint32_t* d_counts,
                              const hg_table* table, void* d_build_ws, size_t build_ws_bytes, void* d_probe_ws,
                              size_t probe_ws_bytes, void* stream) {
  hg_status rc = validate_config(cfg);
  if (rc != HG_OK) return rc;
  if (!table || table->n != n || (n > 0 && (!h_keys || !d_keys)) || (q > 0 && (!h_queries || !h_counts)))
    return HG_ERR_INVALID_ARG;
  const size_t kb = cfg->key_type == HG_KEY_U64 ? 8 : 4;
  // Everything the build and the probe below would refuse is refused here,
  // before the first copy is enqueued, so an argument error launches nothing.
  if (n >= (1ull << 32) || (d_probe_ws && q >= (1ull << 32))) return HG_ERR_INVALID_ARG;
  if (!table->d_offsets || !d_build_ws || (n > 0 && (!table->d_keys || !table->d_ids)) ||
      (q > 0 && (!d_queries || !d_counts)))
    return HG_ERR_INVALID_ARG;
  if (!aligned(d_keys, 16) || !aligned(table->d_keys, 16) || !aligned(table->d_ids, 16) ||
      !aligned(table->d_offsets, 4) || !aligned(d_queries, d_probe_ws ? 16 : kb) || !aligned(d_counts, 4) ||
      !aligned(d_build_ws, 256) || !aligned(d_probe_ws, 256))
    return HG_ERR_INVALID_ARG;
  {
    BuildKind kind = kBuildV1;
    Plan p{};
    SlabPlan sp{};
    rc = choose_algo(cfg, n, &kind, &p, &sp);
    if (rc != HG_OK) return rc;
    if (build_ws_bytes < build_ws_bytes_of(cfg, n, kind, p, sp)) return HG_ERR_WORKSPACE_TOO_SMALL;
  }
  if (q > 0 && d_probe_ws) {
    const size_t need = hg_probe_workspace_size(cfg, n, q);
    if (need == 0) return HG_ERR_UNSUPPORTED;
    if (probe_ws_bytes < need) return HG_ERR_WORKSPACE_TOO_SMALL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // one call at a time per device enqueues, so that the device sees the
  // calls in one order
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe* pp = host_pipe();
  if (!pp) return HG_ERR_CUDA;
  cudaStream_t up = pp->up;
  // uploads start once `stream` is done with the staging buffers, the build
  // waits for the keys and for the previous call's kernels, the probe for
  // the queries as well
  if (!join(st, up)) return HG_ERR_CUDA;
  if (n > 0 && cudaMemcpyAsync(d_keys, h_keys, n * kb, cudaMemcpyHostToDevice, up) != cudaSuccess) return HG_ERR_CUDA;
  if (!join(up, st)) return HG_ERR_CUDA;
  if (pp->recorded && cudaStreamWaitEvent(st, pp->done, 0) != cudaSuccess) return HG_ERR_CUDA;
  if (q > 0 && cudaMemcpyAsync(d_queries, h_queries, q * kb, cudaMemcpyHostToDevice, up) != cudaSuccess)
    return HG_ERR_CUDA;
  // the table's buffers are this call's output (hg_table carries them as const for probes)
  rc = hg_build(cfg, d_keys, nullptr, n, const_cast<uint32_t*>(table->d_offsets), const_cast<void*>(table->d_keys),
                const_cast<uint32_t*>(table->d_ids), d_build_ws, build_ws_bytes, stream);
  if (rc != HG_OK) return rc;
  if (!join(up, st)) return HG_ERR_CUDA;
  if (q == 0) return HG_OK;
  rc = d_probe_ws ? hg_probe_binned(cfg, table, d_queries, q, d_counts, d_probe_ws, probe_ws_bytes, stream)
                  : hg_probe(cfg, table, d_queries, q, d_counts, stream);
  if (rc != HG_OK) return rc;
  if (cudaEventRecord(pp->done, st) != cudaSuccess) return HG_ERR_CUDA;
  pp->recorded = true;
  if (cudaMemcpyAsync(h_counts, d_counts, q * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HG_ERR_CUDA;
  return HG_OK;
}

size_t hg_join_workspace_size(const hg_config* cfg, uint64_t nA, uint64_t nB) {
  (void)nB;
  if (validate_config(cfg) != HG_OK) return 0;
  return join_workspace_bytes(nA, cfg->num_buckets);
}

static hg_status check_join_args(const hg_config* cfg, const hg_table* A, const hg_table* B, const void* d_ws) {
  hg_status rc = validate_config(cfg);
  if (rc != HG_OK) return rc;
  if (!A || !B || !A->d_offsets || !B->d_offsets || !d_ws) return HG_ERR_INVALID_ARG;
  if ((A->n > 0 && (!A->d_keys || !A->d_ids)) || (B->n > 0 && (!B->d_keys || !B->d_ids))) return HG_ERR_INVALID_ARG;
  if (A->n >= (1ull << 32) || B->n >= (1ull << 32)) return HG_ERR_INVALID_ARG;
  const size_t kb = cfg->key_type == HG_KEY_U64 ? 8 : 4;
  if (!aligned(A->d_keys, kb) || !aligned(B->d_keys, kb) || !aligned(d_ws, 256)) return HG_ERR_INVALID_ARG;
  return HG_OK;
}

hg_status hg_join_count(const hg_config* cfg, const hg_table* A, const hg_table* B, int64_t* d_total,
                        int64_t* d_bucket_counts, void* d_ws, size_t ws_bytes, void* stream) {
  hg_status rc = check_join_args(cfg, A, B, d_ws);
  if (rc != HG_OK) return rc;
  if (!d_total || !aligned(d_total, 8) || !aligned(d_bucket_counts, 8)) return HG_ERR_INVALID_ARG;
  if (ws_bytes < join_workspace_bytes(A->n, cfg->num_buckets)) return HG_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_ws, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
  return dispatch_key_map(cfg, [&](auto k, auto map) -> hg_status {
    using K = decltype(k);
    return join_count_impl<K>(cfg, A, B, d_total, d_bucket_counts, (uint8_t*)d_ws, st, map);
  });
}

hg_status hg_join_materialize(const hg_config* cfg, const hg_table* A, const hg_table* B,
                              int64_t* d_build_ids, int64_t* d_probe_ids, uint64_t capacity,
                              int64_t* d_total, void* d_ws, size_t ws_bytes, void* stream) {
  hg_status rc = check_join_args(cfg, A, B, d_ws);
  if (rc != HG_OK) return rc;
  if (!d_total || !aligned(d_total, 8)) return HG_ERR_INVALID_ARG;
  if (capacity > 0 && (!d_build_ids || !d_probe_ids)) return HG_ERR_INVALID_ARG;
  if (!aligned(d_build_ids, 8) || !aligned(d_probe_ids, 8)) return HG_ERR_INVALID_ARG;
  if (ws_bytes < join_workspace_bytes(A->n, cfg->num_buckets)) return HG_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_ws, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
  return dispatch_key_map(cfg, [&](auto k, auto map) -> hg_status {
    using K = decltype(k);
    return join_materialize_impl<K>(cfg, A, B, d_build_ids, d_probe_ids, capacity, d_total, (uint8_t*)d_ws, st,
                                    map, false);
  });
}

hg_status hg_join_materialize_after_count(const hg_config* cfg, const hg_table* A, const hg_table* B,
                                          int64_t* d_build_ids, int64_t* d_probe_ids, uint64_t capacity,
                                          int64_t* d_total, void* d_ws, size_t ws_bytes, void* stream) {
  hg_status rc = check_join_args(cfg, A, B, d_ws);
  if (rc != HG_OK) return rc;
  if (!d_total || !aligned(d_total, 8)) return HG_ERR_INVALID_ARG;
  if (capacity > 0 && (!d_build_ids || !d_probe_ids)) return HG_ERR_INVALID_ARG;
  if (!aligned(d_build_ids, 8) || !aligned(d_probe_ids, 8)) return HG_ERR_INVALID_ARG;
  if (ws_bytes < join_workspace_bytes(A->n, cfg->num_buckets)) return HG_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  // only the status word is cleared: the rest of the header holds the count's stamp
  if (cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), st) != cudaSuccess) return HG_ERR_CUDA;
  return dispatch_key_map(cfg, [&](auto k, auto map) -> hg_status {
    using K = decltype(k);
    return join_materialize_impl<K>(cfg, A, B, d_build_ids, d_probe_ids, capacity, d_total, (uint8_t*)d_ws, st,
                                    map, true);
  });
}

// One CTA waits on a barrier initialised for two arrivals that only ever
// gets one: the bounded wait gives up after limit_ns, records
// HG_ERR_TIMEOUT and the kernel returns.
__global__ void k_selftest_wait(uint32_t* status, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive(&bar);
  mbar_wait_block(&bar, 0, status, limit_ns);
}

hg_status hg_selftest_wait_timeout(void* d_ws, uint32_t limit_ms, void* stream) {
  if (!d_ws || limit_ms == 0 || limit_ms > 5000) return HG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_ws, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
  k_selftest_wait<<<1, 64, 0, st>>>(&((WsHeader*)d_ws)->status, (uint64_t)limit_ms * 1000000ull);
  return last_launch_status();
}

hg_status hg_workspace_status(const void* d_ws, void* stream) {
  if (!d_ws) return HG_ERR_INVALID_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return HG_ERR_CUDA;
  uint32_t s = 0;
  if (cudaMemcpy(&s, d_ws, sizeof(s), cudaMemcpyDeviceToHost) != cudaSuccess) return HG_ERR_CUDA;
  return (hg_status)s;
}

hg_status hg_workspace_clear(void* d_ws, void* stream) {
  if (!d_ws) return HG_ERR_INVALID_ARG;
  return cudaMemsetAsync(d_ws, 0, sizeof(WsHeader), (cudaStream_t)stream) == cudaSuccess ? HG_OK : HG_ERR_CUDA;
}

}  // extern "C"
