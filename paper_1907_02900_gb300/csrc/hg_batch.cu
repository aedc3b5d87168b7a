// Batched tables (not in the paper, which builds one table per call): many
// independent tables of uneven sizes built and probed together.
//
// GB300 design.  All tables share one bucket space: table t owns the global
// buckets [ob_t, ob_t + V_t] (the last one is a spare that no hash reaches)
// and the input positions [kb_t, kb_{t+1}).  A two-level build (Alg. 2) over the
// concatenated keys with the batched bucket map (Eq. 1 per table, the table
// found from the position) then produces every table at once, bit for bit
// the table a standalone build makes, because the canonical order inside a
// bucket is the input order and every table's keys are contiguous.  Every
// table's keys (and queries) start on a 16-byte boundary, as the TMA tile
// loads need; the up to 3 positions of padding in front of the next table
// belong to the table's spare bucket V_t.  The bin
// histogram of Alg. 2 holds at most 2^15 bins, so tables are grouped into
// waves whose buckets fit 2^15 bins of the chosen bin size; per wave one
// build and one binned probe run over the wave's slice of the bucket space.
// The whole launch sequence is captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hg_build.cuh"
#include "hg_internal.h"
#include "hg_probe.cuh"
#include "hg_trace.h"

namespace hg {
namespace {

constexpr uint32_t kBatchPageShift = 12;  // positions per directory page: 4096
constexpr uint32_t kMaxBins = 1u << kMaxBinsLog2;

__global__ void k_fold_status(uint32_t* __restrict__ batch_status, const uint32_t* __restrict__ wave_status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const uint32_t s = *wave_status;
    if (s != 0 && *batch_status == 0) *batch_status = s;
  }
}

__global__ void k_fill_u32(uint32_t* __restrict__ p, uint64_t n, uint32_t v) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

struct Wave {
  uint32_t t0, t1;     // tables [t0, t1)
  uint64_t k0, nk;     // key positions
  uint64_t q0, nq;     // query positions
  uint64_t b0, nb;     // global buckets (sum of V_t + 1)
  Plan bp;
  ProbePlan pp;
};

int ceil_log2(uint64_t x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

}  // namespace
}  // namespace hg

using namespace hg;

struct hg_batch_plan {
  int32_t key_type = HG_KEY_U32;
  uint32_t seed = 0;
  uint32_t T = 0;
  int device = 0;
  std::vector<uint64_t> n, q, V;
  std::vector<uint64_t> kbeg, qbeg, obeg;  // T+1 each; kbeg and qbeg are multiples of 4
  uint64_t nk = 0, nq = 0, nob = 0;        // totals; offsets entries = nob + 1
  uint32_t auto_shift = 12;
  uint32_t bin_shift = 0, tpb = 0;         // current configuration (0 = automatic)
  std::vector<Wave> waves;
  // directory: host copy (pinned) uploaded into the workspace by every run
  uint8_t* h_dir = nullptr;
  size_t dir_bytes = 0, o_kbeg = 0, o_qbeg = 0, o_klen = 0, o_qlen = 0, o_desc = 0, o_kpage = 0, o_qpage = 0;
  size_t dir_off = 0, region_off = 0, ws_total = 0;
  // graph of the current configuration and buffers
  cudaGraphExec_t exec = nullptr;
  const void* bound[8] = {};
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {

hg_config table_config(const hg_batch_plan* P, uint64_t V, uint32_t shift, uint32_t tpb) {
  hg_config c{};
  c.key_type = P->key_type;
  c.map = HG_MAP_MURMUR3;
  c.num_buckets = V;
  c.seed = P->seed;
  c.algo = HG_ALGO_V2;
  c.d_model = nullptr;
  c.bin_shift = shift;
  c.threads_per_bin = tpb;
  return c;
}

// Waves for a bin shift: consecutive tables while their buckets fit 2^15
// bins; a table larger than that forms a wave of its own with a larger shift.
bool plan_waves(const hg_batch_plan* P, uint32_t shift, uint32_t tpb, std::vector<Wave>* out, size_t* region) {
  std::vector<Wave> ws;
  const uint64_t cap = (uint64_t)kMaxBins << shift;
  uint32_t t = 0;
  while (t < P->T) {
    Wave w{};
    w.t0 = t;
    w.k0 = P->kbeg[t];
    w.q0 = P->qbeg[t];
    w.b0 = P->obeg[t];
    uint64_t nb = 0;
    do {
      nb += P->V[t] + 1;
      ++t;
    } while (t < P->T && nb + P->V[t] + 1 <= cap);
    w.t1 = t;
    w.nk = P->kbeg[t] - w.k0;
    w.nq = P->qbeg[t] - w.q0;
    w.nb = nb;
    ws.push_back(w);
  }
  size_t reg = 0;
  for (Wave& w : ws) {
    const uint32_t s = (uint32_t)std::max<int>((int)shift, ceil_log2(w.nb) - (int)kMaxBinsLog2);
    if (s > kMaxBinShift) return false;
    hg_config c = table_config(P, w.nb, s, tpb);
    if (w.nk > 0) {
      if (!make_plan_v2(&c, w.nk, &w.bp)) return false;
      reg = std::max(reg, w.bp.total);
    }
    if (w.nq > 0) {
      if (!make_probe_plan(&c, w.nk, w.nq, &w.pp)) return false;
      reg = std::max(reg, w.pp.total);
    }
  }
  *out = std::move(ws);
  *region = reg;
  return true;
}

uint32_t effective_shift(const hg_batch_plan* P) { return P->bin_shift ? P->bin_shift : P->auto_shift; }

void drop_graph(hg_batch_plan* P) {
  if (P->exec) cudaGraphExecDestroy(P->exec);
  P->exec = nullptr;
  std::memset(P->bound, 0, sizeof(P->bound));
}

hg_status apply_config(hg_batch_plan* P) {
  size_t reg = 0;
  std::vector<Wave> ws;
  if (!plan_waves(P, effective_shift(P), P->tpb, &ws, &reg)) return HG_ERR_UNSUPPORTED;
  if (P->region_off + reg > P->ws_total) return HG_ERR_UNSUPPORTED;
  P->waves = std::move(ws);
  drop_graph(P);
  return HG_OK;
}

struct Bufs {
  const uint32_t* keys;
  const uint32_t* queries;
  uint32_t* offsets;
  uint32_t* csr_k;
  uint32_t* csr_i;
  uint32_t* counts;
  uint8_t* ws;
};

// The whole batch, enqueued on st (no host synchronisation: capturable).
hg_status enqueue(hg_batch_plan* P, const Bufs& b, cudaStream_t st) {
  uint8_t* dir = b.ws + P->dir_off;
  if (cudaMemcpyAsync(dir, P->h_dir, P->dir_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return HG_ERR_CUDA;
  if (cudaMemsetAsync(b.ws, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
  uint32_t* batch_status = &((WsHeader*)b.ws)->status;
  uint8_t* R = b.ws + P->region_off;
  const uint32_t* wave_status = &((WsHeader*)R)->status;
  BatchedMap base{};
  base.seed = P->seed;
  base.page_shift = kBatchPageShift;
  base.desc = (const uint4*)(dir + P->o_desc);
  for (const Wave& w : P->waves) {
    if (w.nk == 0) {
      const unsigned grid = (unsigned)std::min<uint64_t>((w.nb + 1 + 255) / 256, 1024);
      k_fill_u32<<<grid, 256, 0, st>>>(b.offsets + w.b0, w.nb + 1, (uint32_t)w.k0);
    } else {
      BatchedMap km = base;
      km.pos_base = w.k0;
      km.bucket_base = (uint32_t)w.b0;
      km.begin = (const uint64_t*)(dir + P->o_kbeg);
      km.len = (const uint32_t*)(dir + P->o_klen);
      km.page = (const uint32_t*)(dir + P->o_kpage);
      if (cudaMemsetAsync(R, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
      hg_status rc = build_v2<uint32_t>(w.bp, b.keys + w.k0, nullptr, b.offsets + w.b0, b.csr_k + w.k0,
                                        b.csr_i + w.k0, R, st, km, (uint32_t)w.k0);
      if (rc != HG_OK) return rc;
      k_fold_status<<<1, 32, 0, st>>>(batch_status, wave_status);
    }
    if (w.nq > 0) {
      BatchedMap qm = base;
      qm.pos_base = w.q0;
      qm.bucket_base = (uint32_t)w.b0;
      qm.begin = (const uint64_t*)(dir + P->o_qbeg);
      qm.len = (const uint32_t*)(dir + P->o_qlen);
      qm.page = (const uint32_t*)(dir + P->o_qpage);
      hg_table tw{};
      tw.n = w.nk;
      tw.d_offsets = b.offsets + w.b0;
      tw.d_keys = b.csr_k;  // offsets are positions in the concatenated arrays
      tw.d_ids = b.csr_i;
      if (cudaMemsetAsync(R, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
      hg_status rc = probe_binned_impl<uint32_t>(w.pp, w.nb, &tw, b.queries + w.q0, w.nq, b.counts + w.q0, R, st,
                                                 qm);
      if (rc != HG_OK) return rc;
      k_fold_status<<<1, 32, 0, st>>>(batch_status, wave_status);
    }
  }
  return last_launch_status();
}

hg_status check_bufs(const hg_batch_plan* P, const Bufs& b, size_t ws_bytes) {
  if (!b.ws || !b.offsets) return HG_ERR_INVALID_ARG;
  if (P->nk > 0 && (!b.keys || !b.csr_k || !b.csr_i)) return HG_ERR_INVALID_ARG;
  if (P->nq > 0 && (!b.queries || !b.counts)) return HG_ERR_INVALID_ARG;
  auto al = [](const void* p, size_t a) { return ((uintptr_t)p % a) == 0; };
  if (!al(b.keys, 16) || !al(b.queries, 16) || !al(b.csr_k, 16) || !al(b.csr_i, 16) || !al(b.offsets, 4) ||
      !al(b.counts, 4) || !al(b.ws, 256))
    return HG_ERR_INVALID_ARG;
  if (ws_bytes < P->ws_total) return HG_ERR_WORKSPACE_TOO_SMALL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return HG_ERR_INVALID_ARG;
  return HG_OK;
}

// Replays the graph of the current configuration (capturing it first when
// the buffers changed), ordered after and before the caller's stream.
hg_status run_graph(hg_batch_plan* P, const Bufs& b, cudaStream_t user) {
  const void* key[8] = {b.keys, b.queries, b.offsets, b.csr_k, b.csr_i, b.counts, b.ws, nullptr};
  if (!P->exec || std::memcmp(key, P->bound, sizeof(key)) != 0) {
    drop_graph(P);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(P->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HG_ERR_CUDA;
    const hg_status rc = enqueue(P, b, P->st);
    const cudaError_t ce = cudaStreamEndCapture(P->st, &g);
    if (rc != HG_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return rc != HG_OK ? rc : HG_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&P->exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      P->exec = nullptr;
      return HG_ERR_CUDA;
    }
    std::memcpy(P->bound, key, sizeof(key));
  }
  if (cudaEventRecord(P->ev_in, user) != cudaSuccess) return HG_ERR_CUDA;
  if (cudaStreamWaitEvent(P->st, P->ev_in, 0) != cudaSuccess) return HG_ERR_CUDA;
  if (cudaGraphLaunch(P->exec, P->st) != cudaSuccess) return HG_ERR_CUDA;
  if (cudaEventRecord(P->ev_out, P->st) != cudaSuccess) return HG_ERR_CUDA;
  if (cudaStreamWaitEvent(user, P->ev_out, 0) != cudaSuccess) return HG_ERR_CUDA;
  return HG_OK;
}

}  // namespace

extern "C" {

hg_status hg_batch_plan_create(int32_t key_type, uint32_t seed, uint32_t num_tables, const uint64_t* h_table_sizes,
                               const uint64_t* h_query_sizes, const uint64_t* h_num_buckets, hg_batch_plan** out) {
  if (!out) return HG_ERR_INVALID_ARG;
  *out = nullptr;
  if (key_type != HG_KEY_U32) return key_type == HG_KEY_U64 ? HG_ERR_UNSUPPORTED : HG_ERR_INVALID_ARG;
  if (num_tables == 0 || !h_table_sizes || !h_query_sizes) return HG_ERR_INVALID_ARG;
  hg_batch_plan* P = new hg_batch_plan();
  P->key_type = key_type;
  P->seed = seed;
  P->T = num_tables;
  P->n.assign(h_table_sizes, h_table_sizes + num_tables);
  P->q.assign(h_query_sizes, h_query_sizes + num_tables);
  P->V.resize(num_tables);
  P->kbeg.assign(num_tables + 1, 0);
  P->qbeg.assign(num_tables + 1, 0);
  P->obeg.assign(num_tables + 1, 0);
  for (uint32_t t = 0; t < num_tables; ++t) {
    const uint64_t V = h_num_buckets ? h_num_buckets[t] : std::max<uint64_t>(1, P->n[t]);
    if (V == 0 || V >= (1ull << 31)) {
      delete P;
      return HG_ERR_INVALID_ARG;
    }
    if (P->n[t] >= (1ull << 32) || P->q[t] >= (1ull << 32)) {
      delete P;
      return HG_ERR_INVALID_ARG;
    }
    P->V[t] = V;
    P->kbeg[t + 1] = P->kbeg[t] + (P->n[t] + 3) / 4 * 4;
    P->qbeg[t + 1] = P->qbeg[t] + (P->q[t] + 3) / 4 * 4;
    P->obeg[t + 1] = P->obeg[t] + V + 1;
  }
  P->nk = P->kbeg[num_tables];
  P->nq = P->qbeg[num_tables];
  P->nob = P->obeg[num_tables];
  if (P->nk >= (1ull << 32) - 1 || P->nq >= (1ull << 32) || P->nob + 1 >= (1ull << 32)) {
    delete P;
    return HG_ERR_INVALID_ARG;
  }
  // automatic bin size: the shift a single table of the batch's load factor
  // would get (bins of about 3/4 of the shared-memory capacity)
  {
    const double load = P->nob ? (double)P->nk / (double)P->nob : 1.0;
    const double bpb = 0.75 * (double)kBinEmaxU32 / std::max(load, 1e-9);
    P->auto_shift = (uint32_t)std::min<double>(kMaxBinShift, std::max(0.0, std::floor(std::log2(std::max(bpb, 1.0)))));
  }
  // directory layout and host copy
  const uint64_t kpages = (P->nk >> kBatchPageShift) + 1, qpages = (P->nq >> kBatchPageShift) + 1;
  size_t o = 0;
  P->o_kbeg = o;  o = align_up(o + (size_t)(num_tables + 1) * 8);
  P->o_qbeg = o;  o = align_up(o + (size_t)(num_tables + 1) * 8);
  P->o_klen = o;  o = align_up(o + (size_t)num_tables * 4);
  P->o_qlen = o;  o = align_up(o + (size_t)num_tables * 4);
  P->o_desc = o;  o = align_up(o + (size_t)num_tables * 16);
  P->o_kpage = o; o = align_up(o + (size_t)kpages * 4);
  P->o_qpage = o; o = align_up(o + (size_t)qpages * 4);
  P->dir_bytes = o;
  if (cudaGetDevice(&P->device) != cudaSuccess || cudaMallocHost((void**)&P->h_dir, P->dir_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return HG_ERR_CUDA;
  }
  std::memcpy(P->h_dir + P->o_kbeg, P->kbeg.data(), (size_t)(num_tables + 1) * 8);
  std::memcpy(P->h_dir + P->o_qbeg, P->qbeg.data(), (size_t)(num_tables + 1) * 8);
  uint32_t* desc = (uint32_t*)(P->h_dir + P->o_desc);
  uint32_t* klen = (uint32_t*)(P->h_dir + P->o_klen);
  uint32_t* qlen = (uint32_t*)(P->h_dir + P->o_qlen);
  for (uint32_t t = 0; t < num_tables; ++t) {
    klen[t] = (uint32_t)P->n[t];
    qlen[t] = (uint32_t)P->q[t];
    const uint32_t V = (uint32_t)P->V[t];  // < 2^31
    uint32_t m = 0, sh1 = 0, sh2 = 0;
    fastmod_params(V, &m, &sh1, &sh2);    // every V_t, powers of two included
    desc[4 * t + 0] = (uint32_t)P->obeg[t];
    desc[4 * t + 1] = V;
    desc[4 * t + 2] = m;
    desc[4 * t + 3] = sh1 | (sh2 << 8);
  }
  auto pages = [&](const std::vector<uint64_t>& beg, uint64_t np, uint32_t* pg) {
    uint32_t t = 0;
    for (uint64_t p = 0; p < np; ++p) {
      const uint64_t pos = p << kBatchPageShift;
      while (t + 1 < num_tables && beg[t + 1] <= pos) ++t;
      pg[p] = t;
    }
  };
  pages(P->kbeg, kpages, (uint32_t*)(P->h_dir + P->o_kpage));
  pages(P->qbeg, qpages, (uint32_t*)(P->h_dir + P->o_qpage));
  // workspace: batch header, directory, one region reused by every wave (and
  // by the plain loop); sized for every configuration the autotuner tries
  P->dir_off = sizeof(WsHeader);
  P->region_off = align_up(P->dir_off + P->dir_bytes);
  size_t region = 0;
  for (uint32_t s = 0; s <= kMaxBinShift; ++s)
    for (uint32_t tpb : {512u, 1024u}) {
      std::vector<Wave> ws;
      size_t reg = 0;
      if (plan_waves(P, s, tpb, &ws, &reg)) region = std::max(region, reg);
    }
  for (uint32_t t = 0; t < num_tables; ++t) {
    hg_config c = table_config(P, P->V[t], 0, 0);
    c.algo = HG_ALGO_AUTO;
    region = std::max(region, hg_build_workspace_size(&c, P->n[t]));
  }
  P->ws_total = P->region_off + align_up(region);
  if (cudaStreamCreateWithFlags(&P->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    hg_batch_plan_destroy(P);
    return HG_ERR_CUDA;
  }
  const hg_status rc = apply_config(P);
  if (rc != HG_OK) {
    hg_batch_plan_destroy(P);
    return rc;
  }
  *out = P;
  return HG_OK;
}

void hg_batch_plan_destroy(hg_batch_plan* P) {
  if (!P) return;
  drop_graph(P);
  if (P->st) cudaStreamDestroy(P->st);
  if (P->ev_in) cudaEventDestroy(P->ev_in);
  if (P->ev_out) cudaEventDestroy(P->ev_out);
  if (P->h_dir) cudaFreeHost(P->h_dir);
  delete P;
}

hg_status hg_batch_layout(const hg_batch_plan* P, uint64_t* h_totals4, uint64_t* h_key_begin,
                          uint64_t* h_query_begin, uint64_t* h_offset_begin) {
  if (!P) return HG_ERR_INVALID_ARG;
  if (h_totals4) {
    h_totals4[0] = P->nk;
    h_totals4[1] = P->nq;
    h_totals4[2] = P->nob + 1;
    h_totals4[3] = P->T;
  }
  if (h_key_begin) std::memcpy(h_key_begin, P->kbeg.data(), (P->T + 1) * 8);
  if (h_query_begin) std::memcpy(h_query_begin, P->qbeg.data(), (P->T + 1) * 8);
  if (h_offset_begin) std::memcpy(h_offset_begin, P->obeg.data(), (P->T + 1) * 8);
  return HG_OK;
}

size_t hg_batch_workspace_size(const hg_batch_plan* P) { return P ? P->ws_total : 0; }

hg_status hg_batch_set_config(hg_batch_plan* P, uint32_t bin_shift, uint32_t threads_per_bin) {
  if (!P) return HG_ERR_INVALID_ARG;
  if (bin_shift > kMaxBinShift) return HG_ERR_INVALID_ARG;
  if (threads_per_bin != 0 && threads_per_bin != 512 && threads_per_bin != 1024) return HG_ERR_UNSUPPORTED;
  const uint32_t ob = P->bin_shift, ot = P->tpb;
  P->bin_shift = bin_shift;
  P->tpb = threads_per_bin;
  const hg_status rc = apply_config(P);
  if (rc != HG_OK) {
    P->bin_shift = ob;
    P->tpb = ot;
    apply_config(P);
  }
  return rc;
}

hg_status hg_batch_get_config(const hg_batch_plan* P, uint32_t* bin_shift, uint32_t* threads_per_bin,
                              uint32_t* waves) {
  if (!P) return HG_ERR_INVALID_ARG;
  if (bin_shift) *bin_shift = effective_shift(P);
  if (threads_per_bin) *threads_per_bin = P->tpb ? P->tpb : 1024u;
  if (waves) *waves = (uint32_t)P->waves.size();
  return HG_OK;
}

hg_status hg_batch_run(hg_batch_plan* P, const void* d_keys, const void* d_queries, uint32_t* d_offsets,
                       void* d_csr_keys, uint32_t* d_csr_ids, uint32_t* d_counts, void* d_ws, size_t ws_bytes,
                       void* stream) {
  if (!P) return HG_ERR_INVALID_ARG;
  const Bufs b{(const uint32_t*)d_keys, (const uint32_t*)d_queries, d_offsets, (uint32_t*)d_csr_keys,
               d_csr_ids, d_counts, (uint8_t*)d_ws};
  const hg_status rc = check_bufs(P, b, ws_bytes);
  if (rc != HG_OK) return rc;
  return run_graph(P, b, (cudaStream_t)stream);
}

hg_status hg_batch_run_eager(hg_batch_plan* P, const void* d_keys, const void* d_queries, uint32_t* d_offsets,
                             void* d_csr_keys, uint32_t* d_csr_ids, uint32_t* d_counts, void* d_ws, size_t ws_bytes,
                             void* stream) {
  if (!P) return HG_ERR_INVALID_ARG;
  const Bufs b{(const uint32_t*)d_keys, (const uint32_t*)d_queries, d_offsets, (uint32_t*)d_csr_keys,
               d_csr_ids, d_counts, (uint8_t*)d_ws};
  const hg_status rc = check_bufs(P, b, ws_bytes);
  if (rc != HG_OK) return rc;
  return enqueue(P, b, (cudaStream_t)stream);
}

hg_status hg_batch_autotune(hg_batch_plan* P, const void* d_keys, const void* d_queries, uint32_t* d_offsets,
                            void* d_csr_keys, uint32_t* d_csr_ids, uint32_t* d_counts, void* d_ws, size_t ws_bytes,
                            void* stream, uint32_t reps, float* h_best_ms) {
  if (!P || reps == 0) return HG_ERR_INVALID_ARG;
  const Bufs b{(const uint32_t*)d_keys, (const uint32_t*)d_queries, d_offsets, (uint32_t*)d_csr_keys,
               d_csr_ids, d_counts, (uint8_t*)d_ws};
  hg_status rc = check_bufs(P, b, ws_bytes);
  if (rc != HG_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HG_ERR_CUDA;
  const int s0 = (int)P->auto_shift;
  float best = 0.f;
  uint32_t best_s = 0, best_t = 0;
  bool have = false;
  for (int s = std::max(0, s0 - 2); s <= std::min<int>(kMaxBinShift, s0 + 1); ++s) {
    for (uint32_t tpb : {512u, 1024u}) {
      if (hg_batch_set_config(P, (uint32_t)s, tpb) != HG_OK) continue;
      rc = run_graph(P, b, st);  // capture + warm-up
      if (rc != HG_OK) break;
      cudaEventRecord(e0, st);
      for (uint32_t r = 0; r < reps && rc == HG_OK; ++r) rc = run_graph(P, b, st);
      cudaEventRecord(e1, st);
      if (rc != HG_OK || cudaEventSynchronize(e1) != cudaSuccess) {
        if (rc == HG_OK) rc = HG_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= (float)reps;
      if (!have || ms < best) {
        have = true;
        best = ms;
        best_s = (uint32_t)s;
        best_t = tpb;
      }
    }
    if (rc != HG_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HG_OK) return rc;
  if (!have) return HG_ERR_UNSUPPORTED;
  rc = hg_batch_set_config(P, best_s, best_t);
  if (rc == HG_OK && h_best_ms) *h_best_ms = best;
  return rc;
}

hg_status hg_batch_run_plain(hg_batch_plan* P, const void* d_keys, const void* d_queries, uint32_t* d_offsets,
                             void* d_csr_keys, uint32_t* d_csr_ids, uint32_t* d_counts, void* d_ws, size_t ws_bytes,
                             void* stream) {
  if (!P) return HG_ERR_INVALID_ARG;
  const Bufs b{(const uint32_t*)d_keys, (const uint32_t*)d_queries, d_offsets, (uint32_t*)d_csr_keys,
               d_csr_ids, d_counts, (uint8_t*)d_ws};
  hg_status rc = check_bufs(P, b, ws_bytes);
  if (rc != HG_OK) return rc;
  uint8_t* R = b.ws + P->region_off;
  const size_t rbytes = ws_bytes - P->region_off;
  for (uint32_t t = 0; t < P->T; ++t) {
    hg_config c = table_config(P, P->V[t], 0, 0);
    c.algo = HG_ALGO_AUTO;
    const uint64_t k0 = P->kbeg[t];
    rc = hg_build(&c, b.keys + k0, nullptr, P->n[t], b.offsets + P->obeg[t], b.csr_k + k0, b.csr_i + k0, R,
                  rbytes, stream);
    if (rc != HG_OK) return rc;
    hg_table tb{};
    tb.n = P->n[t];
    tb.d_offsets = b.offsets + P->obeg[t];
    tb.d_keys = b.csr_k + k0;
    tb.d_ids = b.csr_i + k0;
    rc = hg_probe(&c, &tb, b.queries + P->qbeg[t], P->q[t], b.counts + P->qbeg[t], stream);
    if (rc != HG_OK) return rc;
  }
  return HG_OK;
}

}  // extern "C"
