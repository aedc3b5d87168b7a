// GPU copy of two seeded input recipes of datagen.py, for batches too large
// to draw quickly on the host: the batched uniform keys and the batched
// queries, written straight into the padded batched layout.  Inputs only:
// this library (libhg_datagen.so) holds none of the hash-table method's
// arithmetic and is not part of libhg.so.
//
// Random source, as in datagen.py: SplitMix64 (Steele, Lea and Flood,
// OOPSLA 2014) used counter-based, output i of stream (seed, s) being the
// SplitMix64 finaliser of state0 + (i + 1) * gamma, with state0 the
// finaliser of seed ^ (s * 0xD1B54A32D192ED03); keys are the 32-bit
// scrambler of datagen.py applied to the top 31 bits of an output.
#include <cstdint>

#include <cuda_runtime.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStreamMul = 0xD1B54A32D192ED03ull;
constexpr uint64_t kStreamKeys = 1, kStreamHit = 2, kStreamPick = 3, kStreamMiss = 4;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

inline uint64_t stream_state(uint64_t seed, uint64_t stream) { return mix64(seed ^ (stream * kStreamMul)); }

__device__ inline uint64_t draw(uint64_t state, uint64_t idx) { return mix64(state + (idx + 1) * kGamma); }

__device__ inline uint32_t scramble32(uint64_t x) {
  uint32_t v = (uint32_t)x;
  v ^= v >> 15;
  v *= 0x7A1F3C9Bu;
  v ^= v >> 13;
  v *= 0x5C2E8D17u;
  v ^= v >> 16;
  return v;
}

// table t with beg[t] <= p < beg[t+1] (beg has T+1 entries, non-decreasing)
__device__ inline uint32_t table_of(const uint64_t* beg, uint32_t T, uint64_t p) {
  uint32_t lo = 0, hi = T;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (beg[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_keys(uint32_t* __restrict__ out, uint64_t total, uint32_t T, const uint64_t* __restrict__ pbeg,
                       const uint64_t* __restrict__ ubeg, const uint32_t* __restrict__ len, uint64_t st) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t t = table_of(pbeg, T, p);
    const uint64_t j = p - pbeg[t];
    out[p] = j < len[t] ? scramble32(draw(st, ubeg[t] + j) >> 33) : 0u;
  }
}

__global__ void k_queries(uint32_t* __restrict__ out, uint64_t total, uint32_t T, const uint64_t* __restrict__ qpbeg,
                          const uint64_t* __restrict__ qubeg, const uint32_t* __restrict__ qlen,
                          const uint64_t* __restrict__ kpbeg, const uint32_t* __restrict__ klen,
                          const uint32_t* __restrict__ keys, uint64_t thr, uint64_t st_hit, uint64_t st_pick,
                          uint64_t st_miss) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t t = table_of(qpbeg, T, p);
    const uint64_t j = p - qpbeg[t];
    if (j >= qlen[t]) {
      out[p] = 0u;
      continue;
    }
    const uint64_t u = qubeg[t] + j;
    const uint32_t n = klen[t];
    if (n > 0 && (draw(st_hit, u) >> 11) < thr) {
      const uint64_t pick = ((draw(st_pick, u) >> 32) * (uint64_t)n) >> 32;
      out[p] = keys[kpbeg[t] + pick];
    } else {
      out[p] = scramble32((draw(st_miss, u) >> 33) | (1ull << 31));
    }
  }
}

unsigned grid_for(uint64_t n) {
  const uint64_t b = (n + 255) / 256;
  return (unsigned)(b < 65536 ? (b ? b : 1) : 65536);
}

}  // namespace

extern "C" {

// Keys of every table: table t's len[t] keys at positions pbeg[t].. (device
// arrays pbeg, ubeg of T+1 entries: padded and unpadded first positions);
// key j of table t is datagen.uniform_keys_u32 output ubeg[t] + j.  Padding
// slots get 0.  Returns a cudaError_t.
int hgd_batched_keys_u32(uint64_t seed, uint32_t T, const uint64_t* d_pbeg, const uint64_t* d_ubeg,
                         const uint32_t* d_len, uint64_t total, uint32_t* d_out, void* stream) {
  if (total == 0) return 0;
  k_keys<<<grid_for(total), 256, 0, (cudaStream_t)stream>>>(d_out, total, T, d_pbeg, d_ubeg, d_len,
                                                              stream_state(seed, kStreamKeys));
  return (int)cudaGetLastError();
}

// Queries of every table, as datagen.batched_queries_u32 (query u of the
// unpadded concatenation), written at the padded positions; hits copy a key
// of the table from the padded key array.
int hgd_batched_queries_u32(uint64_t seed, double hit_rate, uint32_t T, const uint64_t* d_qpbeg,
                            const uint64_t* d_qubeg, const uint32_t* d_qlen, const uint64_t* d_kpbeg,
                            const uint32_t* d_klen, const uint32_t* d_keys, uint64_t total, uint32_t* d_out,
                            void* stream) {
  if (total == 0) return 0;
  const double scaled = hit_rate * 9007199254740992.0;  // 2^53
  const uint64_t thr = (uint64_t)(scaled + 0.5);
  k_queries<<<grid_for(total), 256, 0, (cudaStream_t)stream>>>(
      d_out, total, T, d_qpbeg, d_qubeg, d_qlen, d_kpbeg, d_klen, d_keys, thr, stream_state(seed, kStreamHit),
      stream_state(seed, kStreamPick), stream_state(seed, kStreamMiss));
  return (int)cudaGetLastError();
}

}  // extern "C"
