// Multithreaded CPU HashGraph: a CPU comparison point for the GPU path, not
// part of it and not the oracle (the oracle is single-threaded and plain).
// It shares no code with either.
//
// Build: HashGraph-V2 (Alg. 2, Section 3.3) with OpenMP.
//   Phase 1: every input chunk hashes its keys (Eq. 1: MurmurHash3_x86_32 of
//            the key's little-endian bytes, mod V) and counts them per bin of
//            2^s consecutive buckets.
//   Phase 2: exclusive scan of the (bin, chunk) counts, bin-major, so that
//            chunk c's elements of bin b follow those of chunks 0 .. c-1.
//   Phase 3: every chunk scatters (key, id, bucket) to its bin cursors; the
//            reorganised array holds each bin in input order.
//   Phase 4: bins in parallel: bucket counts, exclusive scan into the CSR
//            offsets, then an in-order scatter of the bin's edges.
// The result is the canonical table: offsets[V+1], and inside each bucket
// the edges in ascending input position (the order the GPU build and the
// oracle produce), so it can be compared byte for byte.
//
// Probe: HashGraph-Probe-Standard (Section 3.4): for every query, the number
// of equal keys in its bucket, queries split statically across threads.
#include <omp.h>

#include <algorithm>
#include <cstdint>
#include <memory>
#include <vector>

namespace {

inline uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

// MurmurHash3_x86_32 (Appleby's published algorithm) of a 4- or 8-byte key:
// one 4-byte block per 32 bits, lowest bytes first, no tail, length mixed in.
template <typename K>
inline uint32_t murmur3(K key, uint32_t seed) {
  constexpr uint32_t c1 = 0xcc9e2d51u, c2 = 0x1b873593u;
  const uint64_t v = (uint64_t)key;
  uint32_t h = seed;
  for (int blk = 0; blk < (int)(sizeof(K) / 4); ++blk) {
    uint32_t k = (uint32_t)(v >> (32 * blk));
    k *= c1;
    k = rotl32(k, 15);
    k *= c2;
    h ^= k;
    h = rotl32(h, 13);
    h = h * 5u + 0xe6546b64u;
  }
  h ^= (uint32_t)sizeof(K);
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

template <typename K>
inline uint32_t bucket_of(K key, uint32_t seed, uint64_t V) {
  return (uint32_t)((uint64_t)murmur3<K>(key, seed) % V);
}

int team(int threads) { return threads > 0 ? threads : omp_get_max_threads(); }

// Buckets per bin: 2^s with about 8192 edges per bin on average (a bin's
// keys, ids and bucket counters then stay in a core's L2), and at most 2^20
// buckets so that every thread's bucket counters stay small.
int bin_shift(uint64_t n, uint64_t V) {
  int s = 0;
  while (s < 20 && ((uint64_t)1 << (s + 1)) <= V && (n << (s + 1)) / V <= 8192) ++s;
  return s;
}

template <typename K>
int build_impl(const K* keys, const uint32_t* ids, uint64_t n, uint64_t V, uint32_t seed, uint32_t* offsets,
               K* csr_keys, uint32_t* csr_ids, int threads) {
  if (n == 0) {
    for (uint64_t v = 0; v <= V; ++v) offsets[v] = 0;
    return 0;
  }
  const int T = (int)std::min<uint64_t>((uint64_t)team(threads), n);
  const int s = bin_shift(n, V);
  const uint64_t nbins = ((V - 1) >> s) + 1;
  // Per-key arrays are left uninitialised: each is first written inside a
  // parallel phase, so its pages are touched by all threads, not zeroed by one.
  std::unique_ptr<uint32_t[]> bk(new uint32_t[n]);   // bucket of every input key
  std::vector<uint32_t> cnt((size_t)T * nbins, 0);   // (chunk, bin) counts, then cursors
  auto chunk_lo = [&](int c) { return n * (uint64_t)c / (uint64_t)T; };

  // Phase 1
#pragma omp parallel for num_threads(T) schedule(static, 1)
  for (int c = 0; c < T; ++c) {
    uint32_t* h = cnt.data() + (size_t)c * nbins;
    for (uint64_t i = chunk_lo(c); i < chunk_lo(c + 1); ++i) {
      const uint32_t b = bucket_of<K>(keys[i], seed, V);
      bk[i] = b;
      ++h[b >> s];
    }
  }
  // Phase 2 (bin-major: bin b of chunk c starts after bin b of chunks < c)
  std::vector<uint64_t> bin_start(nbins + 1);
  uint64_t run = 0;
  for (uint64_t b = 0; b < nbins; ++b) {
    bin_start[b] = run;
    for (int c = 0; c < T; ++c) {
      uint32_t& x = cnt[(size_t)c * nbins + b];
      const uint32_t k = x;
      x = (uint32_t)run;
      run += k;
    }
  }
  bin_start[nbins] = run;
  // Phase 3
  std::unique_ptr<K[]> rk(new K[n]);
  std::unique_ptr<uint32_t[]> ri(new uint32_t[n]), rb(new uint32_t[n]);
#pragma omp parallel for num_threads(T) schedule(static, 1)
  for (int c = 0; c < T; ++c) {
    uint32_t* cur = cnt.data() + (size_t)c * nbins;
    for (uint64_t i = chunk_lo(c); i < chunk_lo(c + 1); ++i) {
      const uint32_t b = bk[i];
      const uint32_t p = cur[b >> s]++;
      rk[p] = keys[i];
      ri[p] = ids ? ids[i] : (uint32_t)i;
      rb[p] = b;
    }
  }
  // Phase 4
#pragma omp parallel num_threads(T)
  {
    std::vector<uint32_t> lc(((size_t)1 << s) + 1);
#pragma omp for schedule(dynamic, 8)
    for (int64_t bi = 0; bi < (int64_t)nbins; ++bi) {
      const uint64_t b0 = (uint64_t)bi << s;
      const uint64_t nb = std::min<uint64_t>((uint64_t)1 << s, V - b0);
      const uint64_t e0 = bin_start[bi], e1 = bin_start[bi + 1];
      std::fill(lc.begin(), lc.begin() + nb, 0u);
      for (uint64_t e = e0; e < e1; ++e) ++lc[rb[e] - b0];
      uint32_t acc = (uint32_t)e0;
      for (uint64_t j = 0; j < nb; ++j) {
        const uint32_t k = lc[j];
        offsets[b0 + j] = acc;
        lc[j] = acc;
        acc += k;
      }
      for (uint64_t e = e0; e < e1; ++e) {
        const uint32_t p = lc[rb[e] - b0]++;
        csr_keys[p] = rk[e];
        csr_ids[p] = ri[e];
      }
    }
  }
  offsets[V] = (uint32_t)n;
  return 0;
}

template <typename K>
int probe_impl(const uint32_t* offsets, const K* csr_keys, uint64_t V, uint32_t seed, const K* queries,
               uint64_t q, uint32_t* counts, int threads) {
  const int T = team(threads);
#pragma omp parallel for num_threads(T) schedule(static)
  for (int64_t i = 0; i < (int64_t)q; ++i) {
    const K x = queries[i];
    const uint32_t b = bucket_of<K>(x, seed, V);
    uint32_t c = 0;
    for (uint32_t j = offsets[b]; j < offsets[b + 1]; ++j) c += csr_keys[j] == x;
    counts[i] = c;
  }
  return 0;
}

bool bad_sizes(uint64_t n, uint64_t V) { return V == 0 || V > ((uint64_t)1 << 32) || n >= ((uint64_t)1 << 32); }

}  // namespace

extern "C" {

// 0 = done, 1 = invalid argument (key_type not 0/1, V = 0 or > 2^32,
// n >= 2^32, a null array that is needed).  key_type 0: uint32 keys,
// 1: uint64 keys.  ids may be null (ids = input positions).  threads <= 0:
// the OpenMP default.  offsets has V+1 entries; csr_keys and csr_ids n.
int hgcpu_build(int key_type, const void* keys, const uint32_t* ids, uint64_t n, uint64_t V, uint32_t seed,
                uint32_t* offsets, void* csr_keys, uint32_t* csr_ids, int threads) {
  if ((key_type != 0 && key_type != 1) || bad_sizes(n, V) || !offsets || (n > 0 && (!keys || !csr_keys || !csr_ids)))
    return 1;
  if (key_type == 0)
    return build_impl<uint32_t>((const uint32_t*)keys, ids, n, V, seed, offsets, (uint32_t*)csr_keys, csr_ids,
                                threads);
  return build_impl<uint64_t>((const uint64_t*)keys, ids, n, V, seed, offsets, (uint64_t*)csr_keys, csr_ids,
                              threads);
}

// counts[i] = number of keys equal to queries[i] in its bucket of the table
// (offsets[V+1], csr_keys) built with the same V and seed.
int hgcpu_probe(int key_type, const uint32_t* offsets, const void* csr_keys, uint64_t V, uint32_t seed,
                const void* queries, uint64_t q, uint32_t* counts, int threads) {
  if ((key_type != 0 && key_type != 1) || V == 0 || V > ((uint64_t)1 << 32) || !offsets ||
      (q > 0 && (!queries || !counts)))
    return 1;
  if (key_type == 0)
    return probe_impl<uint32_t>(offsets, (const uint32_t*)csr_keys, V, seed, (const uint32_t*)queries, q, counts,
                                threads);
  return probe_impl<uint64_t>(offsets, (const uint64_t*)csr_keys, V, seed, (const uint64_t*)queries, q, counts,
                              threads);
}

int hgcpu_max_threads(void) { return omp_get_max_threads(); }

}  // extern "C"
