// HashGraph CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded restatement of what the HashGraph method
// computes (Green, "HashGraph - Scalable Hash Tables Using A Sparse Graph Data
// Structure", 2019).  Only the test-suite, the smoke check and the benchmark's
// CPU-baseline leg may load this library.  It shares no code, header, table or
// constant with the CUDA library: every formula below is written out again
// from the paper (and, for the hash function and the learned bucket map, from
// their published definitions).
//
// Conventions
//   * key_type 0 = uint32 keys, 1 = uint64 keys (little-endian bytes).
//   * A table is in CSR form (Section 3.1, "Compressed Sparse Row"):
//     offsets[0..V], keys[0..n), ids[0..n); bucket v owns [offsets[v], offsets[v+1]).
//   * Order inside a bucket: ascending input position (the paper leaves it open,
//     Section 5.1 notes V1 and V2 may differ; we fix one canonical order so that
//     every variant is comparable bit for bit).
//
// Build with:  g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared
// (-ffp-contract=off: the learned map's fp32 arithmetic must not be fused.)

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// MurmurHash3, 32-bit x86 variant (Appleby; the hash family the paper uses,
// Section 2 "Hashing", Eq. 1).  Written from the published algorithm: 4-byte
// blocks mixed with two multiplications and a rotation, a tail, the length,
// then the 32-bit finaliser.
// ---------------------------------------------------------------------------
inline uint32_t rotl(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

uint32_t murmur3_x86_32(const uint8_t* p, uint64_t len, uint32_t seed) {
  const uint32_t m1 = 0xcc9e2d51u;
  const uint32_t m2 = 0x1b873593u;
  uint32_t h = seed;
  const uint64_t blocks = len / 4;
  for (uint64_t b = 0; b < blocks; ++b) {
    uint32_t k = (uint32_t)p[4 * b] | ((uint32_t)p[4 * b + 1] << 8) |
                 ((uint32_t)p[4 * b + 2] << 16) | ((uint32_t)p[4 * b + 3] << 24);
    k *= m1;
    k = rotl(k, 15);
    k *= m2;
    h ^= k;
    h = rotl(h, 13);
    h = h * 5u + 0xe6546b64u;
  }
  const uint8_t* t = p + 4 * blocks;
  uint32_t k = 0;
  switch (len & 3) {
    case 3: k ^= (uint32_t)t[2] << 16; [[fallthrough]];
    case 2: k ^= (uint32_t)t[1] << 8; [[fallthrough]];
    case 1:
      k ^= (uint32_t)t[0];
      k *= m1;
      k = rotl(k, 15);
      k *= m2;
      h ^= k;
  }
  h ^= (uint32_t)len;
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

uint64_t key_at(int key_type, const void* keys, uint64_t i) {
  if (key_type == 0) return ((const uint32_t*)keys)[i];
  return ((const uint64_t*)keys)[i];
}

uint32_t hash_key(int key_type, uint64_t key, uint32_t seed) {
  uint8_t b[8];
  for (int i = 0; i < 8; ++i) b[i] = (uint8_t)(key >> (8 * i));
  return murmur3_x86_32(b, key_type == 0 ? 4 : 8, seed);
}

// ---------------------------------------------------------------------------
// Learned bucket map (not in the paper; the paper uses Murmur only).  A
// two-layer piecewise-linear CDF model: a linear root picks one of L leaves
// from a monotone log-like feature of the key, and leaf j maps its key range
// linearly onto its bucket range [base_j, base_j + width_j).  Inference is
// fp32 with round-to-nearest and no fused multiply-add, so the CPU and GPU
// results agree bit for bit.  Blob layout (little-endian):
//   header 32 B: u32 magic 'HGLM', u32 L, u64 V, f32 root_a, f32 root_b,
//                u32 key_type, u32 flags
//   leaf   24 B: u64 xmin, f32 slope, f32 icpt, u32 base, u32 width
// ---------------------------------------------------------------------------
struct LeafRec {
  uint64_t xmin;
  float slope;
  float icpt;
  uint32_t base;
  uint32_t width;
};
static_assert(sizeof(LeafRec) == 24, "leaf record layout");

struct Model {
  uint32_t L = 0;
  uint64_t V = 0;
  float a = 0, b = 0;
  uint32_t key_type = 0;
  const LeafRec* leaf = nullptr;
};

bool parse_model(const void* blob, Model& m) {
  const uint8_t* p = (const uint8_t*)blob;
  uint32_t magic;
  std::memcpy(&magic, p, 4);
  if (magic != 0x4D4C4748u) return false;  // bytes 'H','G','L','M'
  std::memcpy(&m.L, p + 4, 4);
  std::memcpy(&m.V, p + 8, 8);
  std::memcpy(&m.a, p + 16, 4);
  std::memcpy(&m.b, p + 20, 4);
  std::memcpy(&m.key_type, p + 24, 4);
  m.leaf = (const LeafRec*)(p + 32);
  return m.L > 0;
}

// Monotone feature: the key rounded to fp32, its IEEE bit pattern read as an
// unsigned integer (roughly 2^23 * (127 + log2 key)), rounded to fp32 again.
float rmi_feature(int key_type, uint64_t key) {
  float fk = key_type == 0 ? (float)(uint32_t)key : (float)key;
  uint32_t bits;
  std::memcpy(&bits, &fk, 4);
  return (float)bits;
}

uint32_t rmi_root(const Model& m, uint64_t key) {
  volatile float f = rmi_feature((int)m.key_type, key);
  volatile float prod = m.a * f;
  volatile float r = prod + m.b;
  float rr = r;
  if (!(rr >= 0.0f)) return 0;
  if (rr >= (float)m.L) return m.L - 1;
  return (uint32_t)rr;
}

uint64_t rmi_bucket(const Model& m, uint64_t key) {
  const LeafRec& lf = m.leaf[rmi_root(m, key)];
  uint32_t local = 0;
  if (lf.width > 0) {
    uint64_t d = key > lf.xmin ? key - lf.xmin : 0;
    volatile float x = (float)d;
    volatile float prod = lf.slope * x;
    volatile float p = prod + lf.icpt;
    float pp = p;
    if (!(pp >= 0.0f)) local = 0;
    else if (pp >= (float)lf.width) local = lf.width - 1;
    else local = std::min((uint32_t)pp, lf.width - 1);
  }
  uint64_t bkt = (uint64_t)lf.base + local;
  return bkt < m.V ? bkt : m.V - 1;
}

struct Map {
  int kind = 0;  // 0 murmur3, 1 learned
  uint32_t seed = 0;
  uint64_t V = 1;
  Model model;
};

// Bucket of a key (Eq. 1: hash(a) mod V, or the learned map).
uint64_t bucket_of(const Map& mp, int key_type, uint64_t key) {
  if (mp.kind == 1) return rmi_bucket(mp.model, key);
  return (uint64_t)hash_key(key_type, key, mp.seed) % mp.V;
}

bool make_map(int kind, uint32_t seed, uint64_t V, const void* model, Map& mp) {
  mp.kind = kind;
  mp.seed = seed;
  mp.V = V;
  if (V == 0) return false;
  if (kind == 1) {
    if (!model || !parse_model(model, mp.model)) return false;
    if (mp.model.V != V) return false;
  }
  return true;
}

}  // namespace

extern "C" {

uint32_t orc_murmur3_x86_32(const uint8_t* data, uint64_t len, uint32_t seed) {
  return murmur3_x86_32(data, len, seed);
}

// Raw 32-bit hash of every key (no reduction).
void orc_hash_keys(int key_type, const void* keys, uint64_t n, uint32_t seed, uint32_t* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = hash_key(key_type, key_at(key_type, keys, i), seed);
}

// Bucket of every key under the map (murmur3 mod V, or the learned model).
int orc_bucket_keys(int key_type, const void* keys, uint64_t n, int map_kind, uint32_t seed,
                    uint64_t V, const void* model, uint64_t* out) {
  Map mp;
  if (!make_map(map_kind, seed, V, model, mp)) return 1;
  for (uint64_t i = 0; i < n; ++i) out[i] = bucket_of(mp, key_type, key_at(key_type, keys, i));
  return 0;
}

// Number of keys in every bucket (the histogram the build's prefix sum turns
// into the CSR offsets, Alg. 1 and Section 3.1), for key sets too large to
// keep one bucket per key in memory.  counts: V entries, overwritten.
int orc_bucket_counts(int key_type, const void* keys, uint64_t n, int map_kind, uint32_t seed, uint64_t V,
                      const void* model, uint32_t* counts) {
  Map mp;
  if (!make_map(map_kind, seed, V, model, mp)) return 1;
  for (uint64_t v = 0; v < V; ++v) counts[v] = 0;
  for (uint64_t i = 0; i < n; ++i) ++counts[bucket_of(mp, key_type, key_at(key_type, keys, i))];
  return 0;
}

// HashGraph build (Alg. 1 / Alg. 2 define the same table): the table is the
// input grouped by bucket.  Definition used here: sort input positions by
// (bucket, position); offsets[v] = number of keys whose bucket is below v.
int orc_build(int key_type, const void* keys, const uint32_t* ids, uint64_t n, int map_kind,
              uint32_t seed, uint64_t V, const void* model, uint32_t* offsets, void* csr_keys,
              uint32_t* csr_ids) {
  Map mp;
  if (!make_map(map_kind, seed, V, model, mp)) return 1;
  std::vector<uint64_t> b(n);
  for (uint64_t i = 0; i < n; ++i) b[i] = bucket_of(mp, key_type, key_at(key_type, keys, i));
  std::vector<uint64_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::sort(perm.begin(), perm.end(), [&](uint64_t x, uint64_t y) {
    return b[x] < b[y] || (b[x] == b[y] && x < y);
  });
  std::vector<uint64_t> sorted_b(n);
  for (uint64_t j = 0; j < n; ++j) sorted_b[j] = b[perm[j]];
  for (uint64_t v = 0; v <= V; ++v)
    offsets[v] = (uint32_t)(std::lower_bound(sorted_b.begin(), sorted_b.end(), v) - sorted_b.begin());
  for (uint64_t j = 0; j < n; ++j) {
    if (key_type == 0)
      ((uint32_t*)csr_keys)[j] = ((const uint32_t*)keys)[perm[j]];
    else
      ((uint64_t*)csr_keys)[j] = ((const uint64_t*)keys)[perm[j]];
    csr_ids[j] = ids ? ids[perm[j]] : (uint32_t)perm[j];
  }
  return 0;
}

// HashGraph-Probe-Standard (Section 3.4): hash the query, scan its bucket,
// count every instance of the query key.
int orc_probe(int key_type, const uint32_t* offsets, const void* csr_keys, uint64_t n,
              int map_kind, uint32_t seed, uint64_t V, const void* model, const void* queries,
              uint64_t q, uint32_t* counts) {
  Map mp;
  if (!make_map(map_kind, seed, V, model, mp)) return 1;
  (void)n;
  for (uint64_t i = 0; i < q; ++i) {
    uint64_t key = key_at(key_type, queries, i);
    uint64_t v = bucket_of(mp, key_type, key);
    uint32_t c = 0;
    for (uint64_t j = offsets[v]; j < offsets[v + 1]; ++j) c += key_at(key_type, csr_keys, j) == key;
    counts[i] = c;
  }
  return 0;
}

// Table-free definition of the probe result: multiplicity of each query in
// the build input (sorted copy + equal_range).  Used to pin orc_probe.
void orc_multiplicity(int key_type, const void* keys, uint64_t n, const void* queries, uint64_t q,
                      uint32_t* counts) {
  std::vector<uint64_t> s(n);
  for (uint64_t i = 0; i < n; ++i) s[i] = key_at(key_type, keys, i);
  std::sort(s.begin(), s.end());
  for (uint64_t i = 0; i < q; ++i) {
    auto r = std::equal_range(s.begin(), s.end(), key_at(key_type, queries, i));
    counts[i] = (uint32_t)(r.second - r.first);
  }
}

// HashGraph-Probe-New (Alg. 3): for every bucket v, intersect A's and B's
// adjacency arrays; the result per bucket is the number of equal-key pairs.
int orc_join_count(int key_type, const uint32_t* offA, const void* keysA, const uint32_t* offB,
                   const void* keysB, uint64_t V, int64_t* bucket_counts, int64_t* total) {
  int64_t t = 0;
  for (uint64_t v = 0; v < V; ++v) {
    int64_t c = 0;
    for (uint64_t a = offA[v]; a < offA[v + 1]; ++a) {
      uint64_t ka = key_at(key_type, keysA, a);
      for (uint64_t b = offB[v]; b < offB[v + 1]; ++b) c += ka == key_at(key_type, keysB, b);
    }
    if (bucket_counts) bucket_counts[v] = c;
    t += c;
  }
  *total = t;
  return 0;
}

// Closed form of the join size: sum over distinct keys of m_A(k) * m_B(k)
// (both inputs sorted, then merged).  Used to pin orc_join_count.
int64_t orc_join_size_by_keys(int key_type, const void* keysA, uint64_t nA, const void* keysB,
                              uint64_t nB) {
  std::vector<uint64_t> a(nA), b(nB);
  for (uint64_t i = 0; i < nA; ++i) a[i] = key_at(key_type, keysA, i);
  for (uint64_t i = 0; i < nB; ++i) b[i] = key_at(key_type, keysB, i);
  std::sort(a.begin(), a.end());
  std::sort(b.begin(), b.end());
  int64_t t = 0;
  uint64_t i = 0, j = 0;
  while (i < nA && j < nB) {
    if (a[i] < b[j]) { ++i; continue; }
    if (b[j] < a[i]) { ++j; continue; }
    uint64_t k = a[i], ca = 0, cb = 0;
    while (i < nA && a[i] == k) { ++i; ++ca; }
    while (j < nB && b[j] == k) { ++j; ++cb; }
    t += (int64_t)(ca * cb);
  }
  return t;
}

// Join materialisation in the canonical order: bucket ascending, then A's
// CSR position, then B's CSR position; each equal-key pair emits
// (A id, B id).  Returns the number of pairs (writes at most cap of them).
int64_t orc_join_materialize(int key_type, const uint32_t* offA, const void* keysA,
                             const uint32_t* idsA, const uint32_t* offB, const void* keysB,
                             const uint32_t* idsB, uint64_t V, int64_t* out_a, int64_t* out_b,
                             int64_t cap) {
  int64_t m = 0;
  for (uint64_t v = 0; v < V; ++v)
    for (uint64_t a = offA[v]; a < offA[v + 1]; ++a) {
      uint64_t ka = key_at(key_type, keysA, a);
      for (uint64_t b = offB[v]; b < offB[v + 1]; ++b)
        if (ka == key_at(key_type, keysB, b)) {
          if (m < cap) {
            out_a[m] = idsA[a];
            out_b[m] = idsB[b];
          }
          ++m;
        }
    }
  return m;
}

}  // extern "C"
