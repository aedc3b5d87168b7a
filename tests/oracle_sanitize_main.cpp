// Test driver for the CPU oracle under AddressSanitizer and
// UndefinedBehaviorSanitizer (tests/test_oracle_sanitized.py compiles it
// together with oracle/*.cpp).  It runs every exported oracle function on
// small seeded inputs -- empty, single-key, ragged, duplicate-heavy, both key
// widths, both bucket maps -- and checks the results against one another
// (offsets end at n, probe counts equal the table-free multiplicity, the
// join count equals the closed form and the number of materialised pairs).
// Any out-of-bounds access or undefined operation aborts the run.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

extern "C" {
uint32_t orc_murmur3_x86_32(const uint8_t* data, uint64_t len, uint32_t seed);
void orc_hash_keys(int key_type, const void* keys, uint64_t n, uint32_t seed, uint32_t* out);
int orc_bucket_keys(int key_type, const void* keys, uint64_t n, int map_kind, uint32_t seed, uint64_t V,
                    const void* model, uint64_t* out);
int orc_bucket_counts(int key_type, const void* keys, uint64_t n, int map_kind, uint32_t seed, uint64_t V,
                      const void* model, uint32_t* counts);
int orc_build(int key_type, const void* keys, const uint32_t* ids, uint64_t n, int map_kind, uint32_t seed,
              uint64_t V, const void* model, uint32_t* offsets, void* csr_keys, uint32_t* csr_ids);
int orc_probe(int key_type, const uint32_t* offsets, const void* csr_keys, uint64_t n, int map_kind, uint32_t seed,
              uint64_t V, const void* model, const void* queries, uint64_t q, uint32_t* counts);
void orc_multiplicity(int key_type, const void* keys, uint64_t n, const void* queries, uint64_t q,
                      uint32_t* counts);
int orc_join_count(int key_type, const uint32_t* offA, const void* keysA, const uint32_t* offB, const void* keysB,
                   uint64_t V, int64_t* bucket_counts, int64_t* total);
int64_t orc_join_size_by_keys(int key_type, const void* keysA, uint64_t nA, const void* keysB, uint64_t nB);
int64_t orc_join_materialize(int key_type, const uint32_t* offA, const void* keysA, const uint32_t* idsA,
                             const uint32_t* offB, const void* keysB, const uint32_t* idsB, uint64_t V,
                             int64_t* out_a, int64_t* out_b, int64_t cap);
void orc_rmi_sample_indices(uint64_t n, uint64_t S, uint64_t seed, uint64_t* idx);
void orc_rmi_sorted_sample(int key_type, const void* keys, uint64_t n, uint64_t S, uint64_t seed, uint64_t* out);
uint32_t orc_rmi_root_leaf(float a, float b, uint32_t L, int key_type, uint64_t key);
uint32_t orc_rmi_knots(float a, float b, uint32_t L, int key_type, uint64_t* kb);
double orc_rmi_leaf_loss_grad(int key_type, const uint64_t* x, uint64_t S, uint64_t V, float a, float b, uint32_t L,
                              const uint64_t* kb, uint32_t J, const double* Y, const double* Y0, double rho,
                              double* grad, double* diag);
void orc_rmi_leaf_init(int key_type, const uint64_t* x, uint64_t S, uint64_t V, uint32_t L, const uint64_t* kb,
                       uint32_t J, double* Y);
void orc_rmi_leaf_train(int key_type, const uint64_t* x, uint64_t S, uint64_t V, float a, float b, uint32_t L,
                        const uint64_t* kb, uint32_t J, const double* Y0, double rho, double gamma, uint32_t iters,
                        double eta, double* Y_out);
void orc_rmi_leaf_project(uint64_t V, uint32_t L, uint32_t J, const double* Y0, double gamma, double* Y);
void orc_rmi_root_lsq(int key_type, const uint64_t* x, uint64_t S, uint32_t L, double* ab);
double orc_rmi_root_loss_grad(int key_type, const uint64_t* x, uint64_t S, uint32_t L, double a, double b, double* g);
}

namespace {

int g_fail = 0;
void check(bool ok, const char* what, uint64_t a = 0, uint64_t b = 0) {
  if (!ok) {
    std::fprintf(stderr, "FAILED: %s (%llu, %llu)\n", what, (unsigned long long)a, (unsigned long long)b);
    ++g_fail;
  }
}

// SplitMix64 (Steele, Lea and Flood 2014): the inputs only.
uint64_t g_state = 0;
uint64_t next_u64() {
  uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Keys of one width as raw bytes; `distinct` values drawn for n keys.
std::vector<uint8_t> make_keys(int kt, uint64_t n, uint64_t distinct) {
  const size_t kb = kt ? 8 : 4;
  std::vector<uint8_t> out(n * kb + 8);
  std::vector<uint64_t> pool(distinct ? distinct : 1);
  for (auto& x : pool) x = next_u64();
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t v = pool[next_u64() % pool.size()];
    if (kt) std::memcpy(&out[i * 8], &v, 8);
    else {
      const uint32_t w = (uint32_t)v;
      std::memcpy(&out[i * 4], &w, 4);
    }
  }
  return out;
}

// A learned-map model blob: header (magic, L, V, a, b, key type, flags) and
// L leaves (xmin, slope, intercept, base, width) that split the key range
// evenly.
std::vector<uint8_t> make_model(int kt, uint32_t L, uint64_t V) {
  std::vector<uint8_t> blob(32 + 24 * (size_t)L, 0);
  const uint32_t magic = 0x4D4C4748u, ktype = (uint32_t)kt, flags = 0;
  // the root maps the feature f(key), about 2^23 (127 + log2 key), of keys
  // from 1 to the largest onto [0, L)
  const double octaves = kt ? 64.0 : 32.0;
  const float a = (float)((double)L / (octaves * 8388608.0)), b = (float)(-127.0 * (double)L / octaves);
  std::memcpy(&blob[0], &magic, 4);
  std::memcpy(&blob[4], &L, 4);
  std::memcpy(&blob[8], &V, 8);
  std::memcpy(&blob[16], &a, 4);
  std::memcpy(&blob[20], &b, 4);
  std::memcpy(&blob[24], &ktype, 4);
  std::memcpy(&blob[28], &flags, 4);
  const double span = kt ? 18446744073709551616.0 : 4294967296.0;
  for (uint32_t j = 0; j < L; ++j) {
    const uint64_t xmin = (uint64_t)(span / L * j);
    const float slope = (float)((double)V / span);
    const float icpt = 0.0f;
    const uint32_t base = (uint32_t)(V * j / L), width = (uint32_t)(V * (j + 1) / L - V * j / L);
    uint8_t* r = &blob[32 + 24 * (size_t)j];
    std::memcpy(r, &xmin, 8);
    std::memcpy(r + 8, &slope, 4);
    std::memcpy(r + 12, &icpt, 4);
    std::memcpy(r + 16, &base, 4);
    std::memcpy(r + 20, &width, 4);
  }
  return blob;
}

void table_case(int kt, uint64_t n, uint64_t V, uint64_t distinct, int map_kind) {
  const size_t kb = kt ? 8 : 4;
  std::vector<uint8_t> keys = make_keys(kt, n, distinct);
  std::vector<uint8_t> model;
  const void* mp = nullptr;
  if (map_kind == 1) {
    model = make_model(kt, 8, V);
    mp = model.data();
  }
  std::vector<uint32_t> off(V + 1), ids(n + 1);
  std::vector<uint8_t> ck(n * kb + 8);
  check(orc_build(kt, keys.data(), nullptr, n, map_kind, 7, V, mp, off.data(), ck.data(), ids.data()) == 0, "build");
  check(off[0] == 0 && off[V] == n, "offsets span", off[V], n);
  for (uint64_t v = 0; v < V; ++v) check(off[v] <= off[v + 1], "offsets monotone", v);
  std::vector<uint32_t> cnt(V);
  check(orc_bucket_counts(kt, keys.data(), n, map_kind, 7, V, mp, cnt.data()) == 0, "bucket counts");
  for (uint64_t v = 0; v < V; ++v) check(cnt[v] == off[v + 1] - off[v], "bucket count = segment", v);
  std::vector<uint64_t> bk(n + 1);
  check(orc_bucket_keys(kt, keys.data(), n, map_kind, 7, V, mp, bk.data()) == 0, "bucket keys");
  // queries: the keys themselves, then as many fresh values (mostly misses)
  const uint64_t q = 2 * n + 3;
  std::vector<uint8_t> qs(q * kb + 8);
  std::memcpy(qs.data(), keys.data(), n * kb);
  std::vector<uint8_t> fresh = make_keys(kt, q - n, q);
  std::memcpy(qs.data() + n * kb, fresh.data(), (q - n) * kb);
  std::vector<uint32_t> pc(q), mc(q);
  check(orc_probe(kt, off.data(), ck.data(), n, map_kind, 7, V, mp, qs.data(), q, pc.data()) == 0, "probe");
  orc_multiplicity(kt, keys.data(), n, qs.data(), q, mc.data());
  for (uint64_t i = 0; i < q; ++i) check(pc[i] == mc[i], "probe = multiplicity", i, pc[i]);
  // join of the table with itself and with the fresh values
  std::vector<int64_t> bc(V);
  int64_t total = -1;
  check(orc_join_count(kt, off.data(), ck.data(), off.data(), ck.data(), V, bc.data(), &total) == 0, "join count");
  check(total == orc_join_size_by_keys(kt, keys.data(), n, keys.data(), n), "join = closed form", (uint64_t)total);
  std::vector<int64_t> pa((size_t)total + 1), pb((size_t)total + 1);
  const int64_t m = orc_join_materialize(kt, off.data(), ck.data(), ids.data(), off.data(), ck.data(), ids.data(), V,
                                         pa.data(), pb.data(), total);
  check(m == total, "materialised pairs", (uint64_t)m, (uint64_t)total);
  if (total > 1) {  // a capacity cut writes only what fits
    const int64_t cut = orc_join_materialize(kt, off.data(), ck.data(), ids.data(), off.data(), ck.data(), ids.data(),
                                             V, pa.data(), pb.data(), total / 2);
    check(cut == total, "pair count independent of capacity", (uint64_t)cut);
  }
}

void learned_case(int kt) {
  const uint64_t n = 3000, S = 300, V = 4096;
  const uint32_t L = 16;
  std::vector<uint8_t> keys = make_keys(kt, n, n);
  std::vector<uint64_t> x(S), idx(S);
  orc_rmi_sample_indices(n, S, 11, idx.data());
  for (uint64_t k = 0; k < S; ++k) check(idx[k] < n, "sample index in range", idx[k]);
  orc_rmi_sorted_sample(kt, keys.data(), n, S, 11, x.data());
  for (uint64_t k = 1; k < S; ++k) check(x[k - 1] <= x[k], "sample sorted", k);
  double ab[2] = {0, 0}, g[2] = {0, 0};
  orc_rmi_root_lsq(kt, x.data(), S, L, ab);
  orc_rmi_root_loss_grad(kt, x.data(), S, L, ab[0], ab[1], g);
  const float a = (float)ab[0], b = (float)ab[1];
  std::vector<uint64_t> kb(L + 1);
  const uint32_t J = orc_rmi_knots(a, b, L, kt, kb.data());
  check(J < L, "last reachable leaf", J);
  for (uint64_t k = 0; k < S; ++k) check(orc_rmi_root_leaf(a, b, L, kt, x[k]) < L, "root leaf in range", k);
  std::vector<double> Y0(L + 1), Y(L + 1), grad(L + 1), diag(L + 1);
  orc_rmi_leaf_init(kt, x.data(), S, V, L, kb.data(), J, Y0.data());
  orc_rmi_leaf_loss_grad(kt, x.data(), S, V, a, b, L, kb.data(), J, Y0.data(), Y0.data(), 1.0, grad.data(),
                         diag.data());
  orc_rmi_leaf_train(kt, x.data(), S, V, a, b, L, kb.data(), J, Y0.data(), 1.0, 0.5, 5, 0.9, Y.data());
  orc_rmi_leaf_project(V, L, J, Y0.data(), 0.5, Y.data());
  for (uint32_t j = 1; j <= J; ++j) check(Y[j] >= Y[j - 1], "projected knots ascend", j);
}

}  // namespace

int main() {
  g_state = 0x4847000Au;
  const uint8_t bytes[8] = {1, 2, 3, 4, 5, 6, 7, 8};
  for (uint64_t len = 0; len <= 8; ++len) (void)orc_murmur3_x86_32(bytes, len, 0x9747b28cu);
  for (int kt = 0; kt < 2; ++kt) {
    std::vector<uint8_t> k = make_keys(kt, 17, 17);
    std::vector<uint32_t> h(17);
    orc_hash_keys(kt, k.data(), 17, 3, h.data());
    for (int map_kind = 0; map_kind < 2; ++map_kind) {
      table_case(kt, 0, 64, 1, map_kind);        // empty input
      table_case(kt, 1, 1, 1, map_kind);         // one key, one bucket
      table_case(kt, 1000, 1, 1000, map_kind);   // every key in one bucket
      table_case(kt, 2001, 97, 2001, map_kind);  // ragged, V not a power of two
      table_case(kt, 4096, 4096, 64, map_kind);  // duplicate-heavy
      table_case(kt, 5003, 1024, 5003, map_kind);
    }
    learned_case(kt);
  }
  if (g_fail) {
    std::fprintf(stderr, "%d checks failed\n", g_fail);
    return 1;
  }
  std::printf("oracle checks passed under the sanitizers\n");
  return 0;
}
