// HashGraph CPU oracle, learned bucket map -- TEST INFRASTRUCTURE ONLY.
//
// The learned map is not in the paper (the paper hashes with Murmur,
// Section 2).  It replaces "hash(a) mod V" by an order-preserving,
// piecewise-linear model of the key CDF:
//   root:   leaf j = clamp(floor(a * f(x) + b), 0, L-1), f(x) a monotone
//           log-like feature of the key (see hg_oracle.cpp)
//   knots:  kb_j = smallest key the root sends to leaf j or beyond
//           (kb_0 = 0); leaf j owns the keys [kb_j, kb_{j+1})
//   spline: the bucket position of x in leaf j is
//           Y_j + (Y_{j+1} - Y_j) * (x - kb_j) / (kb_{j+1} - kb_j),
//           with knot values Y_0 = 0 <= Y_1 <= ... <= Y_L = V
// Prior: the knot values Y0 of the piecewise-linear interpolant of the
// sample's rank targets, through (0, 0), (x_i, V (2i+1) / (2S)) for the
// sorted sample x_0..x_{S-1}, and (key max + 1, V).
// Training fits the knot values to the sample's rank targets:
//   loss(Y) = (1/S) [ sum_i (P(x_i) - V (2i+1) / (2S))^2
//                     + rho * sum_{j=1..J} (Y_j - Y0_j)^2 ]
// by Jacobi-preconditioned gradient steps, each followed by the projection
// onto the knot values that keep every leaf at least gamma times as wide (in
// buckets) as the prior makes it:  Y_j - Y_{j-1} >= gamma (Y0_j - Y0_{j-1}).
// The ridge rho makes the minimiser unique where knots see few samples; the
// width floor keeps leaves that the sample barely sees from collapsing onto
// one bucket.
// This file computes, in double precision and in the plainest way:
//   * the sample indices (SplitMix64, counter-based, as published by Steele,
//     Lea and Flood 2014) and the sorted sample,
//   * the knots of a given root by bisection on the exact fp32 root,
//   * the loss, its gradient and the diagonal of its Hessian,
//   * the prior, the training iteration with its projection,
//   * the exact least-squares knot values without the projection
//     (tridiagonal normal equations),
//   * the root least-squares fit and its gradient.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

uint64_t sm_finalize(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
const uint64_t kGolden = 0x9E3779B97F4A7C15ull;
const uint64_t kSampleStream = 0x4C4541524Eull;  // stream id of the learned-map sample

// Same monotone feature and root as hg_oracle.cpp (fp32, round to nearest, unfused).
float feature(int key_type, uint64_t key) {
  float fk = key_type == 0 ? (float)(uint32_t)key : (float)key;
  uint32_t bits;
  std::memcpy(&bits, &fk, 4);
  return (float)bits;
}
uint32_t root_leaf(float a, float b, uint32_t L, int key_type, uint64_t key) {
  volatile float f = feature(key_type, key);
  volatile float prod = a * f;
  volatile float r = prod + b;
  float rr = r;
  if (!(rr >= 0.0f)) return 0;
  if (rr >= (float)L) return L - 1;
  return (uint32_t)rr;
}
uint64_t key_max(int key_type) { return key_type == 0 ? 0xFFFFFFFFull : ~0ull; }

}  // namespace

extern "C" {

// Sample indices: idx_k = floor(n * (x_k >> 32) / 2^32), x_k the k-th output
// of SplitMix64 stream kSampleStream under `seed` (n <= 2^32).
void orc_rmi_sample_indices(uint64_t n, uint64_t S, uint64_t seed, uint64_t* idx) {
  const uint64_t st = sm_finalize(seed ^ (kSampleStream * 0xD1B54A32D192ED03ull));
  for (uint64_t k = 0; k < S; ++k) {
    const uint64_t x = sm_finalize(st + (k + 1) * kGolden);
    idx[k] = ((x >> 32) * n) >> 32;
  }
}

// Sorted sample of the keys.
void orc_rmi_sorted_sample(int key_type, const void* keys, uint64_t n, uint64_t S, uint64_t seed, uint64_t* out) {
  std::vector<uint64_t> idx(S);
  orc_rmi_sample_indices(n, S, seed, idx.data());
  for (uint64_t k = 0; k < S; ++k)
    out[k] = key_type == 0 ? ((const uint32_t*)keys)[idx[k]] : ((const uint64_t*)keys)[idx[k]];
  std::sort(out, out + S);
}

uint32_t orc_rmi_root_leaf(float a, float b, uint32_t L, int key_type, uint64_t key) {
  return root_leaf(a, b, L, key_type, key);
}

// Knots.  J = root(max key) is the last leaf any key reaches.  kb[0] = 0;
// for 1 <= j <= J, kb[j] = smallest key with root(key) >= j (bisection: the
// root is non-decreasing in the key); kb[j] = max key for j > J.  Leaf j <= J
// owns [kb[j], R_j) with R_j = kb[j+1] for j < J and R_J = max key + 1.
// Returns J.
uint32_t orc_rmi_knots(float a, float b, uint32_t L, int key_type, uint64_t* kb) {
  const uint64_t hi_key = key_max(key_type);
  const uint32_t J = root_leaf(a, b, L, key_type, hi_key);
  kb[0] = 0;
  for (uint32_t j = 1; j <= L; ++j) {
    if (j > J) {
      kb[j] = hi_key;
      continue;
    }
    uint64_t lo = 0, hi = hi_key;  // invariant: root(hi) >= j
    while (lo < hi) {
      const uint64_t mid = lo + ((hi - lo) >> 1);
      if (root_leaf(a, b, L, key_type, mid) >= j) hi = mid; else lo = mid + 1;
    }
    kb[j] = lo;
  }
  return J;
}

// Leaf (the root's choice) and position lambda = (x - kb_j) / (R_j - kb_j)
// of every sorted sample.
static void leaf_coords(int key_type, const uint64_t* x, uint64_t S, float a, float b, uint32_t L,
                        const uint64_t* kb, uint32_t J, std::vector<uint32_t>& leaf, std::vector<double>& lam) {
  leaf.resize(S);
  lam.resize(S);
  for (uint64_t i = 0; i < S; ++i) {
    const uint32_t j = root_leaf(a, b, L, key_type, x[i]);
    const double w = j < J ? (double)(kb[j + 1] - kb[j]) : (double)(key_max(key_type) - kb[j]) + 1.0;
    leaf[i] = j;
    lam[i] = w > 0.0 ? (double)(x[i] - kb[j]) / w : 0.0;
  }
}

// Loss, gradient dL/dY_j and Hessian diagonal d2L/dY_j^2 of the spline fit
// (Y has L+1 entries; all L+1 partials are returned; the ridge term applies
// to the free knots 1..J).
double orc_rmi_leaf_loss_grad(int key_type, const uint64_t* x, uint64_t S, uint64_t V, float a, float b,
                              uint32_t L, const uint64_t* kb, uint32_t J, const double* Y, const double* Y0,
                              double rho, double* grad, double* diag) {
  std::vector<uint32_t> leaf;
  std::vector<double> lam;
  leaf_coords(key_type, x, S, a, b, L, kb, J, leaf, lam);
  for (uint32_t j = 0; j <= L; ++j) grad[j] = diag[j] = 0.0;
  double loss = 0.0;
  for (uint64_t i = 0; i < S; ++i) {
    const uint32_t j = leaf[i];
    const double l = lam[i];
    const double pred = (1.0 - l) * Y[j] + l * Y[j + 1];
    const double target = (double)V * (2.0 * (double)i + 1.0) / (2.0 * (double)S);
    const double r = pred - target;
    loss += r * r;
    grad[j] += 2.0 * r * (1.0 - l);
    grad[j + 1] += 2.0 * r * l;
    diag[j] += 2.0 * (1.0 - l) * (1.0 - l);
    diag[j + 1] += 2.0 * l * l;
  }
  for (uint32_t j = 1; j <= J; ++j) {
    const double d = Y[j] - Y0[j];
    loss += rho * d * d;
    grad[j] += 2.0 * rho * d;
    diag[j] += 2.0 * rho;
  }
  for (uint32_t j = 0; j <= L; ++j) {
    grad[j] /= (double)S;
    diag[j] /= (double)S;
  }
  return loss / (double)S;
}

// Exact minimiser of the loss over the free knots Y_1..Y_J, with Y_0 = 0 and
// Y_j = V for j > J: the normal equations are tridiagonal (each sample
// touches two knots) and, with rho > 0, strictly positive definite.
// Thomas algorithm in double.
void orc_rmi_leaf_lsq(int key_type, const uint64_t* x, uint64_t S, uint64_t V, float a, float b, uint32_t L,
                      const uint64_t* kb, uint32_t J, const double* Y_init, double rho, double* Y_out) {
  std::vector<uint32_t> leaf;
  std::vector<double> lam;
  leaf_coords(key_type, x, S, a, b, L, kb, J, leaf, lam);
  std::vector<double> dg(L + 1, 0.0), off(L + 1, 0.0), rhs(L + 1, 0.0);  // off[j] = A(j, j+1)
  for (uint64_t i = 0; i < S; ++i) {
    const uint32_t j = leaf[i];
    const double l = lam[i];
    const double t = (double)V * (2.0 * (double)i + 1.0) / (2.0 * (double)S);
    dg[j] += (1.0 - l) * (1.0 - l);
    dg[j + 1] += l * l;
    off[j] += (1.0 - l) * l;
    rhs[j] += (1.0 - l) * t;
    rhs[j + 1] += l * t;
  }
  std::vector<int> freev(L + 1, 0);
  for (uint32_t j = 0; j <= L; ++j) {
    Y_out[j] = j == 0 ? 0.0 : (j > J ? (double)V : Y_init[j]);
    freev[j] = j >= 1 && j <= J && dg[j] + rho > 0.0;
    if (freev[j]) {
      dg[j] += rho;
      rhs[j] += rho * Y_init[j];
    }
  }
  std::vector<double> bb(L + 1, 0.0);
  for (uint32_t j = 1; j <= J; ++j) {
    if (!freev[j]) continue;
    bb[j] = rhs[j];
    if (!freev[j - 1]) bb[j] -= off[j - 1] * Y_out[j - 1];
    if (j + 1 <= L && !freev[j + 1]) bb[j] -= off[j] * Y_out[j + 1];
  }
  uint32_t j = 1;
  while (j <= J) {
    if (!freev[j]) { ++j; continue; }
    uint32_t e = j;
    while (e + 1 <= J && freev[e + 1]) ++e;
    const uint32_t m = e - j + 1;
    std::vector<double> c(m), d(m);
    for (uint32_t k = 0; k < m; ++k) {
      const uint32_t q = j + k;
      const double lower = k > 0 ? off[q - 1] : 0.0;
      const double upper = k + 1 < m ? off[q] : 0.0;
      const double denom = dg[q] - (k > 0 ? lower * c[k - 1] : 0.0);
      c[k] = upper / denom;
      d[k] = (bb[q] - (k > 0 ? lower * d[k - 1] : 0.0)) / denom;
    }
    Y_out[e] = d[m - 1];
    for (int k = (int)m - 2; k >= 0; --k) Y_out[j + k] = d[k] - c[k] * Y_out[j + k + 1];
    j = e + 1;
  }
}

void orc_rmi_leaf_project(uint64_t V, uint32_t L, uint32_t J, const double* Y0, double gamma, double* Y);

// The training iteration itself: `iters` rounds of a Jacobi-preconditioned
// gradient step Y_j <- Y_j - eta * g_j / h_j on the free knots 1..J, all
// knots updated from the same gradient (the loss and its partials as
// above), followed by the projection (gamma = 0 skips it), starting from
// and regularised toward the prior Y0.  Double precision.
void orc_rmi_leaf_train(int key_type, const uint64_t* x, uint64_t S, uint64_t V, float a, float b, uint32_t L,
                        const uint64_t* kb, uint32_t J, const double* Y0, double rho, double gamma, uint32_t iters,
                        double eta, double* Y_out) {
  std::vector<double> g(L + 1), h(L + 1);
  for (uint32_t j = 0; j <= L; ++j) Y_out[j] = Y0[j];
  for (uint32_t it = 0; it < iters; ++it) {
    orc_rmi_leaf_loss_grad(key_type, x, S, V, a, b, L, kb, J, Y_out, Y0, rho, g.data(), h.data());
    for (uint32_t j = 1; j <= J; ++j)
      if (h[j] > 0.0) Y_out[j] -= eta * g[j] / h[j];
    if (gamma > 0.0) orc_rmi_leaf_project(V, L, J, Y0, gamma, Y_out);
  }
}

// Prior knot values: the interpolant of the rank targets at each knot kb_j
// (1 <= j <= J).  With lo = #{sample < kb_j}, kb_j lies in (x_{lo-1}, x_lo]
// and Y0_j interpolates linearly in the key between the targets of those
// two samples; the end points (0, 0) and (key max + 1, V) close the ends.
// Y0_0 = 0, Y0_j = V for j > J.  Double, unfused, in the order written.
void orc_rmi_leaf_init(int key_type, const uint64_t* x, uint64_t S, uint64_t V, uint32_t L, const uint64_t* kb,
                       uint32_t J, double* Y) {
  const uint64_t kmax = key_max(key_type);
  for (uint32_t j = 0; j <= L; ++j) {
    if (j == 0) { Y[j] = 0.0; continue; }
    if (j > J) { Y[j] = (double)V; continue; }
    const uint64_t k = kb[j];
    const uint64_t lo = (uint64_t)(std::lower_bound(x, x + S, k) - x);
    const uint64_t xl = lo == 0 ? 0 : x[lo - 1];
    const double yl = lo == 0 ? 0.0 : (double)(2 * lo - 1) / (double)(2 * S);
    const double yr = lo == S ? 1.0 : (double)(2 * lo + 1) / (double)(2 * S);
    const double num = (double)(k - xl);
    const double den = lo == S ? (double)(kmax - xl) + 1.0 : (double)(x[lo] - xl);
    const double f = den > 0.0 ? num / den : 0.0;
    const double dy = yr - yl;
    const double t = f * dy;
    const double y = yl + t;
    Y[j] = (double)V * y;
  }
}

// Projection onto { Y_j - Y_{j-1} >= gamma (Y0_j - Y0_{j-1}), Y_0 = 0,
// Y_{J+1} = V }: with Z = Y - gamma Y0 the constraint is Z non-decreasing
// between Z_0 = 0 and (1 - gamma) V, so Z becomes its running maximum capped
// at (1 - gamma) V.
void orc_rmi_leaf_project(uint64_t V, uint32_t L, uint32_t J, const double* Y0, double gamma, double* Y) {
  const double cap = (1.0 - gamma) * (double)V;
  double run = 0.0;
  for (uint32_t j = 1; j <= J && j <= L; ++j) {
    const double gy = gamma * Y0[j];
    const double z = Y[j] - gy;
    run = std::max(run, z);
    const double zc = std::min(run, cap);
    Y[j] = zc + gy;
  }
}

// Root fit: targets t_i = L (2i+1) / (2S) against the feature f(x_i);
// least-squares line (a, b) in double, and the loss gradient at (a, b).
void orc_rmi_root_lsq(int key_type, const uint64_t* x, uint64_t S, uint32_t L, double* ab) {
  double sf = 0, st = 0, sff = 0, sft = 0;
  for (uint64_t i = 0; i < S; ++i) {
    const double f = (double)feature(key_type, x[i]);
    const double t = (double)L * (2.0 * (double)i + 1.0) / (2.0 * (double)S);
    sf += f; st += t; sff += f * f; sft += f * t;
  }
  const double n = (double)S;
  const double var = sff - sf * sf / n;
  const double a = var > 0 ? (sft - sf * st / n) / var : 0.0;
  ab[0] = a;
  ab[1] = (st - a * sf) / n;
}

double orc_rmi_root_loss_grad(int key_type, const uint64_t* x, uint64_t S, uint32_t L, double a, double b,
                              double* g) {
  double loss = 0, ga = 0, gb = 0;
  for (uint64_t i = 0; i < S; ++i) {
    const double f = (double)feature(key_type, x[i]);
    const double t = (double)L * (2.0 * (double)i + 1.0) / (2.0 * (double)S);
    const double r = a * f + b - t;
    loss += r * r;
    ga += 2.0 * r * f;
    gb += 2.0 * r;
  }
  g[0] = ga / (double)S;
  g[1] = gb / (double)S;
  return loss / (double)S;
}

}  // extern "C"
