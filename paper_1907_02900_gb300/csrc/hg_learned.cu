// Learned bucket map (not in the paper, which hashes with Murmur; Section 2).
//
// A two-layer, order-preserving, piecewise-linear model of the key CDF used
// in place of "hash(a) mod V":
//   root   leaf j = clamp(floor(a * f(x) + b), 0, L-1), f a monotone
//          log-like feature (fp32 bits of the key, as fp32)
//   knots  kb_j = smallest key the root sends to leaf j or beyond; leaf j
//          owns [kb_j, kb_{j+1}); the last reached leaf J ends at max + 1
//   spline bucket position Y_j + (Y_{j+1} - Y_j) * lambda, lambda the
//          position of the key inside its leaf; Y_0 = 0, Y_j = V for j > J
// Training, all on the GPU, on a key sample the build draws itself:
//   sample   SplitMix64 indices (counter-based), gather, radix sort
//   root     least squares of the leaf index target L*(2i+1)/(2S) on the
//            centred, normalised feature, by forward/backward passes and
//            Newton steps on the (diagonal) Hessian
//   knots    exact bisection on the fp32 root
//   leaves   loss (1/S) sum_i (P(x_i) - V*(2i+1)/(2S))^2 over the knot
//            values; forward/backward per leaf (one warp per leaf, fixed
//            summation order, so training is deterministic) and
//            Jacobi-preconditioned gradient steps on Y = B + o (B integer,
//            o fp32 offset)
//   finalize monotone projection and the model blob.
#include <cmath>
#include <mutex>

#include "hg_build.cuh"
#include "hg_trace.h"

namespace hg {

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea and Flood 2014) as a counter-based generator.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t sm64_finalize(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t kGammaSM = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kSampleStream = 0x4C4541524Eull;
constexpr uint64_t kStreamMul = 0xD1B54A32D192ED03ull;

__device__ __forceinline__ float root_feature(int kt, uint64_t x) {
  return kt == 0 ? rmi_feature((uint32_t)x) : rmi_feature(x);
}
__device__ __forceinline__ uint32_t root_leaf_dev(float a, float b, uint32_t L, int kt, uint64_t x) {
  const float r = __fadd_rn(__fmul_rn(a, root_feature(kt, x)), b);
  if (!(r >= 0.0f)) return 0;
  if (r >= __uint2float_rn(L)) return L - 1;
  return (uint32_t)r;
}
__host__ __device__ __forceinline__ uint64_t key_max_of(int kt) { return kt == 0 ? 0xFFFFFFFFull : ~0ull; }

template <typename K>
__global__ void k_sample(const K* __restrict__ keys, uint64_t n, uint64_t S, uint64_t state,
                         uint64_t* __restrict__ out) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x = sm64_finalize(state + (k + 1) * kGammaSM);
    const uint64_t idx = ((x >> 32) * n) >> 32;
    out[k] = (uint64_t)keys[idx];
  }
}

// Deterministic block reduction of NV doubles per thread into out[blockIdx.x*NV + k].
template <int NV>
__device__ __forceinline__ void block_reduce_out(double (&v)[NV], double* out, double* sh) {
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[w * NV + k] = v[k];
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0;
    for (int i = 0; i < nw; ++i) s += sh[i * NV + threadIdx.x];
    out[(uint64_t)blockIdx.x * NV + threadIdx.x] = s;
  }
}

// Root state in the workspace.
struct RootState {
  double fmin, delta, ubar;  // feature normalisation u = (f - fmin) / delta, centred by ubar
  double w, c;               // model: leaf target ~ w * (u - ubar) + c
  double a, b;               // folded fp32-ready root: a * f + b
  double loss;
};

constexpr int kLrnBlocks = 256, kLrnThreads = 256;
// Ridge weight rho of the knot values (one sample's squared error per unit
// of squared deviation from the initial knot value).
constexpr float kLeafRidge = 1.0f;
// Width floor gamma of the projection: every leaf keeps at least this share
// of the bucket width the prior gives it.
constexpr double kLeafMinWidth = 0.5;

// mode 0: sum of u; mode 1: sums of r*(u-ubar), r, (u-ubar)^2, r^2
__global__ void __launch_bounds__(kLrnThreads) k_root_partials(const uint64_t* __restrict__ x, uint64_t S, uint32_t L,
                                                               int kt, const RootState* __restrict__ rs, int mode,
                                                               double* __restrict__ partials) {
  __shared__ double sh[32 * 4];
  double v[4] = {0, 0, 0, 0};
  const double fmin = rs->fmin, delta = rs->delta, ubar = rs->ubar, w = rs->w, c = rs->c;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (uint64_t)gridDim.x * blockDim.x) {
    const double u = ((double)root_feature(kt, x[i]) - fmin) / delta;
    if (mode == 0) {
      v[0] += u;
    } else {
      const double t = (double)L * (2.0 * (double)i + 1.0) / (2.0 * (double)S);
      const double uc = u - ubar;
      const double r = w * uc + c - t;
      v[0] += r * uc;
      v[1] += r;
      v[2] += uc * uc;
      v[3] += r * r;
    }
  }
  block_reduce_out<4>(v, partials, sh);
}

// Sums the block partials in order; mode 0 sets ubar, mode 1 takes one
// Newton step w -= g_w / h_w, c -= g_c / h_c (the Hessian is diagonal in
// centred coordinates) and records the loss before the step.
__global__ void k_root_step(const double* __restrict__ partials, int nblocks, RootState* rs, uint64_t S, int mode) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[4] = {0, 0, 0, 0};
  for (int i = 0; i < nblocks; ++i)
    for (int k = 0; k < 4; ++k) s[k] += partials[i * 4 + k];
  if (mode == 0) {
    rs->ubar = s[0] / (double)S;
    return;
  }
  const double gw = 2.0 * s[0] / (double)S, gc = 2.0 * s[1] / (double)S;
  const double hw = 2.0 * s[2] / (double)S, hc = 2.0;
  rs->loss = s[3] / (double)S;
  if (hw > 0) rs->w -= gw / hw;
  rs->c -= gc / hc;
}

__global__ void k_root_init(const uint64_t* __restrict__ x, uint64_t S, int kt, RootState* rs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double f0 = (double)root_feature(kt, x[0]), f1 = (double)root_feature(kt, x[S - 1]);
  rs->fmin = f0;
  rs->delta = f1 > f0 ? f1 - f0 : 1.0;
  rs->ubar = 0;
  rs->w = 0;
  rs->c = 0;
  rs->loss = 0;
}

// Folds (w, c) into the raw-feature root and rounds it to fp32.
__global__ void k_root_fold(RootState* rs, float* ab) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double a = rs->w / rs->delta;
  const double b = rs->c - rs->w * rs->ubar - a * rs->fmin;
  rs->a = a;
  rs->b = b;
  ab[0] = (float)a;
  ab[1] = (float)b;
}

// Raw-coordinate root loss and gradient (double), for checking against the oracle.
__global__ void __launch_bounds__(kLrnThreads) k_root_grad_ab(const uint64_t* __restrict__ x, uint64_t S, uint32_t L,
                                                              int kt, double a, double b, double* __restrict__ partials) {
  __shared__ double sh[32 * 4];
  double v[4] = {0, 0, 0, 0};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (uint64_t)gridDim.x * blockDim.x) {
    const double f = (double)root_feature(kt, x[i]);
    const double t = (double)L * (2.0 * (double)i + 1.0) / (2.0 * (double)S);
    const double r = a * f + b - t;
    v[0] += r * r;
    v[1] += 2.0 * r * f;
    v[2] += 2.0 * r;
  }
  block_reduce_out<4>(v, partials, sh);
}

__global__ void k_sum_partials(const double* __restrict__ partials, int nblocks, int nv, uint64_t S,
                               double* __restrict__ out) {
  if (threadIdx.x >= (unsigned)nv || blockIdx.x != 0) return;
  double s = 0;
  for (int i = 0; i < nblocks; ++i) s += partials[i * nv + threadIdx.x];
  out[threadIdx.x] = s / (double)S;
}

// Knots by bisection on the exact fp32 root; J = root(max key).
__global__ void k_knots(const float* __restrict__ ab, uint32_t L, int kt, uint64_t* __restrict__ kb,
                        uint32_t* __restrict__ Jout) {
  const float a = ab[0], b = ab[1];
  const uint64_t hi_key = key_max_of(kt);
  const uint32_t J = root_leaf_dev(a, b, L, kt, hi_key);
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= L; j += gridDim.x * blockDim.x) {
    if (j == 0) {
      kb[0] = 0;
      *Jout = J;
      continue;
    }
    if (j > J) {
      kb[j] = hi_key;
      continue;
    }
    uint64_t lo = 0, hi = hi_key;
    while (lo < hi) {
      const uint64_t mid = lo + ((hi - lo) >> 1);
      if (root_leaf_dev(a, b, L, kt, mid) >= j) hi = mid; else lo = mid + 1;
    }
    kb[j] = lo;
  }
}

// Prior knot values Y0_j: the piecewise-linear interpolant, in the key, of
// the rank targets (0, 0), (x_i, V (2i+1) / (2S)), (key max + 1, V) at the
// knot kb_j.  With lo = #{sample < kb_j} the knot lies in (x_{lo-1}, x_lo].
// Double arithmetic, round-to-nearest intrinsics in a fixed order (no
// contraction), so Y0 is reproducible bit for bit by any IEEE double
// implementation of the same steps.  Y0 is kept in double (Y0d) and split
// into an integer B_j = floor(Y0_j) and an fp32 offset o_j.
__global__ void k_leaf_init(const uint64_t* __restrict__ x, uint64_t S, uint64_t V, uint32_t L, int kt,
                            const uint64_t* __restrict__ kb, const uint32_t* __restrict__ Jp,
                            uint64_t* __restrict__ B, float* __restrict__ o, double* __restrict__ Y0d) {
  const uint32_t J = *Jp;
  const uint64_t kmax = key_max_of(kt);
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= L; j += gridDim.x * blockDim.x) {
    double y;
    if (j == 0) {
      y = 0.0;
    } else if (j > J) {
      y = __ull2double_rn(V);
    } else {
      const uint64_t k = kb[j];
      uint64_t lo = 0, hi = S;
      while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (x[mid] < k) lo = mid + 1; else hi = mid;
      }
      const uint64_t xl = lo == 0 ? 0 : x[lo - 1];
      const double s2 = __ull2double_rn(2 * S);
      const double yl = lo == 0 ? 0.0 : __ddiv_rn(__ull2double_rn(2 * lo - 1), s2);
      const double yr = lo == S ? 1.0 : __ddiv_rn(__ull2double_rn(2 * lo + 1), s2);
      const double num = __ull2double_rn(k - xl);
      const double den = lo == S ? __dadd_rn(__ull2double_rn(kmax - xl), 1.0) : __ull2double_rn(x[lo] - xl);
      const double f = den > 0.0 ? __ddiv_rn(num, den) : 0.0;
      const double t = __dmul_rn(f, __dsub_rn(yr, yl));
      y = __dmul_rn(__ull2double_rn(V), __dadd_rn(yl, t));
    }
    const uint64_t bj = (uint64_t)floor(y);
    Y0d[j] = y;
    B[j] = bj;
    o[j] = __double2float_rn(__dsub_rn(y, __ull2double_rn(bj)));
  }
}

// Projection onto { Y_j - Y_{j-1} >= gamma (Y0_j - Y0_{j-1}) }: with
// Z = Y - gamma Y0 (Z_0 = 0), Z becomes its running maximum capped at
// (1 - gamma) V.  One block; inclusive max-scan in double over tiles of
// blockDim knots with a carry.  Only the offsets o_j of knots 1..J change.
__global__ void k_leaf_project(uint32_t L, const uint32_t* __restrict__ Jp, uint64_t V, double gamma,
                               const double* __restrict__ Y0d, const uint64_t* __restrict__ B,
                               float* __restrict__ o) {
  __shared__ double wmax[32];
  __shared__ double carry_s;
  const uint32_t J = min(*Jp, L);
  const double cap = __dmul_rn(__dsub_rn(1.0, gamma), __ull2double_rn(V));
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry_s = 0.0;
  __syncthreads();
  for (uint32_t base = 1; base <= J; base += blockDim.x) {
    const uint32_t j = base + threadIdx.x;
    double gy = 0.0, z = 0.0;
    if (j <= J) {
      gy = __dmul_rn(gamma, Y0d[j]);
      const double y = __dadd_rn(__ull2double_rn(B[j]), (double)o[j]);
      z = __dsub_rn(y, gy);
    }
    double v = z;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, v, d);
      if ((int)lane >= d) v = fmax(v, u);
    }
    if (lane == 31) wmax[warp] = v;
    __syncthreads();
    if (warp == 0) {
      double w = lane < nw ? wmax[lane] : 0.0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, w, d);
        if ((int)lane >= d) w = fmax(w, u);
      }
      if (lane < nw) wmax[lane] = w;
    }
    __syncthreads();
    const double carry = carry_s;
    double run = fmax(carry, v);
    if (warp > 0) run = fmax(run, wmax[warp - 1]);
    if (j <= J) {
      const double zc = fmin(run, cap);
      o[j] = __double2float_rn(__dsub_rn(__dadd_rn(zc, gy), __ull2double_rn(B[j])));
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_s = fmax(carry, wmax[nw - 1]);
    __syncthreads();
  }
}

// Leaf and in-leaf position lambda of each sample; target relative to B_leaf.
__global__ void k_leaf_coords(const uint64_t* __restrict__ x, uint64_t S, uint64_t V, const float* __restrict__ ab,
                              uint32_t L, int kt, const uint64_t* __restrict__ kb, const uint32_t* __restrict__ Jp,
                              const uint64_t* __restrict__ B, uint32_t* __restrict__ leaf, float* __restrict__ lam,
                              float* __restrict__ yrel) {
  const float a = ab[0], b = ab[1];
  const uint32_t J = *Jp;
  const uint64_t kmax = key_max_of(kt);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t xi = x[i];
    const uint32_t j = root_leaf_dev(a, b, L, kt, xi);
    const double w = j < J ? (double)(kb[j + 1] - kb[j]) : (double)(kmax - kb[j]) + 1.0;
    leaf[i] = j;
    lam[i] = w > 0.0 ? (float)((double)(xi - kb[j]) / w) : 0.0f;
    yrel[i] = (float)((double)V * (2.0 * (double)i + 1.0) / (2.0 * (double)S) - (double)B[j]);
  }
}

// First sample of each leaf (samples are sorted, the root is monotone).
__global__ void k_leaf_ranges(const uint32_t* __restrict__ leaf, uint64_t S, uint32_t L, uint32_t* __restrict__ ls) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= L; j += gridDim.x * blockDim.x) {
    uint64_t lo = 0, hi = S;
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (leaf[mid] < j) lo = mid + 1; else hi = mid;
    }
    ls[j] = (uint32_t)lo;
  }
}

// Forward + backward of the spline loss, one warp per leaf:
//   pred = (1 - lambda) * o_j + lambda * (B_{j+1} - B_j + o_{j+1})   (relative to B_j)
//   r = pred - yrel;  sums over the leaf (fixed order):
//   A = sum r (1-lambda), Bs = sum r lambda, C = sum (1-lambda)^2, D = sum lambda^2, E = sum r^2
__global__ void __launch_bounds__(kLrnThreads) k_leaf_fwdbwd(const float* __restrict__ lam,
                                                             const float* __restrict__ yrel,
                                                             const uint32_t* __restrict__ ls,
                                                             const uint64_t* __restrict__ B,
                                                             const float* __restrict__ o, uint32_t L,
                                                             float* __restrict__ sums) {
  const uint32_t lane = lane_id();
  const uint32_t wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t j = wg; j < L; j += nwarps) {
    const float oj = o[j], oj1 = o[j + 1];
    const float dB = (float)(double)(B[j + 1] - B[j]);
    const float right = __fadd_rn(dB, oj1);
    float A = 0.f, Bs = 0.f, C = 0.f, D = 0.f, E = 0.f;
    for (uint32_t i = ls[j] + lane; i < ls[j + 1]; i += 32) {
      const float l = lam[i], m = __fsub_rn(1.0f, l);
      const float pred = __fadd_rn(__fmul_rn(m, oj), __fmul_rn(l, right));
      const float r = __fsub_rn(pred, yrel[i]);
      A = __fadd_rn(A, __fmul_rn(r, m));
      Bs = __fadd_rn(Bs, __fmul_rn(r, l));
      C = __fadd_rn(C, __fmul_rn(m, m));
      D = __fadd_rn(D, __fmul_rn(l, l));
      E = __fadd_rn(E, __fmul_rn(r, r));
    }
    A = warp_sum(A);
    Bs = warp_sum(Bs);
    C = warp_sum(C);
    D = warp_sum(D);
    E = warp_sum(E);
    if (lane == 0) {
      sums[5 * j + 0] = A;
      sums[5 * j + 1] = Bs;
      sums[5 * j + 2] = C;
      sums[5 * j + 3] = D;
      sums[5 * j + 4] = E;
    }
  }
}

// Deviation d_j = Y_j - Y0_j of a free knot from its initial value (the
// ridge term); B/o hold Y, B0/o0 hold Y0.
__device__ __forceinline__ float knot_dev(const uint64_t* B, const float* o, const uint64_t* B0, const float* o0,
                                          uint32_t j) {
  const float dB = (float)((double)(int64_t)(B[j] - B0[j]));
  return __fadd_rn(dB, __fsub_rn(o[j], o0[j]));
}

// Knot gradient g_j = (2/S)(Bs_{j-1} + A_j + rho d_j), Hessian diagonal
// h_j = (2/S)(D_{j-1} + C_j + rho), the ridge on the free knots 1..J only;
// Jacobi step o_j -= eta * g_j / h_j on the free knots.  grad/diag
// (optional) receive g and h for every knot.
__global__ void k_leaf_update(const float* __restrict__ sums, uint32_t L, const uint32_t* __restrict__ Jp, uint64_t S,
                              float rho, const uint64_t* __restrict__ B, const uint64_t* __restrict__ B0,
                              const float* __restrict__ o0, float eta, float* __restrict__ o, float* __restrict__ grad,
                              float* __restrict__ diag) {
  const uint32_t J = *Jp;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= L; j += gridDim.x * blockDim.x) {
    const float left_B = j > 0 ? sums[5 * (j - 1) + 1] : 0.f, left_D = j > 0 ? sums[5 * (j - 1) + 3] : 0.f;
    const float right_A = j < L ? sums[5 * j + 0] : 0.f, right_C = j < L ? sums[5 * j + 2] : 0.f;
    const bool free_knot = j >= 1 && j <= J;
    const float rg = free_knot ? __fmul_rn(rho, knot_dev(B, o, B0, o0, j)) : 0.f;
    const float rh = free_knot ? rho : 0.f;
    const float scale = (float)(2.0 / (double)S);
    const float g = __fmul_rn(scale, __fadd_rn(__fadd_rn(left_B, right_A), rg));
    const float h = __fmul_rn(scale, __fadd_rn(__fadd_rn(left_D, right_C), rh));
    if (grad) grad[j] = g;
    if (diag) diag[j] = h;
    if (eta > 0.f && free_knot && h > 0.f) o[j] = __fsub_rn(o[j], __fmul_rn(eta, __fdiv_rn(g, h)));
  }
}

// loss = (sum_leaves E + rho sum_{j=1..J} d_j^2) / S
__global__ void k_leaf_loss(const float* __restrict__ sums, uint32_t L, const uint32_t* __restrict__ Jp, uint64_t S,
                            float rho, const uint64_t* __restrict__ B, const float* __restrict__ o,
                            const uint64_t* __restrict__ B0, const float* __restrict__ o0, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint32_t J = *Jp;
  double e = 0;
  for (uint32_t j = 0; j < L; ++j) e += (double)sums[5 * j + 4];
  double r = 0;
  for (uint32_t j = 1; j <= J && j <= L; ++j) {
    const double d = (double)knot_dev(B, o, B0, o0, j);
    r += d * d;
  }
  *out = (e + (double)rho * r) / (double)S;
}

// Model blob: monotone projection of Y = B + o, then per leaf
// base = floor(Y_j), icpt = Y_j - base, slope = (Y_{j+1} - Y_j) / (key width),
// width = base_{j+1} - base_j; leaves above J are empty.
__global__ void k_finalize(const float* __restrict__ ab, uint32_t L, uint64_t V, int kt,
                           const uint64_t* __restrict__ kb, const uint32_t* __restrict__ Jp,
                           const uint64_t* __restrict__ B, const float* __restrict__ o, uint8_t* __restrict__ blob,
                           double* __restrict__ Y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint32_t J = *Jp;
  const uint64_t kmax = key_max_of(kt);
  double run = 0.0;
  for (uint32_t j = 0; j <= L; ++j) {
    double y = (double)B[j] + (double)o[j];
    y = y < 0.0 ? 0.0 : (y > (double)V ? (double)V : y);
    run = y > run ? y : run;
    Y[j] = run < (double)V ? run : (double)V;
  }
  uint32_t* h32 = (uint32_t*)blob;
  h32[0] = kModelMagic;
  h32[1] = L;
  *(uint64_t*)(blob + 8) = V;
  *(float*)(blob + 16) = ab[0];
  *(float*)(blob + 20) = ab[1];
  h32[6] = (uint32_t)kt;
  h32[7] = 0;
  LearnedLeaf* lf = (LearnedLeaf*)(blob + kModelHeaderBytes);
  for (uint32_t j = 0; j < L; ++j) {
    LearnedLeaf e;
    if (j <= J) {
      const double wkeys = j < J ? (double)(kb[j + 1] - kb[j]) : (double)(kmax - kb[j]) + 1.0;
      const uint64_t base = (uint64_t)floor(Y[j]);
      const uint64_t nb = j < J ? (uint64_t)floor(Y[j + 1]) : V;
      double slope;
      if (wkeys > 0 && j < J) slope = (Y[j + 1] - Y[j]) / wkeys;
      else slope = wkeys > 0 ? ((double)V - Y[j]) / wkeys : 0.0;
      e.xmin = kb[j];
      e.slope = (float)slope;
      e.icpt = (float)(Y[j] - (double)base);
      e.base = (uint32_t)base;
      e.width = (uint32_t)(nb - base);
    } else {
      e.xmin = kmax;
      e.slope = 0.f;
      e.icpt = 0.f;
      e.base = (uint32_t)V;
      e.width = 0;
    }
    lf[j] = e;
  }
}

__global__ void k_set_root(float* ab, float a, float b) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ab[0] = a;
    ab[1] = b;
  }
}

// Y (double) -> integer part B and fp32 offset o.
__global__ void k_split_Y(const double* __restrict__ Y, uint32_t L, uint64_t* __restrict__ B, float* __restrict__ o) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= L; j += gridDim.x * blockDim.x) {
    const double y = Y[j] > 0.0 ? Y[j] : 0.0;
    const double f = floor(y);
    B[j] = (uint64_t)f;
    o[j] = (float)(y - f);
  }
}

// ---------------------------------------------------------------------------
// Bucket-length statistics of a map over a key set.
// ---------------------------------------------------------------------------
template <typename K, typename Map>
__global__ void k_bucket_count(const K* __restrict__ keys, uint64_t n, uint32_t* __restrict__ counts, Map map) {
  map.init();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[map(keys[i])], 1u);
}

__global__ void __launch_bounds__(kLrnThreads) k_bucket_moments(const uint32_t* __restrict__ counts, uint64_t V,
                                                                double* __restrict__ partials) {
  __shared__ double sh[32 * 4];
  double v[4] = {0, 0, 0, 0};  // max, sum, sum of squares, non-empty
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (uint64_t)gridDim.x * blockDim.x) {
    const double c = counts[i];
    v[0] = c > v[0] ? c : v[0];
    v[1] += c;
    v[2] += c * c;
    v[3] += c > 0 ? 1.0 : 0.0;
  }
  // max needs its own reduction
  double m = v[0];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
  v[0] = 0;
  block_reduce_out<4>(v, partials, sh);
  __syncthreads();
  if (lane_id() == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = fmax(mm, sh[i]);
    partials[(uint64_t)blockIdx.x * 4] = mm;
  }
}

__global__ void k_bucket_final(const double* __restrict__ partials, int nblocks, uint64_t V, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double mx = 0, s = 0, s2 = 0, ne = 0;
  for (int i = 0; i < nblocks; ++i) {
    mx = fmax(mx, partials[i * 4]);
    s += partials[i * 4 + 1];
    s2 += partials[i * 4 + 2];
    ne += partials[i * 4 + 3];
  }
  const double mean = s / (double)V;
  out[0] = mx;
  out[1] = mean;
  out[2] = s2 / (double)V - mean * mean;
  out[3] = ne;
}

// ---------------------------------------------------------------------------
// Workspace of the learned-map training.
// ---------------------------------------------------------------------------
struct LrnLayout {
  size_t sample, radix, leaf, lam, yrel, kb, B, o, B0, o0, Y0d, ls, sums, rs, partials, ab, J, Yd, total;
};

static LrnLayout lrn_layout(uint64_t S, uint32_t L) {
  LrnLayout l{};
  size_t o = sizeof(WsHeader);
  l.sample = o;   o = align_up(o + (S + 16) * 8);
  l.radix = o;    o = align_up(o + radix_sort_workspace_bytes(S));
  l.leaf = o;     o = align_up(o + S * 4);
  l.lam = o;      o = align_up(o + S * 4);
  l.yrel = o;     o = align_up(o + S * 4);
  l.kb = o;       o = align_up(o + ((size_t)L + 1) * 8);
  l.B = o;        o = align_up(o + ((size_t)L + 1) * 8);
  l.o = o;        o = align_up(o + ((size_t)L + 1) * 4);
  l.B0 = o;       o = align_up(o + ((size_t)L + 1) * 8);
  l.o0 = o;       o = align_up(o + ((size_t)L + 1) * 4);
  l.Y0d = o;      o = align_up(o + ((size_t)L + 1) * 8);
  l.ls = o;       o = align_up(o + ((size_t)L + 2) * 4);
  l.sums = o;     o = align_up(o + (size_t)L * 5 * 4);
  l.rs = o;       o = align_up(o + sizeof(RootState));
  l.partials = o; o = align_up(o + (size_t)kLrnBlocks * 4 * 8);
  l.ab = o;       o = align_up(o + 16);
  l.J = o;        o = align_up(o + 16);
  l.Yd = o;       o = align_up(o + ((size_t)L + 1) * 8);
  l.total = o;
  return l;
}

static hg_status sample_and_sort(int kt, const void* keys, uint64_t n, uint64_t S, uint64_t seed, uint64_t* out,
                                 uint8_t* radix_ws, cudaStream_t st) {
  const uint64_t state = sm64_finalize(seed ^ (kSampleStream * kStreamMul));
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((S + 255) / 256, 4096));
  {
    HG_TRACE("k_learn_sample", st);
    if (kt == HG_KEY_U64) k_sample<uint64_t><<<grid, 256, 0, st>>>((const uint64_t*)keys, n, S, state, out);
    else k_sample<uint32_t><<<grid, 256, 0, st>>>((const uint32_t*)keys, n, S, state, out);
  }
  if (cudaMemsetAsync(radix_ws, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
  return radix_sort_u64(out, S, radix_ws, st);
}

}  // namespace hg

using namespace hg;

extern "C" {

size_t hg_learned_model_bytes(uint32_t num_leaves) { return kModelHeaderBytes + (size_t)num_leaves * sizeof(LearnedLeaf); }

size_t hg_learned_workspace_size(int32_t key_type, uint64_t n, uint64_t sample_size, uint32_t num_leaves) {
  (void)key_type;
  (void)n;
  if (sample_size == 0 || num_leaves == 0) return 0;
  return lrn_layout(sample_size, num_leaves).total;
}

hg_status hg_learned_sorted_sample(int32_t key_type, const void* d_keys, uint64_t n, uint64_t sample_size,
                                   uint64_t seed, uint64_t* d_out, void* d_ws, size_t ws_bytes, void* stream) {
  if ((key_type != HG_KEY_U32 && key_type != HG_KEY_U64) || !d_keys || !d_out || !d_ws) return HG_ERR_INVALID_ARG;
  if (n == 0 || n > (1ull << 32) || sample_size == 0 || sample_size >= (1ull << 32)) return HG_ERR_INVALID_ARG;
  if ((uintptr_t)d_out % 16 || (uintptr_t)d_ws % 256) return HG_ERR_INVALID_ARG;
  if (ws_bytes < radix_sort_workspace_bytes(sample_size)) return HG_ERR_WORKSPACE_TOO_SMALL;
  return sample_and_sort(key_type, d_keys, n, sample_size, seed, d_out, (uint8_t*)d_ws, (cudaStream_t)stream);
}

hg_status hg_learned_root_grad(int32_t key_type, const uint64_t* d_sorted, uint64_t S, uint32_t num_leaves,
                               double a, double b, double* d_out3, void* d_ws, size_t ws_bytes, void* stream) {
  if ((key_type != HG_KEY_U32 && key_type != HG_KEY_U64) || !d_sorted || !d_out3 || !d_ws || S == 0)
    return HG_ERR_INVALID_ARG;
  if (ws_bytes < (size_t)kLrnBlocks * 4 * 8) return HG_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  double* partials = (double*)d_ws;
  k_root_grad_ab<<<kLrnBlocks, kLrnThreads, 0, st>>>(d_sorted, S, num_leaves, key_type, a, b, partials);
  k_sum_partials<<<1, 32, 0, st>>>(partials, kLrnBlocks, 4, S, d_out3);
  return last_launch_status();
}

hg_status hg_learned_leaf_grad(int32_t key_type, const uint64_t* d_sorted, uint64_t S, uint64_t num_buckets,
                               float a, float b, uint32_t num_leaves, const double* d_Y, float* d_grad,
                               float* d_diag, double* d_loss, void* d_ws, size_t ws_bytes, void* stream);

hg_status hg_learned_train(int32_t key_type, const void* d_keys, uint64_t n, uint64_t num_buckets,
                           uint32_t num_leaves, uint64_t sample_size, uint64_t seed, uint32_t iters, void* d_model,
                           double* d_diag, void* d_ws, size_t ws_bytes, void* stream) {
  if ((key_type != HG_KEY_U32 && key_type != HG_KEY_U64) || !d_keys || !d_model || !d_ws) return HG_ERR_INVALID_ARG;
  if (n == 0 || n > (1ull << 32) || num_buckets == 0 || num_buckets > (1ull << 32)) return HG_ERR_INVALID_ARG;
  if (num_leaves == 0 || num_leaves > (1u << 20) || sample_size == 0 || sample_size >= (1ull << 32))
    return HG_ERR_INVALID_ARG;
  if ((uintptr_t)d_ws % 256 || (uintptr_t)d_model % 8) return HG_ERR_INVALID_ARG;
  const LrnLayout l = lrn_layout(sample_size, num_leaves);
  if (ws_bytes < l.total) return HG_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* ws = (uint8_t*)d_ws;
  const uint64_t S = sample_size, V = num_buckets;
  const uint32_t L = num_leaves;
  const int kt = key_type;
  uint64_t* x = (uint64_t*)(ws + l.sample);
  uint32_t* leaf = (uint32_t*)(ws + l.leaf);
  float* lam = (float*)(ws + l.lam);
  float* yrel = (float*)(ws + l.yrel);
  uint64_t* kb = (uint64_t*)(ws + l.kb);
  uint64_t* B = (uint64_t*)(ws + l.B);
  float* o = (float*)(ws + l.o);
  uint64_t* B0 = (uint64_t*)(ws + l.B0);
  float* o0 = (float*)(ws + l.o0);
  double* Y0d = (double*)(ws + l.Y0d);
  uint32_t* ls = (uint32_t*)(ws + l.ls);
  float* sums = (float*)(ws + l.sums);
  RootState* rs = (RootState*)(ws + l.rs);
  double* partials = (double*)(ws + l.partials);
  float* ab = (float*)(ws + l.ab);
  uint32_t* Jd = (uint32_t*)(ws + l.J);
  double* Yd = (double*)(ws + l.Yd);
  if (cudaMemsetAsync(ws, 0, sizeof(WsHeader), st) != cudaSuccess) return HG_ERR_CUDA;
  hg_status rc = sample_and_sort(kt, d_keys, n, S, seed, x, ws + l.radix, st);
  if (rc != HG_OK) return rc;
  // root: normalise, centre, Newton steps
  {
    HG_TRACE("k_learn_root", st);
    k_root_init<<<1, 32, 0, st>>>(x, S, kt, rs);
    k_root_partials<<<kLrnBlocks, kLrnThreads, 0, st>>>(x, S, L, kt, rs, 0, partials);
    k_root_step<<<1, 32, 0, st>>>(partials, kLrnBlocks, rs, S, 0);
    for (int k = 0; k < 3; ++k) {
      k_root_partials<<<kLrnBlocks, kLrnThreads, 0, st>>>(x, S, L, kt, rs, 1, partials);
      k_root_step<<<1, 32, 0, st>>>(partials, kLrnBlocks, rs, S, 1);
    }
    k_root_fold<<<1, 32, 0, st>>>(rs, ab);
  }
  const unsigned gL = (L + 256) / 256;
  {
    HG_TRACE("k_learn_knots", st);
    k_knots<<<gL, 256, 0, st>>>(ab, L, kt, kb, Jd);
    k_leaf_init<<<gL, 256, 0, st>>>(x, S, V, L, kt, kb, Jd, B, o, Y0d);
    if (cudaMemcpyAsync(B0, B, ((size_t)L + 1) * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(o0, o, ((size_t)L + 1) * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return HG_ERR_CUDA;
    const unsigned gS = (unsigned)std::min<uint64_t>((S + 255) / 256, 4096);
    k_leaf_coords<<<gS, 256, 0, st>>>(x, S, V, ab, L, kt, kb, Jd, B, leaf, lam, yrel);
    k_leaf_ranges<<<gL + 1, 256, 0, st>>>(leaf, S, L, ls);
  }
  const unsigned gW = (L * 32 + kLrnThreads - 1) / kLrnThreads;
  {
    HG_TRACE("k_learn_leaves", st);
    for (uint32_t it = 0; it < iters; ++it) {
      k_leaf_fwdbwd<<<gW, kLrnThreads, 0, st>>>(lam, yrel, ls, B, o, L, sums);
      if (it == 0 && d_diag) k_leaf_loss<<<1, 32, 0, st>>>(sums, L, Jd, S, kLeafRidge, B, o, B0, o0, d_diag + 0);
      k_leaf_update<<<gL, 256, 0, st>>>(sums, L, Jd, S, kLeafRidge, B, B0, o0, 0.9f, o, nullptr, nullptr);
      k_leaf_project<<<1, 1024, 0, st>>>(L, Jd, V, kLeafMinWidth, Y0d, B, o);
    }
    k_leaf_fwdbwd<<<gW, kLrnThreads, 0, st>>>(lam, yrel, ls, B, o, L, sums);
    if (d_diag) k_leaf_loss<<<1, 32, 0, st>>>(sums, L, Jd, S, kLeafRidge, B, o, B0, o0, d_diag + 1);
  }
  {
    HG_TRACE("k_learn_finalize", st);
    k_finalize<<<1, 32, 0, st>>>(ab, L, V, kt, kb, Jd, B, o, (uint8_t*)d_model, Yd);
  }
  if (d_diag) {
    // d_diag: [loss at start, loss at end, root loss, J, Y_0..Y_L]
    cudaMemcpyAsync(d_diag + 2, &rs->loss, 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(d_diag + 4, Yd, ((size_t)L + 1) * 8, cudaMemcpyDeviceToDevice, st);
  }
  return last_launch_status();
}

hg_status hg_learned_leaf_grad(int32_t key_type, const uint64_t* d_sorted, uint64_t S, uint64_t num_buckets,
                               float a, float b, uint32_t num_leaves, const double* d_Y, float* d_grad,
                               float* d_diag, double* d_loss, void* d_ws, size_t ws_bytes, void* stream) {
  if ((key_type != HG_KEY_U32 && key_type != HG_KEY_U64) || !d_sorted || !d_Y || !d_grad || !d_diag || !d_loss ||
      !d_ws || S == 0 || num_leaves == 0 || num_buckets == 0)
    return HG_ERR_INVALID_ARG;
  const LrnLayout l = lrn_layout(S, num_leaves);
  if (ws_bytes < l.total) return HG_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t* ws = (uint8_t*)d_ws;
  const uint32_t L = num_leaves;
  uint32_t* leaf = (uint32_t*)(ws + l.leaf);
  float* lam = (float*)(ws + l.lam);
  float* yrel = (float*)(ws + l.yrel);
  uint64_t* kb = (uint64_t*)(ws + l.kb);
  uint64_t* B = (uint64_t*)(ws + l.B);
  float* o = (float*)(ws + l.o);
  uint64_t* B0 = (uint64_t*)(ws + l.B0);
  float* o0 = (float*)(ws + l.o0);
  double* Y0d = (double*)(ws + l.Y0d);
  uint32_t* ls = (uint32_t*)(ws + l.ls);
  float* sums = (float*)(ws + l.sums);
  float* ab = (float*)(ws + l.ab);
  uint32_t* Jd = (uint32_t*)(ws + l.J);
  const unsigned gL = (L + 256) / 256;
  k_set_root<<<1, 32, 0, st>>>(ab, a, b);
  k_knots<<<gL, 256, 0, st>>>(ab, L, key_type, kb, Jd);
  k_split_Y<<<gL, 256, 0, st>>>(d_Y, L, B, o);
  k_leaf_init<<<gL, 256, 0, st>>>(d_sorted, S, num_buckets, L, key_type, kb, Jd, B0, o0, Y0d);
  const unsigned gS = (unsigned)std::min<uint64_t>((S + 255) / 256, 4096);
  k_leaf_coords<<<gS, 256, 0, st>>>(d_sorted, S, num_buckets, ab, L, key_type, kb, Jd, B, leaf, lam, yrel);
  k_leaf_ranges<<<gL + 1, 256, 0, st>>>(leaf, S, L, ls);
  const unsigned gW = (L * 32 + kLrnThreads - 1) / kLrnThreads;
  k_leaf_fwdbwd<<<gW, kLrnThreads, 0, st>>>(lam, yrel, ls, B, o, L, sums);
  k_leaf_update<<<gL, 256, 0, st>>>(sums, L, Jd, S, kLeafRidge, B, B0, o0, 0.0f, o, d_grad, d_diag);
  k_leaf_loss<<<1, 32, 0, st>>>(sums, L, Jd, S, kLeafRidge, B, o, B0, o0, d_loss);
  return last_launch_status();
}

hg_status hg_bucket_stats(const hg_config* cfg, const void* d_keys, uint64_t n, uint32_t* d_counts,
                          double* d_out4, void* d_ws, size_t ws_bytes, void* stream) {
  hg_status rc = validate_config(cfg);
  if (rc != HG_OK) return rc;
  if ((n > 0 && !d_keys) || !d_counts || !d_out4 || !d_ws) return HG_ERR_INVALID_ARG;
  if (ws_bytes < (size_t)kLrnBlocks * 4 * 8) return HG_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t V = cfg->num_buckets;
  if (cudaMemsetAsync(d_counts, 0, V * 4, st) != cudaSuccess) return HG_ERR_CUDA;
  const int sms = dev_info().sms;
  rc = dispatch_key_map(cfg, [&](auto k, auto map) -> hg_status {
    using K = decltype(k);
    if (n > 0) k_bucket_count<K><<<(unsigned)std::max(1, sms * 8), 256, 0, st>>>((const K*)d_keys, n, d_counts, map);
    return last_launch_status();
  });
  if (rc != HG_OK) return rc;
  double* partials = (double*)d_ws;
  k_bucket_moments<<<kLrnBlocks, kLrnThreads, 0, st>>>(d_counts, V, partials);
  k_bucket_final<<<1, 32, 0, st>>>(partials, kLrnBlocks, V, d_out4);
  return last_launch_status();
}

size_t hg_learned_judge_workspace_size(void) { return (size_t)kLrnBlocks * 4 * 8 + 8 * 8; }

// Murmur judges the learned map: bucket-length statistics of both maps over
// the same keys (hg_bucket_stats twice, the learned map from cfg->d_model,
// Murmur with cfg->seed), then the fallback rule on the host.
hg_status hg_learned_judge(const hg_config* cfg, const void* d_keys, uint64_t n, double var_tolerance,
                           double max_factor, uint32_t* d_counts, void* d_ws, size_t ws_bytes, double* h_stats8,
                           int32_t* h_keep, void* stream) {
  hg_status rc = validate_config(cfg);
  if (rc != HG_OK) return rc;
  if (cfg->map != HG_MAP_LEARNED || !h_keep || !d_ws) return HG_ERR_INVALID_ARG;
  if (ws_bytes < hg_learned_judge_workspace_size()) return HG_ERR_WORKSPACE_TOO_SMALL;
  if (!(var_tolerance > 0.0)) var_tolerance = HG_LEARNED_VAR_TOLERANCE;
  if (!(max_factor > 0.0)) max_factor = HG_LEARNED_MAX_FACTOR;
  const size_t part = (size_t)kLrnBlocks * 4 * 8;
  double* d_out = (double*)((uint8_t*)d_ws + part);  // learned [0..3], Murmur [4..7]
  hg_config mm = *cfg;
  mm.map = HG_MAP_MURMUR3;
  mm.d_model = nullptr;
  rc = hg_bucket_stats(cfg, d_keys, n, d_counts, d_out, d_ws, part, stream);
  if (rc != HG_OK) return rc;
  rc = hg_bucket_stats(&mm, d_keys, n, d_counts, d_out + 4, d_ws, part, stream);
  if (rc != HG_OK) return rc;
  double st[8];
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(st, d_out, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess) return HG_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return HG_ERR_CUDA;
  // kept while the learned map's bucket-length variance and longest bucket
  // stay within the tolerances of Murmur's on the same keys
  *h_keep = (st[2] <= var_tolerance * st[6] && st[0] <= max_factor * st[4]) ? 1 : 0;
  if (h_stats8)
    for (int i = 0; i < 8; ++i) h_stats8[i] = st[i];
  return HG_OK;
}

}  // extern "C"
