// Pathwise (reparameterisation) gradients of gamma and beta variates:
// z = F^{-1}(u; theta) at fixed u gives dz/dtheta = -(dF/dtheta)(z) / f(z).
//
// Gamma(alpha, 1), F = P(alpha, z), f = z^(alpha-1) e^-z / Gamma(alpha):
//   z < alpha + 1:  P/f = z sum_k c_k, c_k = z^k / (alpha (alpha+1) ... (alpha+k)),
//                   dz/dalpha = -z sum_k c_k (ln z - psi(alpha + k + 1))
//                   (term-by-term alpha-derivative of the power series of P);
//   z >= alpha + 1: Q = 1 - P = e^-z z^alpha Phi / Gamma(alpha) with Phi the
//                   Legendre continued fraction of the upper incomplete gamma,
//                   dz/dalpha = +dQ/dalpha / f = z ((ln z - psi(alpha)) Phi + dPhi/dalpha),
//                   with Phi and its alpha-derivative from one backward
//                   evaluation of the fraction in dual numbers.
// Beta(a, b), F = I_z(a, b): the incomplete beta continued fraction
//   I_x(p, q) = x^p (1-x)^q / (p B(p, q)) K(p, q, x),  x < (p+1)/(p+q+2),
// evaluated with its p- and q-derivatives; I/f = x (1-x) K / p, so
//   dI/dp / f = (x (1-x) / p) ((ln x - 1/p - psi(p) + psi(p+q)) K + dK/dp),
//   dI/dq / f = (x (1-x) / p) ((ln(1-x) - psi(q) + psi(p+q)) K + dK/dq),
// and the reflection I_x(a, b) = 1 - I_{1-x}(b, a) for the other half.
//
// All in FP64; sums by fixed-shape reductions (deterministic).  The bar for
// these values is 1e-12 relative, not bit identity, so this file is built
// with FMA contraction and takes reciprocals from the hardware estimate and
// Newton steps.  The FP64 pipe is what bounds these kernels, so the gamma
// gradient spends FP64 operations only on the arithmetic of its terms: the
// series runs on per-fill tables, the continued fraction's depth comes from
// an FP32 error bound, and each warp sorts its samples so that its lanes run
// the same branch with similar trip counts.
#include <cuda_runtime.h>

#include <cmath>

#include "rp_internal.h"

namespace rp {
namespace {

constexpr int kGradThreads = 256;

__device__ double digamma_dev(double x) {
  // psi(x + n) - sum 1/(x + j), then the Stirling-type asymptotic series
  double acc = 0.0;
  while (x < 10.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  double r = 1.0 / (x * x);
  // B2/2, B4/4, ... / x^2k terms
  double s = r * (1.0 / 12.0 - r * (1.0 / 120.0 - r * (1.0 / 252.0 - r * (1.0 / 240.0 - r * (1.0 / 132.0 - r * (691.0 / 32760.0 - r / 12.0))))));
  return acc + log(x) - 0.5 / x - s;
}

// 1/x for a nonzero normal x, within one ulp: the hardware estimate
// (relative error about 2^-23) and two Newton steps.
__device__ __forceinline__ double rcp_nr(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = __fma_rn(-x, r, 1.0);
  r = __fma_rn(r, e, r);
  e = __fma_rn(-x, r, 1.0);
  return __fma_rn(r, e, r);
}

// ---------------------------------------------------------------------------
// Gamma: per-fill tables.  With s = alpha + 1 and w = z / s (< 1 on the
// series side), c_k = z^k / (alpha (alpha+1) ... (alpha+k)) = w^k R_k,
// R_k = s^k / (alpha (alpha+1) ... (alpha+k)) <= 1/alpha, so a term is
// w^k (R_k ln z - Q_k) with Q_k = R_k psi(alpha + k + 1): three FP64
// operations and nothing that can overflow.  The continued fraction's partial
// numerators a_i = -i (i - alpha) and their alpha-derivatives i are tabled too.
constexpr int kSerTerms = 2048;   // series terms at most (the table's length)
constexpr int kCfMax = 400;       // continued-fraction depth at most
constexpr int kTabR = 8, kTabQ = kTabR + kSerTerms, kTabA = kTabQ + kSerTerms, kTabAd = kTabA + kCfMax + 8;
constexpr int kTabDoubles = kTabAd + kCfMax + 8;
constexpr int kTabThreads = 256;

__global__ void __launch_bounds__(kTabThreads) k_gamma_tab(double a, double* __restrict__ tab) {
  __shared__ double ratio[kSerTerms];
  const int t = threadIdx.x;
  double* R = tab + kTabR;
  double* Q = tab + kTabQ;
  for (int k = t; k < kSerTerms; k += kTabThreads) {
    ratio[k] = k == 0 ? 1.0 / a : (a + 1.0) / (a + k);
    Q[k] = digamma_dev(a + k + 1.0);   // psi, scaled by R_k below
  }
  for (int i = t; i <= kCfMax; i += kTabThreads) {
    tab[kTabA + i] = -(double)i * ((double)i - a);
    tab[kTabAd + i] = (double)i;
  }
  if (t == 0) {
    tab[0] = digamma_dev(a);
    tab[1] = 1.0 / (a + 1.0);
  }
  __syncthreads();
  if (t < 32) {
    // R_k = prod_{j <= k} ratio_j: lane L multiplies its 64 entries, then an
    // exclusive product scan over the lanes seeds each run
    constexpr int kRun = kSerTerms / 32;
    double p = 1.0;
    for (int j = 0; j < kRun; ++j) p *= ratio[t * kRun + j];
    double v = p;
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, v, o);
      if (t >= o) v *= u;
    }
    double ex = __shfl_up_sync(0xffffffffu, v, 1);
    if (t == 0) ex = 1.0;
    for (int j = 0; j < kRun; ++j) {
      ex *= ratio[t * kRun + j];
      R[t * kRun + j] = ex;
    }
  }
  __syncthreads();
  for (int k = t; k < kSerTerms; k += kTabThreads) Q[k] = R[k] * Q[k];
}

__device__ __forceinline__ int ebits(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); }

// dz/dalpha for one sample per lane of a warp whose lanes hold z values of
// similar size (sorted windows, below).  valid: the lane holds a sample.
// Series lanes (0 < z < alpha + 1) run the table series until every one of
// them has a last term and coefficient below 2^-57 of its sum; fraction
// lanes (z >= alpha + 1) take the depth from an FP32 forward pass and then
// evaluate the fraction backward in dual numbers at the warp's largest depth.
__device__ double gamma_dzda_warp(double z, bool valid, double a, const double* __restrict__ tab) {
  const unsigned FULL = 0xffffffffu;
  const double a1 = a + 1.0;
  const bool pos = valid && z > 0.0;
  const bool ser = pos && z < a1, cf = pos && !(z < a1);
  const unsigned smask = __ballot_sync(FULL, ser), cmask = __ballot_sync(FULL, cf);
  double d = 0.0;
  if (ser) {
    const double* __restrict__ R = tab + kTabR;
    const double* __restrict__ Q = tab + kTabQ;
    const double lz = log(z);
    const double w = z * __ldg(tab + 1);
    double zk = 1.0, inner = 0.0;
    double sum = __fma_rn(__ldg(R), lz, -__ldg(Q));
    int k = 1;
    for (;;) {
#pragma unroll
      for (int u = 0; u < 4; ++u, ++k) {
        zk *= w;
        inner = __fma_rn(__ldg(R + k), lz, -__ldg(Q + k));
        sum = __fma_rn(zk, inner, sum);
      }
      // |c_k| < 2^(ec-1021), |t_k| < 2^(et-1021), |sum| >= 2^(es-1023)
      const int ez = ebits(zk);
      const int ec = ez + ebits(__ldg(R + k - 1)) - 1023, et = ez + ebits(inner) - 1023;
      const bool done = max(ec, et) + 59 <= ebits(sum) || k + 4 > kSerTerms;
      if (__all_sync(smask, done)) break;
    }
    d = -z * sum;
  }
  if (cf) {
    const double* __restrict__ A = tab + kTabA;
    const double* __restrict__ Ad = tab + kTabAd;
    // Depth: with c_j, d_j the ratios of successive numerators and
    // denominators of the convergents of b_0 + a_1/(b_1 + ...), the k-th
    // convergent moves by the fraction eps_k = |a_1 ... a_k| / |A_k B_{k-1}|
    // of itself, eps_k = eps_{k-1} |a_k| / (|c_k| |d_{k-1}|).  |a_j| is taken
    // at least j, so that a fraction that terminates (integer alpha) still
    // gets the depth its alpha-derivative needs; stop at eps < 2^-60.
    const float af = (float)a, zb = (float)(z + 1.0 - a);
    auto amag = [&](int j) { return (float)j * fmaxf(fabsf((float)j - af), 1.0f); };
    float c = zb + 2.0f + __fdividef(-(1.0f - af), zb), dd = zb + 2.0f;
    float eps = __fdividef(amag(1), fabsf(zb * c));
    int kf = 1;
    bool fin = !(eps >= 8.67361738e-19f);
    while (!__all_sync(cmask, fin)) {
      if (!fin) {
        ++kf;
        const float bk = zb + 2.0f * (float)kf, ak = -(float)kf * ((float)kf - af);
        const float dprev = dd;
        c = bk + __fdividef(ak, c);
        dd = bk + __fdividef(ak, dd);
        if (fabsf(c) < 1e-30f) c = 1e-30f;
        if (fabsf(dd) < 1e-30f) dd = 1e-30f;
        eps = eps * __fdividef(amag(kf), fabsf(c) * fabsf(dprev));
        fin = !(eps >= 8.67361738e-19f) || kf >= kCfMax - 2;
      }
    }
    const int N = (int)__reduce_max_sync(cmask, (unsigned)(kf + 2));
    const double zb1 = z + 1.0 - a;
    double tv = zb1 + 2.0 * N, td = -1.0, bi = zb1 + 2.0 * (N - 1);
    for (int i = N; i >= 1; --i) {
      // t <- b_{i-1} + a_i / t in duals; 1/t from the estimate and one
      // third-order Newton step (error below 2^-60)
      double r;
      asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(tv));
      const double e = __fma_rn(-tv, r, 1.0);
      r = __fma_rn(r, __fma_rn(e, e, e), r);
      const double q = __ldg(A + i) * r;
      const double wv = __fma_rn(-q, td, __ldg(Ad + i));
      td = __fma_rn(wv, r, -1.0);
      tv = bi + q;
      bi -= 2.0;
    }
    const double phi = rcp_nr(tv), dphi = -phi * td * phi;
    d = z * ((log(z) - __ldg(tab)) * phi + dphi);
  }
  return d;
}

// Continued fraction K(p, q, x) of the incomplete beta with dK/dp, dK/dq:
// K = 1/(1 + d1/(1 + d2/(1 + ...))), d_{2m+1} = -(p+m)(p+q+m) x / ((p+2m)(p+2m+1)),
// d_{2m} = m (q-m) x / ((p+2m-1)(p+2m)); backward evaluation with a fixed depth.
struct Tri {
  double v, p, q;
};
__device__ __forceinline__ Tri tdiv(Tri a, Tri b) {
  const double ib = rcp_nr(b.v);
  const double r = a.v * ib;
  return {r, (a.p - r * b.p) * ib, (a.q - r * b.q) * ib};
}

__device__ Tri beta_cf(double p, double q, double x, int depth) {
  Tri t = {1.0, 0.0, 0.0};
  for (int j = depth; j >= 1; --j) {
    Tri dj;
    if (j & 1) {
      int m = (j - 1) / 2;
      double A = p + m, B = p + q + m, C = p + 2 * m, D = C + 1.0;
      double num = -A * B * x, iden = rcp_nr(C * D);
      double v = num * iden;
      // d/dp: num' = -(B + A) x, den' = C + D ; d/dq: num' = -A x, den' = 0
      double dp = (-(A + B) * x - v * (C + D)) * iden;
      double dq = (-A * x) * iden;
      dj = {v, dp, dq};
    } else {
      int m = j / 2;
      double C = p + 2 * m - 1.0, D = C + 1.0;
      double num = m * (q - m) * x, iden = rcp_nr(C * D);
      double v = num * iden;
      double dp = (-v * (C + D)) * iden;
      double dq = (m * x) * iden;
      dj = {v, dp, dq};
    }
    Tri one_plus = {1.0 + 0.0, 0.0, 0.0};
    Tri r = tdiv(dj, t);
    t = {one_plus.v + r.v, r.p, r.q};
  }
  return tdiv(Tri{1.0, 0.0, 0.0}, t);
}

// d z / d a and d z / d b for z ~ Beta(a, b); pa, pb, pab = psi(a), psi(b),
// psi(a + b) (fixed per fill)
__device__ void beta_dzdab_dev(double z, double a, double b, double pa, double pb, double pab, double* dza,
                               double* dzb) {
  if (!(z > 0.0) || !(z < 1.0)) { *dza = 0.0; *dzb = 0.0; return; }
  int depth = 40 + (int)(6.0 * sqrt(a + b));
  if (depth > 600) depth = 600;
  if (z < (a + 1.0) / (a + b + 2.0)) {
    Tri K = beta_cf(a, b, z, depth);
    double s = z * (1.0 - z) / a;
    double dIa = s * ((log(z) - 1.0 / a - pa + pab) * K.v + K.p);
    double dIb = s * ((log1p(-z) - pb + pab) * K.v + K.q);
    *dza = -dIa;
    *dzb = -dIb;
  } else {
    // I_z(a, b) = 1 - I_y(b, a), y = 1 - z: p = b, q = a
    double y = 1.0 - z;
    Tri K = beta_cf(b, a, y, depth);
    double s = y * (1.0 - y) / b;
    double dIy_dp = s * ((log(y) - 1.0 / b - pb + pab) * K.v + K.p);   // d/db
    double dIy_dq = s * ((log1p(-y) - pa + pab) * K.v + K.q);          // d/da
    *dza = dIy_dq;
    *dzb = dIy_dp;
  }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kGradThreads / 32; ++w) s += sh[w];
  __syncthreads();
  return s;
}

// One warp per window of 256 consecutive samples: the window is sorted by
// a key of z (eighth-binades below and above alpha + 1, series side first)
// with a deterministic counting sort in shared memory, then taken 32 at a
// time, so that each batch of lanes runs the same branch with similar trip
// counts.  Each lane's sum takes its samples in an order fixed by the data,
// and the block sums have a fixed shape: the result is deterministic.
constexpr int kWinPerLane = 8, kWin = 32 * kWinPerLane, kKeys = 32;

__device__ __forceinline__ int gamma_key(double z, long long a1bits) {
  const long long d = (__double_as_longlong(z) - a1bits) >> 49;   // eighth-binades from alpha + 1
  const long long k = d < 0 ? 15 + max(d + 1, -15ll) : 16 + min(d, 15ll);
  return (int)k;
}

__global__ void __launch_bounds__(kGradThreads) k_gamma_grad(const double* __restrict__ z, const double* __restrict__ g,
                                                               size_t n, double alpha, const double* __restrict__ tab,
                                                               double* __restrict__ dz, double* __restrict__ part) {
  constexpr int W = kGradThreads / 32;
  __shared__ double sh[W];
  __shared__ double s_z[W][kWin];
  __shared__ unsigned char s_i[W][kWin];
  __shared__ int s_cnt[W][kKeys];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const long long a1bits = __double_as_longlong(alpha + 1.0);
  const size_t nwin = (n + kWin - 1) / kWin;
  double acc = 0.0;
  for (size_t win = (size_t)blockIdx.x * W + wid; win < nwin; win += (size_t)gridDim.x * W) {
    const size_t base = win * kWin;
    double zv[kWinPerLane];
    int key[kWinPerLane], off[kWinPerLane];
#pragma unroll
    for (int m = 0; m < kWinPerLane; ++m) {
      const size_t i = base + m * 32 + lane;
      zv[m] = i < n ? z[i] : 0.0;
      key[m] = i < n ? gamma_key(zv[m], a1bits) : kKeys - 1;
    }
    s_cnt[wid][lane] = 0;
    __syncwarp();
#pragma unroll
    for (int m = 0; m < kWinPerLane; ++m) {
      const unsigned peers = __match_any_sync(FULL, key[m]);
      const int before = s_cnt[wid][key[m]];
      __syncwarp();
      if ((peers & lt) == 0) s_cnt[wid][key[m]] = before + __popc(peers);
      __syncwarp();
      off[m] = before + __popc(peers & lt);
    }
    int c = s_cnt[wid][lane], incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += u;
    }
    const int excl = incl - c;
#pragma unroll
    for (int m = 0; m < kWinPerLane; ++m) {
      const int p = __shfl_sync(FULL, excl, key[m]) + off[m];
      s_z[wid][p] = zv[m];
      s_i[wid][p] = (unsigned char)(m * 32 + lane);
    }
    __syncwarp();
    for (int b = 0; b < kWinPerLane; ++b) {
      const int p = b * 32 + lane;
      const size_t i = base + s_i[wid][p];
      const bool valid = i < n;
      const double d = gamma_dzda_warp(s_z[wid][p], valid, alpha, tab);
      if (valid) {
        if (dz) dz[i] = d;
        if (g) acc += g[i] * d;
      }
    }
    __syncwarp();
  }
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kGradThreads) k_beta_grad(const double* __restrict__ z, const double* __restrict__ g,
                                                              size_t n, double a, double b, double* __restrict__ dza,
                                                              double* __restrict__ dzb, double* __restrict__ part) {
  __shared__ double sh[kGradThreads / 32];
  const double pa = digamma_dev(a), pb = digamma_dev(b), pab = digamma_dev(a + b);
  double aa = 0.0, ab = 0.0;
  for (size_t i = blockIdx.x * (size_t)kGradThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kGradThreads) {
    double da, db;
    beta_dzdab_dev(z[i], a, b, pa, pb, pab, &da, &db);
    if (dza) dza[i] = da;
    if (dzb) dzb[i] = db;
    if (g) { aa += g[i] * da; ab += g[i] * db; }
  }
  double s1 = block_sum(aa, sh);
  double s2 = block_sum(ab, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s1; part[2 * blockIdx.x + 1] = s2; }
}

// fixed-order final reduction of the block partials (k values of stride k)
__global__ void k_sum_parts(const double* __restrict__ part, int nblk, int k, double* __restrict__ out) {
  __shared__ double sh[kGradThreads / 32];
  for (int c = 0; c < k; ++c) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kGradThreads) v += part[(size_t)i * k + c];
    double s = block_sum(v, sh);
    if (threadIdx.x == 0) out[c] = s;
  }
}

}  // namespace

int grad_blocks() { return 1216; }
size_t grad_scratch_doubles() { return 2 * (size_t)grad_blocks() + 2 + kTabDoubles; }

int launch_gamma_grad(const double* z, const double* g, size_t n, double alpha, double* dz, double* part, double* out,
                      void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  double* tab = part + 2 * (size_t)grad_blocks() + 2;
  k_gamma_tab<<<1, kTabThreads, 0, s>>>(alpha, tab);
  k_gamma_grad<<<grad_blocks(), kGradThreads, 0, s>>>(z, g, n, alpha, tab, dz, part);
  k_sum_parts<<<1, kGradThreads, 0, s>>>(part, grad_blocks(), 1, out);
  return (int)cudaGetLastError();
}

int launch_beta_grad(const double* z, const double* g, size_t n, double a, double b, double* dza, double* dzb,
                     double* part, double* out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  k_beta_grad<<<grad_blocks(), kGradThreads, 0, s>>>(z, g, n, a, b, dza, dzb, part);
  k_sum_parts<<<1, kGradThreads, 0, s>>>(part, grad_blocks(), 2, out);
  return (int)cudaGetLastError();
}

}  // namespace rp
