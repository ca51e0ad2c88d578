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

// ---------------------------------------------------------------------------
// Beta: the continued fraction K(p, q, x) of the incomplete beta with dK/dp,
// dK/dq, K = 1/(1 + d_1/(1 + d_2/(1 + ...))),
//   d_{2m+1} = -(p+m)(p+q+m) x / ((p+2m)(p+2m+1)),
//   d_{2m}   = m (q-m) x / ((p+2m-1)(p+2m)),
// evaluated backward in triples (value, d/dp, d/dq).  Every d_j and both its
// derivatives are x times a per-fill coefficient, tabled for the two
// orientations o = 0 ((p, q, x) = (a, b, z)) and o = 1 ((b, a, 1 - z), the
// reflection I_z(a, b) = 1 - I_{1-z}(b, a)); FP32 copies of the coefficients
// and of derivative-safe magnitudes serve the depth bound.
constexpr int kBetaMax = 600;                 // depth at most
constexpr int kBJ = kBetaMax + 1;             // entries per orientation
constexpr int kBE = 16, kBEp = kBE + 2 * kBJ, kBEq = kBEp + 2 * kBJ, kBF = kBEq + 2 * kBJ;
constexpr int kBetaTabDoubles = kBF + 2 * kBJ;   // then 2 x 2 x kBJ floats (= 2 kBJ doubles)
// constants: [0] split (a+1)/(a+b+2), [1] its mirror (b+1)/(a+b+2), then per
// orientation [2+3o] 1/p, [3+3o] -1/p - psi(p) + psi(p+q), [4+3o] psi(p+q) - psi(q)

__global__ void __launch_bounds__(kTabThreads) k_beta_tab(double a, double b, double* __restrict__ tab) {
  float* Ff = (float*)(tab + kBF);    // [o][j] coefficient, then [o][j] magnitude
  for (int idx = threadIdx.x; idx < 2 * kBJ; idx += kTabThreads) {
    const int o = idx / kBJ, j = idx % kBJ;
    const double p = o ? b : a, q = o ? a : b;
    double v = 0.0, dp = 0.0, dq = 0.0, mag = 0.0;
    if (j & 1) {
      const int m = (j - 1) / 2;
      const double A = p + m, B = p + q + m, C = p + 2 * m, D = C + 1.0;
      v = -A * B / (C * D);
      // d/dp: num' = -(B + A), den' = C + D; d/dq: num' = -A, den' = 0
      dp = (-(A + B) - v * (C + D)) / (C * D);
      dq = -A / (C * D);
      mag = fabs(v);
    } else if (j > 0) {
      const int m = j / 2;
      const double C = p + 2 * m - 1.0, D = C + 1.0;
      v = m * (q - m) / (C * D);
      dp = -v * (C + D) / (C * D);
      dq = m / (C * D);
      // at least m / (C D): a fraction that terminates (integer q) still
      // gets the depth its q-derivative needs
      mag = m * fmax(fabs(q - m), 1.0) / (C * D);
    }
    tab[kBE + idx] = v;
    tab[kBEp + idx] = dp;
    tab[kBEq + idx] = dq;
    Ff[idx] = (float)v;
    Ff[2 * kBJ + idx] = (float)mag;
  }
  if (threadIdx.x == 0) {
    const double pa = digamma_dev(a), pb = digamma_dev(b), pab = digamma_dev(a + b);
    tab[0] = (a + 1.0) / (a + b + 2.0);
    tab[1] = (b + 1.0) / (a + b + 2.0);
    tab[2] = 1.0 / a;
    tab[3] = -1.0 / a - pa + pab;
    tab[4] = pab - pb;
    tab[5] = 1.0 / b;
    tab[6] = -1.0 / b - pb + pab;
    tab[7] = pab - pa;
  }
}

// dz/da and dz/db for one sample per lane (lanes of similar z, as for the
// gamma gradient); both orientations run the same loop at the warp's
// largest depth.
__device__ void beta_dzdab_warp(double z, bool valid, const double* __restrict__ tab, double* dza, double* dzb) {
  const unsigned FULL = 0xffffffffu;
  valid = valid && z > 0.0 && z < 1.0;
  const int o = valid && !(z < __ldg(tab)) ? 1 : 0;
  const double x = valid ? (o ? 1.0 - z : z) : 0.5;
  const float* Ef = (const float*)(tab + kBF) + o * kBJ;
  const float* Mf = Ef + 2 * kBJ;
  // depth: eps_k = eps_{k-1} |d_k| / (|c_k| |e_{k-1}|), c and e the ratios
  // of successive convergents' numerators and denominators; stop at 2^-60
  const float xf = (float)x;
  float c = 1.0f + xf * __ldg(Ef + 1), e = 1.0f;
  float eps = __fdividef(xf * __ldg(Mf + 1), fabsf(c));
  int kf = 1;
  bool fin = !valid || !(eps >= 8.67361738e-19f);
  while (!__all_sync(FULL, fin)) {
    if (!fin) {
      ++kf;
      const float dk = xf * __ldg(Ef + kf), eprev = e;
      c = 1.0f + __fdividef(dk, c);
      e = 1.0f + __fdividef(dk, e);
      if (fabsf(c) < 1e-30f) c = 1e-30f;
      if (fabsf(e) < 1e-30f) e = 1e-30f;
      eps = eps * __fdividef(xf * __ldg(Mf + kf), fabsf(c) * fabsf(eprev));
      fin = !(eps >= 8.67361738e-19f) || kf >= kBetaMax - 2;
    }
  }
  const int N = (int)__reduce_max_sync(FULL, valid ? (unsigned)(kf + 2) : 0u);
  const double* E = tab + kBE + o * kBJ;
  const double* Ep = tab + kBEp + o * kBJ;
  const double* Eq = tab + kBEq + o * kBJ;
  // t <- 1 + d_j / t in triples, with the derivative parts kept divided by
  // x (every d_j is x times a coefficient): with r = 1/t and v = E_j x r,
  // t_p / x <- r (E^p_j - v t_p / x); 1/t as for the gamma fraction
  double tv = 1.0, up = 0.0, uq = 0.0;
  for (int j = N; j >= 1; --j) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(tv));
    const double ee = __fma_rn(-tv, r, 1.0);
    r = __fma_rn(r, __fma_rn(ee, ee, ee), r);
    const double rv = __ldg(E + j) * (x * r);
    up = r * __fma_rn(-rv, up, __ldg(Ep + j));
    uq = r * __fma_rn(-rv, uq, __ldg(Eq + j));
    tv = 1.0 + rv;
  }
  const double K = rcp_nr(tv), Kp = -K * (x * up) * K, Kq = -K * (x * uq) * K;
  const double s = x * (1.0 - x) * __ldg(tab + 2 + 3 * o);
  const double dIp = s * ((log(x) + __ldg(tab + 3 + 3 * o)) * K + Kp);
  const double dIq = s * ((log1p(-x) + __ldg(tab + 4 + 3 * o)) * K + Kq);
  *dza = !valid ? 0.0 : (o ? dIq : -dIp);
  *dzb = !valid ? 0.0 : (o ? dIp : -dIq);
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

// One warp per window of 256 consecutive samples: the window is sorted by a
// key of z with a deterministic counting sort in shared memory, then taken 32
// at a time, so that each batch of lanes runs the same branch with similar
// trip counts.  Each lane's sum takes its samples in an order fixed by the
// data, and the block sums have a fixed shape: the result is deterministic.
constexpr int kWinPerLane = 8, kWin = 32 * kWinPerLane, kKeys = 32;
constexpr int kWarps = kGradThreads / 32;

struct WindowSmem {
  double z[kWarps][kWin];
  unsigned char i[kWarps][kWin];
  int cnt[kWarps][kKeys];
};

// Sorts window `base` of z into sm.z[wid] / sm.i[wid] (slot -> offset in the
// window) by key(z) in [0, kKeys); entries past n get key kKeys - 1.
template <class KeyFn>
__device__ __forceinline__ void sort_window(const double* __restrict__ z, size_t n, size_t base, KeyFn key_of,
                                            WindowSmem& sm, int wid, int lane) {
  const unsigned FULL = 0xffffffffu, lt = (1u << lane) - 1u;
  double zv[kWinPerLane];
  int key[kWinPerLane], off[kWinPerLane];
#pragma unroll
  for (int m = 0; m < kWinPerLane; ++m) {
    const size_t i = base + m * 32 + lane;
    zv[m] = i < n ? z[i] : 0.0;
    key[m] = i < n ? key_of(zv[m]) : kKeys - 1;
  }
  sm.cnt[wid][lane] = 0;
  __syncwarp();
#pragma unroll
  for (int m = 0; m < kWinPerLane; ++m) {
    const unsigned peers = __match_any_sync(FULL, key[m]);
    const int before = sm.cnt[wid][key[m]];
    __syncwarp();
    if ((peers & lt) == 0) sm.cnt[wid][key[m]] = before + __popc(peers);
    __syncwarp();
    off[m] = before + __popc(peers & lt);
  }
  const int c = sm.cnt[wid][lane];
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += u;
  }
  const int excl = incl - c;
#pragma unroll
  for (int m = 0; m < kWinPerLane; ++m) {
    const int p = __shfl_sync(FULL, excl, key[m]) + off[m];
    sm.z[wid][p] = zv[m];
    sm.i[wid][p] = (unsigned char)(m * 32 + lane);
  }
  __syncwarp();
}

// eighth-binades of x below the bit pattern `ref` (x < ref: keys 0-15, the
// nearest 15), or above it (keys 16-31)
__device__ __forceinline__ int binade_key(double x, long long ref) {
  const long long d = (__double_as_longlong(x) - ref) >> 49;
  return (int)(d < 0 ? 15 + max(d + 1, -15ll) : 16 + min(d, 15ll));
}

__global__ void __launch_bounds__(kGradThreads) k_gamma_grad(const double* __restrict__ z, const double* __restrict__ g,
                                                               size_t n, double alpha, const double* __restrict__ tab,
                                                               double* __restrict__ dz, double* __restrict__ part) {
  __shared__ double sh[kWarps];
  __shared__ WindowSmem sm;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long a1bits = __double_as_longlong(alpha + 1.0);
  const size_t nwin = (n + kWin - 1) / kWin;
  double acc = 0.0;
  for (size_t win = (size_t)blockIdx.x * kWarps + wid; win < nwin; win += (size_t)gridDim.x * kWarps) {
    const size_t base = win * kWin;
    // series side (z < alpha + 1) first, then the continued fraction's
    sort_window(z, n, base, [&](double v) { return binade_key(v, a1bits); }, sm, wid, lane);
    for (int b = 0; b < kWinPerLane; ++b) {
      const int p = b * 32 + lane;
      const size_t i = base + sm.i[wid][p];
      const bool valid = i < n;
      const double d = gamma_dzda_warp(sm.z[wid][p], valid, alpha, tab);
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
                                                              size_t n, const double* __restrict__ tab,
                                                              double* __restrict__ dza, double* __restrict__ dzb,
                                                              double* __restrict__ part) {
  __shared__ double sh[kWarps];
  __shared__ WindowSmem sm;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double split = tab[0];
  const long long s0 = __double_as_longlong(split), s1 = __double_as_longlong(tab[1]);
  const size_t nwin = (n + kWin - 1) / kWin;
  double aa = 0.0, ab = 0.0;
  for (size_t win = (size_t)blockIdx.x * kWarps + wid; win < nwin; win += (size_t)gridDim.x * kWarps) {
    const size_t base = win * kWin;
    // orientation 0 (x = z below the split) on keys 0-15, orientation 1
    // (x = 1 - z at or below the mirrored split) on 16-31; within each, x's
    // eighth-binades below its split, the slowest (nearest) last
    auto key = [&](double v) {
      if (!(v > 0.0 && v < 1.0)) return 0;
      const bool o = !(v < split);
      const int k = min(binade_key(o ? 1.0 - v : v, o ? s1 : s0), 15);
      return o ? 16 + k : k;
    };
    sort_window(z, n, base, key, sm, wid, lane);
    for (int b = 0; b < kWinPerLane; ++b) {
      const int p = b * 32 + lane;
      const size_t i = base + sm.i[wid][p];
      const bool valid = i < n;
      double da, db;
      beta_dzdab_warp(sm.z[wid][p], valid, tab, &da, &db);
      if (valid) {
        if (dza) dza[i] = da;
        if (dzb) dzb[i] = db;
        if (g) { aa += g[i] * da; ab += g[i] * db; }
      }
    }
    __syncwarp();
  }
  const double s1s = block_sum(aa, sh);
  const double s2s = block_sum(ab, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s1s; part[2 * blockIdx.x + 1] = s2s; }
}

// Beta through its gamma pair (z = X / (X + Y), each gamma reparameterised by
// its own CDF): dz/da = Y / (X + Y)^2 dX/da, dz/db = -X / (X + Y)^2 dY/db.
// dzda and dzdb hold dX/da and dY/db on entry (the gamma gradient kernel's
// outputs) and the beta gradients on exit; the sums with g as for k_beta_grad.
__global__ void __launch_bounds__(kGradThreads) k_beta_compose(const double* __restrict__ x,
                                                                 const double* __restrict__ y,
                                                                 const double* __restrict__ g, size_t n,
                                                                 double* __restrict__ dzda, double* __restrict__ dzdb,
                                                                 double* __restrict__ part) {
  __shared__ double sh[kWarps];
  double aa = 0.0, ab = 0.0;
  for (size_t i = blockIdx.x * (size_t)kGradThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kGradThreads) {
    const double X = x[i], Y = y[i];
    const double s = X + Y, s2 = s * s;
    const double da = Y / s2 * dzda[i], db = -X / s2 * dzdb[i];
    dzda[i] = da;
    dzdb[i] = db;
    if (g) {
      aa += g[i] * da;
      ab += g[i] * db;
    }
  }
  const double s1 = block_sum(aa, sh);
  const double s2s = block_sum(ab, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s1; part[2 * blockIdx.x + 1] = s2s; }
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
size_t grad_scratch_doubles() { return 2 * (size_t)grad_blocks() + 2 + (size_t)max(kTabDoubles, kBetaTabDoubles); }

int launch_gamma_grad(const double* z, const double* g, size_t n, double alpha, double* dz, double* part, double* out,
                      void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  double* tab = part + 2 * (size_t)grad_blocks() + 2;
  k_gamma_tab<<<1, kTabThreads, 0, s>>>(alpha, tab);
  k_gamma_grad<<<grad_blocks(), kGradThreads, 0, s>>>(z, g, n, alpha, tab, dz, part);
  k_sum_parts<<<1, kGradThreads, 0, s>>>(part, grad_blocks(), 1, out);
  return (int)cudaGetLastError();
}

int launch_beta_compose(const double* x, const double* y, const double* g, size_t n, double* dzda, double* dzdb,
                        double* part, double* out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  k_beta_compose<<<grad_blocks(), kGradThreads, 0, s>>>(x, y, g, n, dzda, dzdb, part);
  k_sum_parts<<<1, kGradThreads, 0, s>>>(part, grad_blocks(), 2, out);
  return (int)cudaGetLastError();
}

int launch_beta_grad(const double* z, const double* g, size_t n, double a, double b, double* dza, double* dzb,
                     double* part, double* out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  double* tab = part + 2 * (size_t)grad_blocks() + 2;
  k_beta_tab<<<1, kTabThreads, 0, s>>>(a, b, tab);
  k_beta_grad<<<grad_blocks(), kGradThreads, 0, s>>>(z, g, n, tab, dza, dzb, part);
  k_sum_parts<<<1, kGradThreads, 0, s>>>(part, grad_blocks(), 2, out);
  return (int)cudaGetLastError();
}

}  // namespace rp
