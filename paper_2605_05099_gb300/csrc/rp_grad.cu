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
// All in FP64.  One thread per sample; sums by fixed-shape block reductions
// (deterministic).  The bar for these values is 1e-12 relative, not bit
// identity, so this file is built with FMA contraction, each series or
// fraction step takes one reciprocal (a hardware estimate and two Newton
// steps, within one ulp) instead of its divisions, and the digammas of the
// fixed shapes are taken once per thread.
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

struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual dadd(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual ddivd(Dual a, Dual b) {
  const double ib = rcp_nr(b.v);
  const double q = a.v * ib;
  return {q, (a.d - q * b.d) * ib};
}

// psi_a = psi(alpha), psi_a1 = psi(alpha + 1) (fixed per fill)
__device__ double gamma_dzda_dev(double z, double a, double psi_a, double psi_a1) {
  if (!(z > 0.0) || !(a > 0.0)) return 0.0;
  if (z < a + 1.0) {
    double lz = log(z);
    double psi = psi_a1;
    double c = rcp_nr(a), sum = c * (lz - psi);
    for (int k = 1; k < 2000; ++k) {
      const double ik = rcp_nr(a + k);
      psi += ik;
      c *= z * ik;
      double t = c * (lz - psi);
      sum += t;
      if (fabs(t) <= 1e-17 * fabs(sum) && c < 1e-17 * fabs(sum)) break;
    }
    return -z * sum;
  }
  // Legendre continued fraction Phi = 1/(b0 + a1/(b1 + a2/(b2 + ...))),
  // b_i = z + 2i + 1 - alpha, a_i = -i (i - alpha); backward in duals.
  int N = 30 + (int)(8.0 * sqrt(a)) + (int)(40.0 / (z - a + 0.5));
  if (N > 400) N = 400;
  Dual t = {z + 2.0 * N + 1.0 - a, -1.0};
  for (int i = N; i >= 1; --i) {
    Dual ai = {-(double)i * ((double)i - a), (double)i};
    Dual bi = {z + 2.0 * (i - 1) + 1.0 - a, -1.0};
    t = dadd(bi, ddivd(ai, t));
  }
  Dual phi = ddivd(Dual{1.0, 0.0}, t);
  return z * ((log(z) - psi_a) * phi.v + phi.d);
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

__global__ void __launch_bounds__(kGradThreads) k_gamma_grad(const double* __restrict__ z, const double* __restrict__ g,
                                                               size_t n, double alpha, double* __restrict__ dz,
                                                               double* __restrict__ part) {
  __shared__ double sh[kGradThreads / 32];
  const double psi_a = digamma_dev(alpha), psi_a1 = digamma_dev(alpha + 1.0);
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)kGradThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kGradThreads) {
    double d = gamma_dzda_dev(z[i], alpha, psi_a, psi_a1);
    if (dz) dz[i] = d;
    if (g) acc += g[i] * d;
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

int launch_gamma_grad(const double* z, const double* g, size_t n, double alpha, double* dz, double* part, double* out,
                      void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  k_gamma_grad<<<grad_blocks(), kGradThreads, 0, s>>>(z, g, n, alpha, dz, part);
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
