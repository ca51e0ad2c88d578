// Device building blocks of librp: engines with jump-ahead, exact integer
// conversions, double-double elementary functions for rare exact decisions,
// and the ziggurat tables.  sm_103a only.
#pragma once
#include <cstdint>

#include "rp_internal.h"

namespace rp {

typedef unsigned long long u64;
typedef unsigned __int128 u128;

// ------------------------------------------------------------------ bits
__device__ __forceinline__ u64 rotl64(u64 x, int k) { return (x << k) | (x >> (64 - k)); }

// 53-bit uniform floor(u / 2^11) 2^-53 assembled from integer operations
// (exact: the value has at most 53 significant bits), Sec. 3.1 method 1.
__device__ __forceinline__ double u53_bits(u64 u) {
  u64 v = u >> 11;
  if (v == 0) return 0.0;
  int lz = __clzll(v);                       // >= 11
  u64 mt = v << (lz - 11);                   // in [2^52, 2^53)
  return __longlong_as_double((long long)((((u64)(1032 - lz)) << 52) + mt));
}

// Exact RN(r * w) for 0 <= r < 2^53 and w = wm 2^we with wm in [2^52, 2^53),
// using integer multiplies only (the FP64 pipe of this GPU is ~40x slower
// than its integer pipes).  msh = wm << 11, wtz = trailing zeros of wm.
__device__ __forceinline__ double mul_rn_int(u64 r, u64 msh, int wtz, int we) {
  if (r == 0) return 0.0;
  int lz = __clzll(r);
  u64 rn = r << lz;                          // top bit 63
  u64 hi = __umul64hi(rn, msh);              // r wm 2^(lz+11) = hi 2^64 + lo
  int tzr = __ffsll((long long)r) - 1;
  bool lo_nz = (tzr + lz + wtz + 11) < 64;   // lo != 0
  int top = (int)(hi >> 63);
  int sh = 10 + top;
  u64 mt = hi >> sh;                         // 53-bit significand (truncated)
  u64 rem = hi & ((1ull << sh) - 1);
  u64 half = 1ull << (sh - 1);
  bool up = (rem > half) || (rem == half && (lo_nz || (mt & 1)));
  mt += up ? 1 : 0;                          // a carry into bit 53 bumps the exponent below
  int q = sh + 53 - lz + we;                 // value = mt 2^q
  return __longlong_as_double((long long)((((u64)(q + 1074)) << 52) + mt));
}

// Negate a double by flipping its sign bit (no FP64 instruction).
__device__ __forceinline__ double neg_if(double x, u64 bit) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)(bit << 63));
}

// ------------------------------------------------------------------ FP32 estimates
// Positive integer v < 2^64 times 2^e2 as a float with the significand
// truncated to 24 bits (relative error < 2^-23).  v = 0 gives 0.
__device__ __forceinline__ float int_scaled_f(u64 v, int e2) {
  if (v == 0) return 0.0f;
  int lz = __clzll(v);
  unsigned m = (unsigned)((v << lz) >> 40);          // bit 23 = leading one
  int e = 63 - lz + e2 + 127;
  return __uint_as_float(((unsigned)e << 23) | (m & 0x7fffffu));
}
// U = floor(u / 2^11) 2^-53 and 1 - U as floats (truncated, relative error < 2^-23)
__device__ __forceinline__ float u53_f(u64 u) { return int_scaled_f(u >> 11, -53); }
__device__ __forceinline__ float one_minus_u53_f(u64 u) { return int_scaled_f((1ull << 53) - (u >> 11), -53); }
// log(1 - U) in FP32 with relative error below 2^-20 for U in [0, 1)
__device__ __forceinline__ float log1m_u53_f(u64 u) {
  float U = u53_f(u);
  return U < 0.5f ? log1pf(-U) : logf(one_minus_u53_f(u));
}

// Exact double of an integer 0 < r < 2^53 from integer operations.
__device__ __forceinline__ double exact_double(u64 r) {
  int lz = __clzll(r);
  u64 mt = r << (lz - 11);                   // leading one at bit 52
  return __longlong_as_double((long long)((((u64)(1085 - lz)) << 52) + mt));
}
// RN(r * w) for 0 <= r < 2^53: r converts exactly, so one FP64 multiply
// gives the correctly rounded product (same value as the integer-only
// mul_rn_int, on the otherwise idle FP64 pipe).
__device__ __forceinline__ double mul_rn_dmul(u64 r, double w) {
  return r ? __dmul_rn(exact_double(r), w) : 0.0;
}

// ------------------------------------------------------------------ double-double
struct dd { double hi, lo; };

__device__ __forceinline__ dd dd_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dd dd_quick(double a, double b) {
  double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_prod(double a, double b) {
  double p = __dmul_rn(a, b);
  return {p, __fma_rn(a, b, -p)};
}
__device__ __forceinline__ dd dd_addx(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  dd t = dd_two_sum(a.lo, b.lo);
  s.lo = __dadd_rn(s.lo, t.hi);
  s = dd_quick(s.hi, s.lo);
  s.lo = __dadd_rn(s.lo, t.lo);
  return dd_quick(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_mulx(dd a, dd b) {
  dd p = dd_prod(a.hi, b.hi);
  p.lo = __dadd_rn(p.lo, __dadd_rn(__dmul_rn(a.hi, b.lo), __dmul_rn(a.lo, b.hi)));
  return dd_quick(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_scale_inv(dd a, double k) {  // a / k, k a small integer
  double q = __ddiv_rn(a.hi, k);
  dd p = dd_prod(q, k);
  double r = __ddiv_rn(__dadd_rn(__dsub_rn(__dsub_rn(a.hi, p.hi), p.lo), a.lo), k);
  return dd_quick(q, r);
}

// exp(x) to ~2^-100 relative: x = k ln2 + r (ln 2 in three parts), exp(r) =
// exp(r/256)^256 with the degree-11 Taylor polynomial evaluated by Horner in
// double-double with the coefficients 1/j! stored as double-double (no
// divisions), then 2^k.
__device__ __noinline__ static dd dd_exp_dev(double x) {
  const double L1 = 0x1.62e42fefa39efp-1, L2 = 0x1.abc9e3b39803fp-56, L3 = 0x1.7b57a079a1934p-111;
  const double INV_LN2 = 0x1.71547652b82fep+0;
  // 1/j!, j = 2..11, as (hi, lo)
  const double CH[10] = {0x1.0000000000000p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5, 0x1.1111111111111p-7,
                         0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19,
                         0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26};
  const double CL[10] = {0.0, 0x1.5555555555555p-57, 0x1.5555555555555p-59, 0x1.1111111111111p-63,
                         -0x1.f49f49f49f49fp-65, 0x1.a01a01a01a01ap-73, 0x1.a01a01a01a01ap-76, -0x1.c154f8ddc6c00p-73,
                         0x1.cbbc05b4fa99ap-76, -0x1.c062e06d1f209p-80};
  double k = rint(__dmul_rn(x, INV_LN2));
  dd a = dd_prod(k, L1);
  dd r = dd_addx({x, 0.0}, {-a.hi, -a.lo});
  dd b = dd_prod(k, L2);
  r = dd_addx(r, {-b.hi, -b.lo});
  r = dd_addx(r, {-__dmul_rn(k, L3), 0.0});
  r.hi = ldexp(r.hi, -8);
  r.lo = ldexp(r.lo, -8);
  dd p = {CH[9], CL[9]};
  for (int j = 8; j >= 0; --j) p = dd_addx(dd_mulx(p, r), {CH[j], CL[j]});
  p = dd_addx(dd_mulx(p, r), {1.0, 0.0});  // 1 + r (1 + r/2 + ...)
  p = dd_addx(dd_mulx(p, r), {1.0, 0.0});
  for (int j = 0; j < 8; ++j) p = dd_mulx(p, p);
  int ki = (int)k;
  return {ldexp(p.hi, ki), ldexp(p.lo, ki)};
}

// log(y), y > 0: near 1 the series r - r^2/2 + r^3/3 - ... in double-double
// (r = y - 1 exact, |r| < 2^-4; relative accuracy, where a Newton step on
// exp would only be accurate in absolute terms), elsewhere one Newton step on
// exp from the libm value.
__device__ __noinline__ static dd dd_log_dev(double y) {
  if (y > 0.9375 && y < 1.0625) {
    const dd r = {__dsub_rn(y, 1.0), 0.0};
    dd pk = r, sum = r;
    for (int k = 2; k < 60; ++k) {
      pk = dd_mulx(pk, r);
      dd term = dd_scale_inv(pk, (double)k);
      if (k & 1) sum = dd_addx(sum, term);
      else sum = dd_addx(sum, {-term.hi, -term.lo});
      if (fabs(term.hi) < ldexp(fabs(r.hi), -112)) break;
    }
    return sum;
  }
  double y0 = log(y);
  dd e = dd_exp_dev(-y0);
  dd z = dd_addx(dd_mulx(e, {y, 0.0}), {-1.0, 0.0});
  dd zz = dd_mulx(z, z);
  z = dd_addx(z, {-0.5 * zz.hi, -0.5 * zz.lo});
  return dd_addx({y0, 0.0}, z);
}

// Correctly rounded exp / log via the normalised double-double value.
__device__ __forceinline__ double cr_exp_dev(double x) {
  if (x == 0.0) return 1.0;
  if (x < -708.0) return exp(x);
  return dd_exp_dev(x).hi;
}
__device__ __forceinline__ double cr_log_dev(double y) {
  if (y == 1.0) return 0.0;
  if (y == 0.0) return -__longlong_as_double(0x7ff0000000000000ll);
  if (y == __longlong_as_double(0x7ff0000000000000ll)) return y;   // log(+inf) = +inf
  return dd_log_dev(y).hi;
}

// Correctly rounded log of a positive normal double, fast path: Tang's
// table-driven reduction y = 2^e m, r = m inv_j - 1 (exact in one fused
// multiply-add, |r| <= 2^-10), log y = e ln2 - log(inv_j) + log1p(r) with
// log1p(r) = r + r^2 q(r) (degree 7, truncation below 2^-83), summed as a
// double-double whose error is below 2^-69 absolute (below 2^-49 |q| r^2
// when the result is r + r^2 q(r) alone).  Ziv's rounding test: if both ends
// of the error interval round to the same double, that double is the
// correctly rounded log; otherwise the double-double Newton log decides.
#include "log_table.inc"

__device__ __forceinline__ double cr_log_fast(double y) {
  const long long b = __double_as_longlong(y);
  const int be = (int)((b >> 52) & 0x7ff);
  if (!(y > 0.0) || y == 1.0 || be == 0 || be == 0x7ff) return cr_log_dev(y);   // 0, 1, subnormal, inf: general path
  const int j = (int)((b >> 42) & 0x3ff);
  const double m = __longlong_as_double((b & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
  const double inv = g_log_tab[j][0];
  const double Lh = g_log_tab[j][1], Ll = g_log_tab[j][2];
  const double e = (double)(be - 1023 + (j == 1023 ? 1 : 0));
  const double r = __fma_rn(m, inv, -1.0);
  const double r2 = __dmul_rn(r, r);
  double q = __dadd_rn(-1.0 / 6.0, __dmul_rn(r, 1.0 / 7.0));
  q = __dadd_rn(0.2, __dmul_rn(r, q));
  q = __dadd_rn(-0.25, __dmul_rn(r, q));
  q = __dadd_rn(1.0 / 3.0, __dmul_rn(r, q));
  q = __dadd_rn(-0.5, __dmul_rn(r, q));
  const double p = __dmul_rn(r2, q);
  const double LN2_HI = 0x1.62e42fefa3800p-1, LN2_LO = 0x1.ef35793c76730p-45;
  const double A = __dmul_rn(e, LN2_HI);   // exact: 42-bit constant, |e| < 2^11
  dd s = dd_two_sum(A, Lh);
  dd t = dd_two_sum(s.hi, r);
  const double lo = __dadd_rn(__dadd_rn(s.lo, t.lo), __dadd_rn(__dmul_rn(e, LN2_LO), __dadd_rn(Ll, p)));
  const dd v = dd_quick(t.hi, lo);
  const double eps = (e == 0.0 && Lh == 0.0) ? __dadd_rn(__dmul_rn(fabs(p), 0x1.0p-49), 0x1.0p-1070) : 0x1.0p-69;
  const double up = __dadd_rn(v.hi, __dadd_rn(v.lo, eps));
  const double dn = __dadd_rn(v.hi, __dsub_rn(v.lo, eps));
  if (up == dn) return up;
  return cr_log_dev(y);
}

// Out-of-line copy for the samplers (keeps their register count down).
__device__ __noinline__ static double cr_log_nl(double y) { return cr_log_fast(y); }

// Counts of the exact decisions' fallback stages, for tests (one copy per
// translation unit; read and reset through rp_debug_counters):
//   0 wedge tests past the FP32 margin, 1 of those past the libm margin;
//   2, 3 the same for normal tail pairs; 4, 5 for Marsaglia-Tsang tests.
// Each is bumped only on its rare path.
enum { DBG_WEDGE_FP64 = 0, DBG_WEDGE_CR, DBG_TAIL_FP64, DBG_TAIL_CR, DBG_MT_FP64, DBG_MT_CR, DBG_N = 8 };
static __device__ unsigned long long g_dbg[DBG_N];
__device__ __forceinline__ void dbg_count(int k) { atomicAdd(&g_dbg[k], 1ull); }

// Exact decision y < RN(exp(t)): CUDA exp (max error a few ulp) decides
// unless y lies within 2^-48 relative of it; then the correctly rounded value
// decides.
__device__ __forceinline__ bool lt_cr_exp(double y, double t) {
  double e = exp(t);
  double m = __dmul_rn(e, 0x1.0p-48);
  if (y < __dsub_rn(e, m)) return true;
  if (y > __dadd_rn(e, m)) return false;
  dbg_count(DBG_WEDGE_CR);
  return y < cr_exp_dev(t);
}

// ------------------------------------------------------------------ ziggurat tables
struct ZigDev {
  u64 k[256];
  u64 msh[256];     // significand of w_i shifted to bit 63
  double f[256];
  int we[256];      // w_i = (msh >> 11) 2^we
  int wtz[256];     // trailing zeros of the significand
  float ff[256];    // f_i, f_{i-1} - f_i and w_i rounded to float (estimates only)
  float fd[256];
  float wf[256];
  double w[256];    // w_i
  double R;
  float Rf;
  float pad;
};

// ------------------------------------------------------------------ engines
// GF(2) matrix-vector product with a nibble table: out = XOR over the 64
// four-bit chunks c of the input of tab[c][chunk value] (32-byte entries).
__device__ __forceinline__ void gf2_apply(const ulonglong4_32a* __restrict__ tab, u64& s0, u64& s1, u64& s2, u64& s3) {
  u64 a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  u64 in[4] = {s0, s1, s2, s3};
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    u64 x = in[w];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      int v = (int)((x >> (4 * q)) & 15u);
      const ulonglong2* e = (const ulonglong2*)(tab + ((w * 16 + q) * 16 + v));
      ulonglong2 t0 = __ldg(e), t1 = __ldg(e + 1);
      a0 ^= t0.x; a1 ^= t0.y; a2 ^= t1.x; a3 ^= t1.y;
    }
  }
  s0 = a0; s1 = a1; s2 = a2; s3 = a3;
}

// xoshiro256++ and xoshiro256** (Blackman & Vigna; Table "engines"): the
// scrambler's output of the current state, then the linear transition that
// both engines share, so they share the jump tables too.  kSS selects the
// "**" scrambler, rotl(5 s1, 7) 9, over "++", rotl(s0 + s3, 23) + s0.
// Jumps by precomputed GF(2) matrices T^(2^j).
template <bool kSS>
struct XoshiroT {
  u64 s0, s1, s2, s3;
  __device__ __forceinline__ u64 next() {
    u64 r = kSS ? rotl64(s1 * 5ull, 7) * 9ull : rotl64(s0 + s3, 23) + s0;
    u64 t = s1 << 17;
    s2 ^= s0; s3 ^= s1; s1 ^= s2; s0 ^= s3; s2 ^= t; s3 = rotl64(s3, 45);
    return r;
  }
  // Unrolled loops take kStep words per step (one: the chain through the
  // state is the critical path either way); kLeanCtas resident CTAs per SM
  // for the bitmap kernel.
  static constexpr int kStep = 1, kLeanCtas = 4;
  __device__ __forceinline__ void next_step(u64 (&u)[kStep]) { u[0] = next(); }
  __device__ void init(const EngineArgs& a, u64 off) {
    s0 = a.s[0]; s1 = a.s[1]; s2 = a.s[2]; s3 = a.s[3];
    const ulonglong4_32a* tab = (const ulonglong4_32a*)a.gf2_pow;
    while (off) {
      int j = __ffsll((long long)off) - 1;
      gf2_apply(tab + (size_t)j * 1024, s0, s1, s2, s3);
      off &= off - 1;
    }
  }
  __device__ __forceinline__ void advance(const EngineArgs& a) {
    gf2_apply((const ulonglong4_32a*)a.gf2_stride, s0, s1, s2, s3);
  }
  // State at word c T + t C (thread t of CTA c): warp 0 computes the CTA
  // base T^(c T) s with warp-cooperative GF(2) products (two nibble lookups
  // per lane and an XOR reduction), then every thread applies T^(t C).
  // `sh` is 4 words of shared memory.  Call with the whole CTA.
  __device__ void init_tile(const EngineArgs& a, unsigned c, int t, u64* sh) {
    if (t < 32) {
      u64 v[4] = {a.s[0], a.s[1], a.s[2], a.s[3]};
      const ulonglong4_32a* base = (const ulonglong4_32a*)a.gf2_cta;
      for (int j = 0; j < 16; ++j) {
        if (!((c >> j) & 1)) continue;
        const ulonglong4_32a* tab = base + (size_t)j * 1024;
        u64 acc[4] = {0, 0, 0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int ch = 2 * t + h;                       // nibble chunk 0..63
          int v4 = (int)((v[ch >> 4] >> (4 * (ch & 15))) & 15u);
          const ulonglong2* e = (const ulonglong2*)(tab + (ch * 16 + v4));
          ulonglong2 t0 = __ldg(e), t1 = __ldg(e + 1);
          acc[0] ^= t0.x; acc[1] ^= t0.y; acc[2] ^= t1.x; acc[3] ^= t1.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[w] ^= __shfl_xor_sync(0xffffffffu, acc[w], o);
#pragma unroll
        for (int w = 0; w < 4; ++w) v[w] = acc[w];
      }
      if (t == 0) { sh[0] = v[0]; sh[1] = v[1]; sh[2] = v[2]; sh[3] = v[3]; }
    }
    __syncthreads();
    s0 = sh[0]; s1 = sh[1]; s2 = sh[2]; s3 = sh[3];
    __syncthreads();
    if (t) gf2_apply((const ulonglong4_32a*)a.gf2_thread + (size_t)t * 1024, s0, s1, s2, s3);
  }
};
using XoshiroDev = XoshiroT<false>;
using XoshiroSSDev = XoshiroT<true>;

// PCG64-DXSM (O'Neill): DXSM output of the current state, then the LCG step
// with the 64-bit multiplier.  Jumps by affine powers (A, G): s <- A s + G inc.
struct PcgDev {
  u128 st, inc;
  __device__ __forceinline__ u64 next() {
    u64 hi = (u64)(st >> 64), lo = (u64)st | 1ull;
    hi ^= hi >> 32;
    hi *= 0xda942042e4dd58b5ull;
    hi ^= hi >> 48;
    hi *= lo;
    st = st * (u128)0xda942042e4dd58b5ull + inc;
    return hi;
  }
  static constexpr int kStep = 1, kLeanCtas = 5;
  __device__ __forceinline__ void next_step(u64 (&u)[kStep]) { u[0] = next(); }
  __device__ void init(const EngineArgs& a, u64 off) {
    st = ((u128)a.s[0] << 64) | a.s[1];
    inc = ((u128)a.s[2] << 64) | a.s[3];
    while (off) {
      int j = __ffsll((long long)off) - 1;
      const u64* p = a.pcg_pow + 4 * j;
      u128 A = ((u128)p[0] << 64) | p[1], G = ((u128)p[2] << 64) | p[3];
      st = A * st + G * inc;
      off &= off - 1;
    }
  }
  __device__ void init_tile(const EngineArgs& a, unsigned c, int t, u64*) { init(a, (u64)c * a.tile_words + (u64)t * a.chunk_words); }
  __device__ __forceinline__ void advance(const EngineArgs& a) {
    u128 A = ((u128)a.pcg_stride[0] << 64) | a.pcg_stride[1];
    u128 G = ((u128)a.pcg_stride[2] << 64) | a.pcg_stride[3];
    st = A * st + G * inc;
  }
};

// Philox4x32-10 (Salmon et al.): word i of the stream is half (i & 1) of
// block (counter + i/2); the block's 32-bit lanes x0..x3 give x0|x1<<32 and
// x2|x3<<32.
struct PhiloxDev {
  u64 c_lo, c_hi;
  unsigned k0, k1;
  u64 idx;         // next word index relative to the seeded counter
  u64 buf;
  __device__ __forceinline__ void block(u64 b, u64& w0, u64& w1) const {
    u128 c = (((u128)c_hi << 64) | c_lo) + (u128)b;
    unsigned x0 = (unsigned)c, x1 = (unsigned)(c >> 32), x2 = (unsigned)(c >> 64), x3 = (unsigned)(c >> 96);
    unsigned ka = k0, kb = k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      unsigned h0 = __umulhi(0xD2511F53u, x0), l0 = 0xD2511F53u * x0;
      unsigned h1 = __umulhi(0xCD9E8D57u, x2), l1 = 0xCD9E8D57u * x2;
      unsigned y0 = h1 ^ x1 ^ ka, y2 = h0 ^ x3 ^ kb;
      x0 = y0; x1 = l1; x2 = y2; x3 = l0;
      ka += 0x9E3779B9u; kb += 0xBB67AE85u;
    }
    w0 = (u64)x0 | ((u64)x1 << 32);
    w1 = (u64)x2 | ((u64)x3 << 32);
  }
  __device__ __forceinline__ u64 next() {
    u64 r;
    if ((idx & 1) == 0) {
      u64 w0, w1;
      block(idx >> 1, w0, w1);
      buf = w1;
      r = w0;
    } else {
      r = buf;
    }
    ++idx;
    return r;
  }
  // Unrolled loops take two consecutive words per step, one block and no
  // branch: the parity of idx is the same for every thread of a fill but
  // unknown at compile time.  Odd phase: the pending word and the low half
  // of the next block, whose high half becomes pending.
  static constexpr int kStep = 2, kLeanCtas = 5;
  __device__ __forceinline__ void next_step(u64 (&u)[kStep]) {
    const bool odd = (idx & 1) != 0;
    u64 w0, w1;
    block((idx + 1) >> 1, w0, w1);
    u[0] = odd ? buf : w0;
    u[1] = odd ? w0 : w1;
    buf = w1;
    idx += 2;
  }
  __device__ void init(const EngineArgs& a, u64 off) {
    c_lo = a.s[0]; c_hi = a.s[1];
    k0 = (unsigned)a.s[2]; k1 = (unsigned)(a.s[2] >> 32);
    idx = a.word0 + off;
    if (idx & 1) {  // starting on the odd half: fetch it
      u64 w0;
      block(idx >> 1, w0, buf);
    }
  }
  __device__ void init_tile(const EngineArgs& a, unsigned c, int t, u64*) { init(a, (u64)c * a.tile_words + (u64)t * a.chunk_words); }
  __device__ __forceinline__ void advance(const EngineArgs& a) {
    u64 start = idx;  // callers advance a saved chunk-start copy
    idx = start + a.stride;
    if (idx & 1) { u64 w0; block(idx >> 1, w0, buf); }
  }
};

// Philox4x64-10 (Salmon, Moraes, Dror & Shaw 2011; the paper's Philox): ten
// rounds of two 64 x 64 -> 128 products with a Weyl key schedule; word p is
// word p mod 4 of the block at counter + 1 + p / 4 (the counter is
// incremented before each block).  State: 128-bit counter (c_lo, c_hi), key
// (k0, k1).  The unrolled loops take four words per step, one block: the
// word index's phase within a block is the same for every thread of a fill
// but unknown at compile time, so the held block and the new one are
// combined by selects.
struct Philox64Dev {
  u64 c_lo, c_hi, k0, k1;
  u64 idx;              // next word index relative to the seeded counter
  u64 b0, b1, b2, b3;   // the block that holds word idx - 1 (when idx % 4 != 0)
  __device__ __forceinline__ void block(u64 b, u64& w0, u64& w1, u64& w2, u64& w3) const {
    const u128 c = (((u128)c_hi << 64) | c_lo) + (u128)b + 1u;
    u64 x0 = (u64)c, x1 = (u64)(c >> 64), x2 = 0, x3 = 0;
    u64 ka = k0, kb = k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      const u64 h0 = __umul64hi(0xD2E7470EE14C6C93ull, x0), l0 = 0xD2E7470EE14C6C93ull * x0;
      const u64 h1 = __umul64hi(0xCA5A826395121157ull, x2), l1 = 0xCA5A826395121157ull * x2;
      const u64 y0 = h1 ^ x1 ^ ka, y2 = h0 ^ x3 ^ kb;
      x0 = y0; x1 = l1; x2 = y2; x3 = l0;
      ka += 0x9E3779B97F4A7C15ull; kb += 0xBB67AE8584CAA73Bull;
    }
    w0 = x0; w1 = x1; w2 = x2; w3 = x3;
  }
  __device__ __forceinline__ u64 next() {
    const int q = (int)(idx & 3);
    if (q == 0) block(idx >> 2, b0, b1, b2, b3);
    const u64 r = q == 0 ? b0 : q == 1 ? b1 : q == 2 ? b2 : b3;
    ++idx;
    return r;
  }
  static constexpr int kStep = 4, kLeanCtas = 5;
  __device__ __forceinline__ void next_step(u64 (&u)[kStep]) {
    const int q = (int)(idx & 3);
    u64 n0, n1, n2, n3;
    block((idx + 3) >> 2, n0, n1, n2, n3);   // phase 0: this block; else the next one
    // words idx .. idx + 3: positions q .. 3 of the held block, then 0 .. q - 1 of the new one
    u[0] = q == 0 ? n0 : q == 1 ? b1 : q == 2 ? b2 : b3;
    u[1] = q == 0 ? n1 : q == 1 ? b2 : q == 2 ? b3 : n0;
    u[2] = q == 0 ? n2 : q == 1 ? b3 : q == 2 ? n0 : n1;
    u[3] = q == 0 ? n3 : q == 1 ? n0 : q == 2 ? n1 : n2;
    b0 = n0; b1 = n1; b2 = n2; b3 = n3;
    idx += 4;
  }
  __device__ void init(const EngineArgs& a, u64 off) {
    c_lo = a.s[0]; c_hi = a.s[1];
    k0 = a.s[2]; k1 = a.s[3];
    idx = a.word0 + off;
    if (idx & 3) block(idx >> 2, b0, b1, b2, b3);
  }
  __device__ void init_tile(const EngineArgs& a, unsigned c, int t, u64*) { init(a, (u64)c * a.tile_words + (u64)t * a.chunk_words); }
  __device__ __forceinline__ void advance(const EngineArgs& a) {
    idx += a.stride;   // callers advance a saved chunk-start copy
    if (idx & 3) block(idx >> 2, b0, b1, b2, b3);
  }
};

}  // namespace rp
