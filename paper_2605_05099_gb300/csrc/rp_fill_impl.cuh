// Fill kernels of librp (sm_103a), included once per engine translation unit.
//
// A stream is cut into tiles of T = NT*C consecutive words.  Persistent CTAs
// take tiles round-robin (tile k by CTA k mod grid); thread t of a tile owns
// chunk t (C consecutive words) and reaches its chunk in the next tile by one
// constant jump of its engine state, so each thread generates long runs of
// its stream with one jump per C words.
//
// One word per variate (raw words, uniforms, and bounded integers when
// rejections are rare): the output index of a word is known, so every thread
// streams its chunk out through a per-warp staging buffer that turns the
// chunk-contiguous runs into coalesced 128-byte lines.  Bounded integers with
// frequent rejections take one pass with parked runs (rp_rej.cuh).
//
// Rejection samplers: each thread walks the serial sampler's chain of
// candidates over its chunk.  The parallel parse (chains across chunk seams)
// uses sync points for samplers whose candidate length follows from its
// first word (ziggurat normal/exponential, and bounded integers in batches;
// rp_lean.cuh):
//   * len(q) is the number of words a candidate starting at word q would
//     consume (evaluated speculatively for any q);
//   * the sync point of a chunk is the first s in [G, G+S) (relative to the
//     chunk) such that every candidate starting in [0, s) ends by s.  The
//     true chain, which enters the chunk from the previous one, then passes
//     through s unless a candidate longer than G straddles the seam;
//   * thread t walks from its sync point to the next chunk's sync point,
//     which it evaluates itself from the same words with the same rule, and
//     checks that the chain lands on it (E_LANDING otherwise).
// Gamma and beta attempts have no such points; their seams are merge points
// (k_merge below).  Pass 1 counts the outputs of each segment; a block scan
// and a decoupled look-back over tile counts give every thread its first
// output index; pass 2 regenerates the chunk and writes the values through
// the staging buffer.  Outputs whose value needs FP64 libm (ziggurat tails,
// ~3e-4 of outputs) are queued and evaluated by full warps in a second
// kernel.  Derived distributions transform each value as it is written
// (epi_apply below).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "rp_device.cuh"
#include "rp_internal.h"

namespace rp {

// Each translation unit that includes this file owns its copy of the tables
// (no relocatable device code); upload_zig_tu() fills it.
static __device__ ZigDev g_zig[2];

namespace {

constexpr u64 M52 = (1ull << 52) - 1;
constexpr u64 M53 = (1ull << 53) - 1;
constexpr unsigned long long kSpinMax = 1ull << 25;   // bounded waits (x ~100 ns)
constexpr int kStage = 16;                            // outputs staged per lane
constexpr int kRow = kStage + 1;                      // padded row stride (no bank conflicts)
constexpr int kTailPairsMax = 64;                     // speculative tail length cap

__device__ __forceinline__ void set_err(Ctrl* c, unsigned e, unsigned long long info) {
  atomicOr(&c->err, e);
  atomicExch(&c->err_info, info);
}
__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *(volatile const unsigned long long*)p;
}

// ------------------------------------------------------------------ exact decisions
// The FP64 pipe of this GPU is ~70x slower than the FP32 pipe, so each accept
// test is first decided in FP32 with a proven error margin; near-ties fall
// through to the exact FP64 test with the correctly rounded exp/log.

// y < RN(exp(t)) for the wedge of strip i: y = f_i + U (f_{i-1} - f_i),
// t = -x^2/2 (normal) or -x (exponential).  FP32 pass: x_f relative 2^-22,
// y_f relative 2^-21.7, expf 2 ulp -> exp(t) estimate within
// 2^-20.8 (|t| + 1.2); the margin 2^-19 (1 + |t|) is 3.5x that.
template <bool kNormal>
__device__ __forceinline__ bool wedge_accept(u64 r, int i, u64 u2, const ZigDev& z) {
  float xf = int_scaled_f(r, 0) * z.wf[i];
  float tf = kNormal ? -0.5f * xf * xf : -xf;
  float ef = expf(tf);
  float yf = fmaf(u53_f(u2), z.fd[i], z.ff[i]);
  float m = 0x1.0p-19f * (1.0f - tf);
  if (yf < ef * (1.0f - m)) return true;
  if (yf > ef * (1.0f + m)) return false;
  dbg_count(DBG_WEDGE_FP64);
  double x = mul_rn_int(r, z.msh[i], z.wtz[i], z.we[i]);
  double y = __dadd_rn(__dmul_rn(__dsub_rn(z.f[i - 1], z.f[i]), u53_bits(u2)), z.f[i]);
  double t = kNormal ? __dmul_rn(-0.5, __dmul_rn(x, x)) : -x;
  return lt_cr_exp(y, t);
}

// One pair of the normal tail (Marsaglia 1964): a = -log(1-U1)/R,
// b = -log(1-U2), accept when 2b > a^2 (a, b from correctly rounded logs).
// FP32 pass: logs within 2^-20 relative, so a^2 within 2^-18.7.
__device__ __forceinline__ bool tail_pair_accept(u64 w1, u64 w2, const ZigDev& z) {
  float af = -log1m_u53_f(w1) / z.Rf;
  float bf = -log1m_u53_f(w2);
  float lhs = bf + bf, rhs = af * af;
  float m = (lhs + rhs) * 0x1.0p-16f;
  if (lhs > rhs + m) return true;
  if (lhs < rhs - m) return false;
  dbg_count(DBG_TAIL_FP64);
  // libm logs (one ulp) decide unless the sides are within their effect
  double o1 = __dsub_rn(1.0, u53_bits(w1)), o2 = __dsub_rn(1.0, u53_bits(w2));
  double a = __ddiv_rn(-log(o1), z.R), b = -log(o2);
  double l2 = __dadd_rn(b, b), r2 = __dmul_rn(a, a);
  double mg = (l2 + r2) * 0x1.0p-48;
  if (l2 > r2 + mg) return true;
  if (l2 < r2 - mg) return false;
  dbg_count(DBG_TAIL_CR);
  a = __ddiv_rn(-cr_log_nl(o1), z.R);
  b = -cr_log_nl(o2);
  return __dadd_rn(b, b) > __dmul_rn(a, a);
}

// W consecutive words from the engine, in steps of its width (W a multiple).
template <class E, int W>
__device__ __forceinline__ void take_words(E& g, u64 (&u)[W]) {
  static_assert(W % E::kStep == 0, "whole engine steps");
#pragma unroll
  for (int i = 0; i < W; i += E::kStep) {
    u64 t[E::kStep];
    g.next_step(t);
#pragma unroll
    for (int k = 0; k < E::kStep; ++k) u[i + k] = t[k];
  }
}

// ------------------------------------------------------------------ derived distributions
// Output transform of a base variate x (Table "continuous"; Sec. 3.1 "Gamma
// and related", "Extreme value and Weibull"): one IEEE operation per step,
// in the order of the formula.  exp and pow are CUDA's (one and two ulp);
// Gumbel's logs are the library's correctly rounded ones.  Out of line: it
// runs once per output of a derived fill and stays out of the base fills.
__device__ __noinline__ double epi_apply(double x, const SampArgs& a) {
  const double* p = a.ep;
  switch (a.epi) {
    case EPI_AFFINE: return __dadd_rn(p[0], __dmul_rn(p[1], x));
    case EPI_SCALE: return __dmul_rn(p[0], x);
    case EPI_LOGNORMAL: return exp(__dadd_rn(p[0], __dmul_rn(p[1], x)));
    case EPI_GUMBEL: return __dsub_rn(p[0], __dmul_rn(p[1], cr_log_nl(-cr_log_nl(x))));
    case EPI_PARETO: return __dmul_rn(p[0], exp(__ddiv_rn(x, p[1])));
    case EPI_WEIBULL: return __dmul_rn(p[1], pow(x, p[0]));
    case EPI_GPD: {
      if (p[2] == 0.0) return __dadd_rn(p[0], __dmul_rn(p[1], x));
      const double P = exp(__ddiv_rn(x, p[3]));   // Pareto(1, 1/|xi|) = exp(E / (1/|xi|))
      if (p[2] > 0.0) return __dadd_rn(p[0], __ddiv_rn(__dmul_rn(p[1], __dsub_rn(P, 1.0)), p[2]));
      return __dsub_rn(p[0], __ddiv_rn(__dmul_rn(p[1], __dsub_rn(1.0, __ddiv_rn(1.0, P))), p[2]));
    }
    default: return x;
  }
}

// Shift and scale inline; the transcendental transforms out of line.
__device__ __forceinline__ double epi_value(double x, const SampArgs& a) {
  if (a.epi == EPI_AFFINE) return __dadd_rn(a.ep[0], __dmul_rn(a.ep[1], x));
  if (a.epi == EPI_SCALE) return __dmul_rn(a.ep[0], x);
  return epi_apply(x, a);
}

#include "rp_gamma.cuh"

// ------------------------------------------------------------------ samplers
// One word per variate: raw words and 53-bit uniforms.
struct SampU64 {
  static constexpr bool kOnePerWord = true;
  static constexpr bool kCheckReject = false;
  typedef u64 out_t;
  __device__ static __forceinline__ u64 value1(u64 u, const SampArgs&) { return u; }
};
struct SampUniform {
  static constexpr bool kOnePerWord = true;
  static constexpr bool kCheckReject = false;
  typedef double out_t;
  __device__ static __forceinline__ double value1(u64 u, const SampArgs&) { return u53_bits(u); }
};
// 52-bit uniform, the paper's default (Sec. 3.1, method 2): the word's top
// 52 bits as the fraction of a double in [1, 2), minus 1 (exact).
// floor(u / 2^12) 2^-52 is exact and is assembled with integer operations,
// as u53_bits does (no FP64 instruction).
struct SampUniform52 {
  static constexpr bool kOnePerWord = true;
  static constexpr bool kCheckReject = false;
  typedef double out_t;
  __device__ static __forceinline__ double value1(u64 u, const SampArgs&) {
    const u64 v = u >> 12;
    if (v == 0) return 0.0;
    const int lz = __clzll(v);                  // >= 12
    const u64 mt = v << (lz - 11);              // in [2^52, 2^53)
    return __longlong_as_double((long long)((((u64)(1033 - lz)) << 52) + mt));
  }
};
// Uniform base of a derived distribution (unif, Gumbel).
struct SampUniformE {
  static constexpr bool kOnePerWord = true;
  static constexpr bool kCheckReject = false;
  typedef double out_t;
  __device__ static __forceinline__ double value1(u64 u, const SampArgs& a) { return epi_value(u53_bits(u), a); }
};

// Lemire with no rejection assumed: word p gives output p, hi(u m); every
// word whose low product falls below 2^64 mod m is reported, and the host
// keeps the outputs before the first such word (exact: the serial sampler
// produces the same values up to its first rejection).
struct SampBoundedOne {
  static constexpr bool kOnePerWord = true;
  static constexpr bool kCheckReject = true;
  typedef u64 out_t;
  __device__ static __forceinline__ u64 value1(u64 u, const SampArgs& a) { return __umul64hi(u, a.m); }
  // hi(u m) and, in lo, the low 64 bits that decide the rejection
  __device__ static __forceinline__ u64 value_lo(u64 u, const SampArgs& a, u64& lo) {
    lo = u * a.m;
    return __umul64hi(u, a.m);
  }
};
// The same for m < 2^32: u m from two 32 x 32 -> 64 products (u = uh 2^32 +
// ul: u m = uh m 2^32 + ul m), instead of a full 64 x 64 -> 128 product.
struct SampBoundedOne32 {
  static constexpr bool kOnePerWord = true;
  static constexpr bool kCheckReject = true;
  typedef u64 out_t;
  __device__ static __forceinline__ u64 value_lo(u64 u, const SampArgs& a, u64& lo) {
    const unsigned m = (unsigned)a.m;
    const u64 pl = (u64)(unsigned)u * m, ph = (u64)(unsigned)(u >> 32) * m;
    const u64 mid = (pl >> 32) + (unsigned)ph;   // < 2^33
    lo = (mid << 32) | (unsigned)pl;
    return (ph >> 32) + (mid >> 32);
  }
  __device__ static __forceinline__ u64 value1(u64 u, const SampArgs& a) { u64 lo; return value_lo(u, a, lo); }
};

// ------------------------------------------------------------------ float variants
// Table "continuous" (suffix f), Sec. 3.1 and Sec. 4.4: the engines' bit
// stream read as 32-bit words.  Each 64-bit word gives its low half, then its
// high half; a float fill starts at the low half of word *pos, and a fill
// that ends on a low half leaves the high half unused.

// u24(h) = floor(h / 2^8) 2^-24, exact in float and double.
__device__ __forceinline__ double u24d(u64 h) { return (double)((unsigned)h >> 8) * 0x1.0p-24; }

// A word engine read as half-words, each returned in the low 32 bits.  The
// launch geometry in EngineArgs is in words (chunks and tiles of an even
// number of half-words start on whole words).
template <class E>
struct HalfWords {
  E e;
  u64 hi;
  int have;   // the high half of the last word is next
  static constexpr int kStep = 2 * E::kStep, kLeanCtas = E::kLeanCtas;
  __device__ void init_tile(const EngineArgs& a, unsigned c, int t, u64* sh) {
    e.init_tile(a, c, t, sh);
    have = 0;
  }
  __device__ __forceinline__ void advance(const EngineArgs& a) {
    e.advance(a);
    have = 0;
  }
  __device__ __forceinline__ u64 next() {
    if (have) {
      have = 0;
      return hi;
    }
    const u64 w = e.next();
    hi = w >> 32;
    have = 1;
    return w & 0xffffffffull;
  }
  __device__ __forceinline__ void next_step(u64 (&u)[kStep]) {
    if (have) {   // not on a word boundary (the kernels step from chunk starts: never)
#pragma unroll
      for (int i = 0; i < kStep; ++i) u[i] = next();
      return;
    }
    u64 w[E::kStep];
    e.next_step(w);
#pragma unroll
    for (int i = 0; i < E::kStep; ++i) {
      u[2 * i] = w[i] & 0xffffffffull;
      u[2 * i + 1] = w[i] >> 32;
    }
  }
};

// uniformf, the paper's default method in float: the top 23 bits of the
// half-word as the fraction of a float in [1, 2), minus 1, which is exactly
// floor(h / 2^9) 2^-23.  Both halves of a word at once, as the 8 bytes of two
// consecutive floats (low half first).
__device__ __forceinline__ unsigned uniformf_bits(unsigned h) {
  const unsigned v = h >> 9;
  if (v == 0) return 0u;
  const int lz = __clz(v);                          // >= 9
  return ((unsigned)(135 - lz) << 23) + ((v << (lz - 8)) & 0x7fffffu);
}
struct SampUniformF2 {
  static constexpr bool kOnePerWord = true;
  static constexpr bool kCheckReject = false;
  typedef u64 out_t;
  __device__ static __forceinline__ u64 value1(u64 u, const SampArgs&) {
    return (u64)uniformf_bits((unsigned)u) | ((u64)uniformf_bits((unsigned)(u >> 32)) << 32);
  }
};

// Float ziggurat tail values from the queued half-words, computed in double
// with the correctly rounded log and rounded once to float (the reading of
// the float tails).
struct SampNormalF {
  typedef float out_t;
  __device__ static double tail_value(u64 u0, u64 w1, const ZigDev& z) {
    const double a = __ddiv_rn(-cr_log_nl(__dsub_rn(1.0, u24d(w1))), z.R);
    const float v = __double2float_rn(__dadd_rn(z.R, a));
    return ((u0 >> 8) & 1) ? -(double)v : (double)v;
  }
};
struct SampExpF {
  typedef float out_t;
  __device__ static double tail_value(u64, u64 w1, const ZigDev& z) {
    return (double)__double2float_rn(__dsub_rn(z.R, cr_log_nl(__dsub_rn(1.0, u24d(w1)))));
  }
};

// Values of ziggurat tail outputs (FP64 libm log, within 2 ulp of the
// correctly rounded value), evaluated by k_tails from the queued words.
struct SampNormal {
  typedef double out_t;
  // +-(R + a), a = -log(1-U1)/R of the accepted pair; sign from the candidate word
  __device__ static double tail_value(u64 u0, u64 w1, const ZigDev& z) {
    double a = __ddiv_rn(-log(__dsub_rn(1.0, u53_bits(w1))), z.R);
    return neg_if(__dadd_rn(z.R, a), (u0 >> 8) & 1);
  }
};
struct SampExp {
  typedef double out_t;
  // R - log(1 - U)
  __device__ static double tail_value(u64, u64 w1, const ZigDev& z) {
    return __dsub_rn(z.R, log(__dsub_rn(1.0, u53_bits(w1))));
  }
};

// ------------------------------------------------------------------ scans
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < NT / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NT / 32) warp_sums[lane] = s;  // inclusive
    if (lane == NT / 32 - 1) *total = s;
  }
  __syncthreads();
  int before = wid ? warp_sums[wid - 1] : 0;
  return before + x - v;
}

// Decoupled look-back over tile counts, run by one warp.  Status word:
// bit 63 aggregate, bit 62 inclusive, low 62 bits value.  Each round the warp
// inspects the next 32 x kW predecessors, nearest first (lane l, window w:
// tile j - l - 32 w), and consumes them up to the nearest inclusive value once
// every entry before it is at least an aggregate.  `kp` is the CTA's own
// previous tile (-1: none), whose inclusive prefix `incp` the CTA already
// knows: the walk never goes past it, so a look-back spans at most one grid
// of predecessors even when a whole round of tiles finishes together.
// Returns the tile's exclusive prefix in all lanes, or ~0 if the bounded wait
// ran out or the tile became unnecessary.  spin_max (0: kSpinMax) bounds the
// wait; stall_tile1 - 1 names a tile that publishes nothing (test hooks).
__device__ unsigned long long lookback_warp(unsigned long long* st, unsigned long long k, unsigned long long cnt,
                                           Ctrl* ctrl, long long kp = -1, unsigned long long incp = 0,
                                           unsigned long long spin_max = 0, unsigned long long stall_tile1 = 0) {
  constexpr int kW = 1;
  if (stall_tile1 && k + 1 == stall_tile1) return ~0ull;   // test hook: this tile never publishes
  const unsigned long long smax = spin_max ? spin_max : kSpinMax;
  const unsigned long long AGG = 1ull << 63, INC = 1ull << 62, VAL = INC - 1;
  const int lane = threadIdx.x & 31;
  if (k == 0) {
    if (lane == 0) *(volatile unsigned long long*)(st) = INC | cnt;
    return 0;
  }
  if (lane == 0) *(volatile unsigned long long*)(st + k) = AGG | cnt;
  unsigned long long excl = 0;
  long long j = (long long)k - 1;
  unsigned long long spins = 0;
  for (;;) {
    unsigned long long v[kW];
    unsigned incm[kW], rdym[kW];
#pragma unroll
    for (int w = 0; w < kW; ++w) {
      const long long idx = j - lane - 32 * w;
      // at or below the CTA's previous tile: its known inclusive value (or
      // zero before the first tile), never a load
      v[w] = idx > kp ? ld_volatile(st + idx) : (INC | (idx == kp ? incp : 0ull));
      incm[w] = __ballot_sync(0xffffffffu, (v[w] & INC) != 0);
      rdym[w] = __ballot_sync(0xffffffffu, (v[w] & (INC | AGG)) != 0);
    }
    int wi = kW, fi = 31;   // window and lane of the nearest inclusive value
#pragma unroll
    for (int w = kW - 1; w >= 0; --w)
      if (incm[w]) { wi = w; fi = __ffs(incm[w]) - 1; }
    bool ready = true;
#pragma unroll
    for (int w = 0; w < kW; ++w) {
      const unsigned need = w < wi ? 0xffffffffu : (w == wi ? (2u << fi) - 1u : 0u);
      ready = ready && (rdym[w] & need) == need;
    }
    if (!ready) {
      int stop = 0;
      if (lane == 0) {
        if (ld_volatile(&ctrl->done_tile) < k) stop = 1;
        else if (++spins > smax) { set_err(ctrl, E_TIMEOUT, k); stop = 1; }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return ~0ull;
      __nanosleep(64);
      continue;
    }
    unsigned long long c = 0;
#pragma unroll
    for (int w = 0; w < kW; ++w)
      if (w < wi || (w == wi && lane <= fi)) c += v[w] & VAL;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    excl += c;
    if (wi < kW) break;
    j -= 32 * kW;
  }
  if (lane == 0) *(volatile unsigned long long*)(st + k) = INC | (excl + cnt);
  return excl;
}

// The CTA's previous tile and its inclusive prefix, kept by the look-back
// warp across the tiles of a persistent CTA (k = -1: none yet).
struct LookbackFloor {
  long long k = -1;
  unsigned long long inc = 0;
};

// ------------------------------------------------------------------ staging
// Lane rows of kStage outputs, flushed by the warp so that each row (a run of
// consecutive outputs) is written by whole groups of lanes.  In the one-word
// fills every word is an output, so row r's place is fixed, dst0 + r stride,
// and needs no shuffle.  Rows are kRowW words apart: 16-byte aligned, and
// 16-byte accesses by eight lanes of a row or of eight rows hit distinct banks.
constexpr int kRowW = kStage + 2;

__device__ __forceinline__ u64 as_bits(u64 v) { return v; }
__device__ __forceinline__ u64 as_bits(double v) { return (u64)__double_as_longlong(v); }

// 8-byte stores, two rows per instruction (any output alignment).
__device__ __forceinline__ void flush_rows(u64* __restrict__ out, const u64* rows, u64 dst0, int stride, u64 n) {
  const int lane = threadIdx.x & 31;
  const int half = lane >> 4, col = lane & 15;
#pragma unroll 4
  for (int r = 0; r < 32; r += 2) {
    const int rr = r + half;
    const u64 d = dst0 + (u64)(rr * stride + col);
    if (d < n) out[d] = rows[rr * kRowW + col];
  }
}

// 16-byte stores, four rows per instruction (output 16-byte aligned; dst0
// and stride even).
__device__ __forceinline__ void flush_rows_wide(u64* __restrict__ out, const u64* rows, u64 dst0, int stride, u64 n) {
  const int lane = threadIdx.x & 31;
  const int q = lane >> 3, c2 = (lane & 7) * 2;
#pragma unroll 4
  for (int r = 0; r < 32; r += 4) {
    const int rr = r + q;
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(rows + rr * kRowW + c2);
    const u64 d = dst0 + (u64)(rr * stride + c2);
    if (d + 1 < n) *reinterpret_cast<ulonglong2*>(out + d) = v;
    else if (d < n) out[d] = v.x;
  }
}

// ------------------------------------------------------------------ batches
static_assert(sizeof(FillArgs) % 8 == 0, "request arguments are copied as words");

// Claims the CTA's next work item and copies its request's arguments into
// shared memory.  Returns false once the list is exhausted.  All threads of
// the CTA call it; it synchronises the CTA.
__device__ __forceinline__ bool batch_claim(const BatchArgs& b, FillArgs& fa, BatchItem& bi,
                                            unsigned long long* slot) {
  if (threadIdx.x == 0) *slot = atomicAdd(b.next_item, 1ull);
  __syncthreads();
  const unsigned long long it = *slot;
  if (it >= b.n_items) return false;
  bi = b.items[it];
  const u64* src = (const u64*)&b.reqs[bi.req];
  u64* dst = (u64*)&fa;
  for (int i = threadIdx.x; i < (int)(sizeof(FillArgs) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  return true;
}

#include "rp_lean.cuh"
#include "rp_rej.cuh"

// ------------------------------------------------------------------ kernels
// One tile of a one-word-per-variate fill: chunk words stream straight to
// the output through the warp's staging rows.
template <int NT, class E, class S>
__device__ __forceinline__ void onepw_tile(const FillArgs& a, u64 k, const E& e, u64* stage_w, const int C) {
  static_assert(kStage % 2 == 0, "rows are written in pairs of words");
  const u64 T = (u64)NT * C;
  const int t = threadIdx.x, lane = t & 31;
  u64* out = (u64*)a.out;
  const bool wide = ((unsigned long long)a.out & 15) == 0;
  E g = e;
  const u64 base = k * (u64)T + (u64)t * C;
  const u64 wbase = k * (u64)T + (u64)(t - lane) * C;   // lane 0's chunk: row r goes to wbase + r C
  u64* row = stage_w + lane * kRowW;
  for (int j0 = 0; j0 < C; j0 += kStage) {
    constexpr int W = E::kStep > 2 ? E::kStep : 2;   // words per step, in pairs
#pragma unroll
    for (int j = 0; j < kStage; j += W) {
      u64 u[W];
      take_words<E, W>(g, u);
#pragma unroll
      for (int i = 0; i < W; i += 2) {
        if constexpr (S::kCheckReject) {
          u64 lo[2], v[2];
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            v[k] = S::value_lo(u[i + k], a.sp, lo[k]);
            const u64 p = base + j0 + j + i + k;
            if (lo[k] < a.sp.thresh && p < a.n) atomicMin(&a.ctrl->first_reject, p);
          }
          *reinterpret_cast<ulonglong2*>(row + j + i) = make_ulonglong2(v[0], v[1]);
        } else {
          *reinterpret_cast<ulonglong2*>(row + j + i) =
              make_ulonglong2(as_bits(S::value1(u[i], a.sp)), as_bits(S::value1(u[i + 1], a.sp)));
        }
      }
    }
    __syncwarp();
    if (wide) flush_rows_wide(out, stage_w, wbase + j0, C, a.n);
    else flush_rows(out, stage_w, wbase + j0, C, a.n);
    __syncwarp();
  }
}

// One tile per CTA: the host sizes the chunk (a multiple of kStage, in
// a.eng.chunk_words) so that the grid covers the fill, and every thread
// streams one contiguous range of the stream after a single jump.
template <int NT, class E, class S>
__global__ void __launch_bounds__(NT) k_onepw(FillArgs a) {
  __shared__ __align__(16) u64 stage[NT / 32][32 * kRowW];
  __shared__ u64 sh4[4];
  const int t = threadIdx.x, wid = t >> 5;
  E e;
  e.init_tile(a.eng, blockIdx.x, t, sh4);
  onepw_tile<NT, E, S>(a, blockIdx.x, e, stage[wid], (int)a.eng.chunk_words);
}

// One-word fill for Philox4x32-10, whose word p is half of the block at
// counter + p / 2: no thread has to walk a range of its own, so consecutive
// threads take consecutive blocks (grid-stride) and store their two outputs
// straight to the output, 16 bytes per lane, with no staging.  Output i is
// word w0 + i (w0 = the launch's first word), and every block's first output
// index has the parity of w0, so whether the pairs are 16-byte aligned is
// the same for the whole launch.
template <int NT, class S>
__global__ void __launch_bounds__(NT) k_onepw_ctr(FillArgs a) {
  PhiloxDev e;
  e.c_lo = a.eng.s[0];
  e.c_hi = a.eng.s[1];
  e.k0 = (unsigned)a.eng.s[2];
  e.k1 = (unsigned)(a.eng.s[2] >> 32);
  const u64 w0 = a.eng.word0, n = a.n;
  if (n == 0) return;
  u64* out = (u64*)a.out;
  const u64 b_first = w0 >> 1;
  const u64 nb = ((w0 + n - 1) >> 1) - b_first + 1;
  const bool pairs = ((((unsigned long long)out >> 3) + w0) & 1) == 0;
  const u64 G = (u64)gridDim.x * NT;
  for (u64 j = (u64)blockIdx.x * NT + threadIdx.x; j < nb; j += G) {
    u64 u[2];
    e.block(b_first + j, u[0], u[1]);
    const long long p0 = (long long)(2 * (b_first + j) - w0);   // -1 only for the first block of an odd w0
    u64 v[2];
    if constexpr (S::kCheckReject) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        u64 lo;
        v[h] = S::value_lo(u[h], a.sp, lo);
        const long long p = p0 + h;
        if (lo < a.sp.thresh && p >= 0 && (u64)p < n) atomicMin(&a.ctrl->first_reject, (u64)p);
      }
    } else {
      v[0] = as_bits(S::value1(u[0], a.sp));
      v[1] = as_bits(S::value1(u[1], a.sp));
    }
    if (pairs && p0 >= 0 && (u64)p0 + 1 < n) {
      *reinterpret_cast<ulonglong2*>(out + p0) = make_ulonglong2(v[0], v[1]);
    } else {
      if (p0 >= 0 && (u64)p0 < n) out[p0] = v[0];
      if ((u64)(p0 + 1) < n) out[p0 + 1] = v[1];
    }
  }
}

// Engine alone: the xor of the launch's n words, one contiguous range per
// thread as in k_onepw, folded per warp into *a.out (zeroed by the host).
// Nothing else is computed or stored, so its words/s is the engine's
// throughput ceiling for the fills.
template <int NT, class E>
__global__ void __launch_bounds__(NT) k_fold(FillArgs a) {
  __shared__ u64 sh4[4];
  E e;
  e.init_tile(a.eng, blockIdx.x, threadIdx.x, sh4);
  const int C = (int)a.eng.chunk_words;   // a multiple of 16
  const u64 base = (u64)blockIdx.x * NT * C + (u64)threadIdx.x * C;
  u64 f = 0;
  E g = e;
  for (int j0 = 0; j0 < C; j0 += 16) {
    u64 u[16];
    take_words<E, 16>(g, u);
    if (base + j0 + 16 <= a.n) {
#pragma unroll
      for (int i = 0; i < 16; ++i) f ^= u[i];
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) f ^= base + j0 + i < a.n ? u[i] : 0ull;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f ^= __shfl_xor_sync(0xffffffffu, f, o);
  if ((threadIdx.x & 31) == 0) atomicXor((unsigned long long*)a.out, f);
}

// ------------------------------------------------------------------ merge seams
// Gamma and beta attempts are at least two words long, so one-word sync
// points do not exist.  Instead the seam of a chunk is a merge point: run
// the sampler from each of the kE possible entry offsets 0..kE-1 in lockstep;
// chains that are at a variate boundary after the same word are identical
// from there on; the merge point is the first boundary (at or after kE - 1)
// where all of them have coalesced.  The true chain, entering the chunk with
// an overhang below kE, passes through it.  The search is bounded by the
// chunk length, which keeps merge points monotone across chunks; a chunk
// whose chains do not coalesce within it has no merge point, its thread has
// no segment and the previous thread's walk continues to the next chunk's
// merge point (same rule, same words, so both threads agree).
constexpr int kE = 12;
constexpr int kSkipMax = 64;  // chunks a walk may cross to find a merge point
constexpr int kRecW = 8;     // record words per staged variate (7 used + tail flag)
constexpr int kRecS = 4;     // staged records per lane

// Merge point of the chunk starting at the engine's position, searched over
// at most `limit` words.  `own` (nullable) is fed the same words.  Returns the
// boundary (relative), -1 if none within the limit, -2 if `own` is not at a
// boundary there.
template <class E, class S>
__device__ int merge_search(E& g, int limit, const SampArgs& sp, const ZigDev& z, typename S::M* own, int* own_cnt) {
  typename S::M hyp[kE];
  unsigned alive = 0;
  for (int q = 0; q < limit; ++q) {
    if (q < kE) { hyp[q].reset(); alive |= 1u << q; }
    unsigned idle = 0;
    for (int e = 0; e < kE; ++e)
      if (((alive >> e) & 1u) && hyp[e].idle()) idle |= 1u << e;
    if (idle) {
      unsigned keep = idle & (~idle + 1u);
      alive &= ~(idle ^ keep);
    }
    if (q >= kE - 1 && __popc(alive) == 1 && (alive & idle)) {
      if (own && !own->idle()) return -2;
      return q;
    }
    u64 u = g.next();
    for (int e = 0; e < kE; ++e)
      if ((alive >> e) & 1u) (void)hyp[e].feed(u, sp, z);
    if (own) *own_cnt += own->feed(u, sp, z);
  }
  return -1;
}

template <int NT>
struct MergeSmem {
  __align__(16) u64 stage[NT / 32][32 * (kRecS + 1) * kRecW];
  int wsum[32];
  int misc[8];
  u64 sh4[4];
  int sig[NT];    // each chunk's merge point (-1: none)
  int surv[NT];   // phased fills: the phases left there
};

// A merge-seam tile holds NT - 1 chunks.  Its last thread starts at the
// next tile's first chunk and only finds that chunk's merge point, so that
// every walk of the tile can stop at a merge point the tile already knows
// instead of searching for it a second time.
template <int NT, int C>
struct MergeGeom {
  static constexpr int kChunks = NT - 1;
  static constexpr int T = kChunks * C;
};

// One tile of a merge-seam fill (gamma, beta).  Returns false when the fill
// needs no further tiles (or a device check failed): the caller stops.
template <int NT, int C, class E, class S>
__device__ bool merge_tile(const FillArgs& a, u64 k, const E& e, MergeSmem<NT>& sm) {
  constexpr int T = MergeGeom<NT, C>::T;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const ZigDev& z = g_zig[0];   // read through L1 (keeps shared memory small)
  double* out = (double*)a.out;
  // one reader, so that every thread takes the same branch
  if (t == 0) sm.misc[5] = ld_volatile(&a.ctrl->done_tile) < k;
  __syncthreads();
  if (sm.misc[5]) return false;
  // ---------------- pass 1: merge point, walk, count, next merge point
  E g = e;
  int sig = 0, cnt = 0, endp = -1;
  bool ok = true;
  if (!(k == 0 && t == 0)) {
    sig = merge_search<E, S>(g, C, a.sp, z, nullptr, nullptr);
    if (sig < 0) ok = false;   // no merge point in this chunk: no segment
  }
  sm.sig[t] = ok ? sig : -1;
  __syncthreads();
  if (t == NT - 1) ok = false;   // the next tile's first chunk: looked at, not walked
  typename S::M m;
  m.reset();
  if (ok) {
    for (int p = sig; p < C; ++p) cnt += m.feed(g.next(), a.sp, z);
    int q = -1, u = 1;
    for (; u <= kSkipMax; ++u) {
      if (t + u < NT) {
        // a merge point this tile knows: walk to it
        const int qn = sm.sig[t + u];
        const int lim = qn < 0 ? C : qn;
        for (int p = 0; p < lim; ++p) cnt += m.feed(g.next(), a.sp, z);
        if (qn < 0) continue;      // no merge point in that chunk: the walk crosses it
        q = m.idle() ? qn : -2;
        break;
      }
      q = merge_search<E, S>(g, C, a.sp, z, &m, &cnt);
      if (q != -1) break;       // else: the own chain has crossed that chunk; try the next
    }
    if (q == -1) { set_err(a.ctrl, E_NOSYNC, k); ok = false; }
    else if (q == -2) { set_err(a.ctrl, E_LANDING, k); ok = false; }
    else endp = u * C + q;
  }
  // ---------------- offsets
  int off = block_exclusive_scan<NT>(cnt, sm.wsum, &sm.misc[1]);
  if (t < 32) {
    unsigned long long ex = lookback_warp(a.tile_status, k, (unsigned long long)sm.misc[1], a.ctrl, -1, 0,
                                          a.spin_max, a.stall_tile1);
    if (t == 0) {
      sm.misc[2] = (int)(ex & 0x7fffffff);
      sm.misc[3] = (int)(ex >> 31);
      sm.misc[4] = (ex == ~0ull);
    }
  }
  __syncthreads();
  if (sm.misc[4]) return false;
  const u64 base = (u64)(unsigned)sm.misc[2] | ((u64)(unsigned)sm.misc[3] << 31);
  const u64 chunk0 = k * (u64)T + (u64)t * C;
  if (k + 1 == a.n_tiles && base + (u64)sm.misc[1] < a.n) {
    // ran out of tiles: the last segment of the tile ends where the chain continues
    if (t == 0) sm.sh4[0] = 0;
    __syncthreads();
    if (ok) atomicMax((unsigned long long*)&sm.sh4[0], chunk0 + (u64)endp);
    __syncthreads();
    if (t == 0) {
      a.ctrl->total = base + (u64)sm.misc[1];
      a.ctrl->next_pos = sm.sh4[0];
      a.ctrl->last_tile = k;
    }
  }
  // ---------------- pass 2: regenerate, stage records, evaluate while writing
  if (base < a.n) {
    g = e;
    for (int q = 0; q < sig; ++q) (void)g.next();
    m.reset();
    const u64 my0 = base + (u64)off;
    int emitted = 0;
    int p = sig;
    bool active = ok && cnt > 0;
    u64* myrow = &sm.stage[wid][lane * (kRecS + 1) * kRecW];
    while (__any_sync(0xffffffffu, active)) {
      int ns = 0;
      while (active && ns < kRecS) {
        u64 u = g.next();
        ++p;
        if (!m.feed(u, a.sp, z)) continue;
        u64* r = myrow + ns * kRecW;
        m.record(r);
        const u64 gi = my0 + emitted + ns;
        r[7] = 0;
        if (S::needs_tail(r) && gi < a.n) {
          unsigned long long qi = atomicAdd(a.tail_count, 1ull);
          if (qi < a.tail_cap) {
            TailEntry te;
            te.g = a.tail_abs ? (u64)(out + gi) : gi;
            te.w0 = r[0];
            te.w1 = (u64)a.req;
            for (int j = 0; j < 6; ++j) te.x[j] = r[1 + j];
            a.tailq[qi] = te;
            r[7] = 1;
          }
        }
        ++ns;
        if (gi == a.n - 1) {
          a.ctrl->next_pos = chunk0 + (u64)p;
          atomicMin(&a.ctrl->done_tile, k);
        }
        if (emitted + ns == cnt) active = false;
      }
      __syncwarp();
      // evaluate and write: 32 lanes on 32 consecutive (row, slot) entries
      const u64 dst = my0 + emitted;
      for (int it = 0; it < kRecS; ++it) {
        int ent = it * 32 + lane;
        int rr = ent / kRecS, col = ent % kRecS;
        u64 d = __shfl_sync(0xffffffffu, dst, rr);
        int c = __shfl_sync(0xffffffffu, ns, rr);
        if (col < c && d + col < a.n) {
          const u64* r = &sm.stage[wid][(rr * (kRecS + 1) + col) * kRecW];
          if (!r[7]) out[d + col] = S::value(r, a.sp, z);
        }
      }
      __syncwarp();
      emitted += ns;
    }
  }
  __syncthreads();
  return true;
}

// ------------------------------------------------------------------ phased merge seams
// Beta (and F) draw X ~ Gamma(a), then Y ~ Gamma(b), from one stream.  When
// the two shapes consume words alike, chains that enter a chunk at different
// offsets soon sit at the same gamma boundary but one gamma apart, and stay
// so: full merge points become rare.  A phased merge point only needs every
// hypothesis (entry offset, entry phase) at a gamma boundary after the same
// word; at most two states remain there, one per phase (0: X next, 1: Y
// next).  Each thread walks from its phased merge point once per entry phase
// to the next one, which gives a map: entry phase -> (exit phase, outputs).
// The warp scan and the decoupled look-back compose these maps.  A variate
// in progress at a seam (phase 1: X drawn, Y not) belongs to the walk that
// reaches the seam: it goes on until Y is complete, and the next thread,
// entering in phase 1, skips that first completion.  Every walk thus ends
// at a variate boundary, as in the unphased fills.

struct PMap {
  int f;        // bit p: exit phase for entry phase p
  int c0, c1;   // outputs for entry phase 0, 1
};
__device__ __forceinline__ PMap pm_identity() { return PMap{2, 0, 0}; }
// (a after b)(x) = a(b(x))
__device__ __forceinline__ PMap pm_compose(PMap a, PMap b) {
  const int b0 = b.f & 1, b1 = (b.f >> 1) & 1;
  PMap r;
  r.f = ((a.f >> b0) & 1) | (((a.f >> b1) & 1) << 1);
  r.c0 = b.c0 + (b0 ? a.c1 : a.c0);
  r.c1 = b.c1 + (b1 ? a.c1 : a.c0);
  return r;
}
__device__ __forceinline__ PMap pm_shfl_up(PMap m, int o) {
  return PMap{__shfl_up_sync(0xffffffffu, m.f, o), __shfl_up_sync(0xffffffffu, m.c0, o),
              __shfl_up_sync(0xffffffffu, m.c1, o)};
}
__device__ __forceinline__ PMap pm_shfl_down(PMap m, int o) {
  return PMap{__shfl_down_sync(0xffffffffu, m.f, o), __shfl_down_sync(0xffffffffu, m.c0, o),
              __shfl_down_sync(0xffffffffu, m.c1, o)};
}
__device__ __forceinline__ PMap pm_shfl(PMap m, int l) {
  return PMap{__shfl_sync(0xffffffffu, m.f, l), __shfl_sync(0xffffffffu, m.c0, l), __shfl_sync(0xffffffffu, m.c1, l)};
}

// The two walks of a thread (entry phase 0 and 1), fed in lockstep until
// they meet (both at a gamma boundary in one phase: the same state), then as
// one.
template <class S>
struct PhWalk {
  typename S::L m[2];
  int cnt[2];
  bool same;
  __device__ __forceinline__ void feed(u64 u, const SampArgs& sp, const ZigDev& z) {
    if (!same && m[0].idle() && m[1].idle() && m[0].phase() == m[1].phase()) same = true;
    const int c = m[0].feed(u, sp, z);
    cnt[0] += c;
    if (same) cnt[1] += c;
    else cnt[1] += m[1].feed(u, sp, z);
  }
};

// Phased merge point of the chunk at the engine's position, within `limit`
// words: hypotheses typename S::L started at each offset below kE in both
// phases, all fed the same words, until every one is at a gamma boundary
// after the same word (at most one state per phase is then left).  *surv:
// bit p set if a state in phase p is left.  `w` (nullable) is fed the same
// words; *bad gets bit x when walk x is not in a surviving state there (that
// walk cannot be the true chain).  Returns the point (relative) or -1 if
// none within `limit` words.  (Requiring full coalescence first, where it
// comes within a few hundred words, was measured slower: the 12 extra
// hypotheses run longer than the second walk they save.)
template <class E, class S>
__device__ int seam_search(E& g, int limit, const SampArgs& sp, const ZigDev& z, int* surv, PhWalk<S>* w, int* bad) {
  typename S::L hyp[2 * kE];   // hypothesis 2e + p: entry offset e, phase p
  unsigned alive = 0;
  for (int q = 0; q < limit; ++q) {
    if (q < kE) {
      hyp[2 * q].reset(0);
      hyp[2 * q + 1].reset(1);
      alive |= 3u << (2 * q);
    }
    unsigned idle = 0, ph1 = 0;
    for (int h = 0; h < 2 * kE; ++h)
      if (((alive >> h) & 1u) && hyp[h].idle()) {
        idle |= 1u << h;
        if (hyp[h].phase()) ph1 |= 1u << h;
      }
    if (idle) {
      // at a boundary after the same word, equal phases are equal states
      const unsigned i0 = idle & ~ph1, i1 = idle & ph1;
      const unsigned keep = (i0 & (~i0 + 1u)) | (i1 & (~i1 + 1u));
      alive &= ~(idle ^ keep);
    }
    if (q >= kE - 1 && (alive & ~idle) == 0) {
      *surv = ((alive & ~ph1) ? 1 : 0) | ((alive & ph1) ? 2 : 0);
      if (w) {
        for (int x = 0; x < 2; ++x) {
          const typename S::L& m = w->m[w->same ? 0 : x];
          if (!(m.idle() && ((*surv >> m.phase()) & 1))) *bad |= 1 << x;
        }
      }
      return q;
    }
    const u64 u = g.next();
    for (int h = 0; h < 2 * kE; ++h)
      if ((alive >> h) & 1u) (void)hyp[h].feed(u, sp, z);
    if (w) w->feed(u, sp, z);
  }
  return -1;
}

// Decoupled look-back over phase maps, run by one warp (as lookback_warp).
// Status word: bit 63 aggregate (bits 60-61 the map's exit phases, 30-59 and
// 0-29 its counts), bit 62 inclusive (bit 61 the phase, 0-60 the count).
// Returns the state entering tile k as an inclusive payload, or ~0 if the
// bounded wait ran out or the tile became unnecessary.
__device__ unsigned long long lookback_warp_ph(unsigned long long* st, unsigned long long k, PMap agg, Ctrl* ctrl,
                                              unsigned long long spin_max, unsigned long long stall_tile1) {
  if (stall_tile1 && k + 1 == stall_tile1) return ~0ull;   // test hook: this tile never publishes
  const unsigned long long smax = spin_max ? spin_max : kSpinMax;
  const unsigned long long AGG = 1ull << 63, INC = 1ull << 62, CNT = (1ull << 61) - 1, C30 = (1ull << 30) - 1;
  const int lane = threadIdx.x & 31;
  auto apply = [&](PMap m, unsigned long long in) {
    const int p = (int)((in >> 61) & 1);
    return ((unsigned long long)((m.f >> p) & 1) << 61) | ((in & CNT) + (unsigned long long)(p ? m.c1 : m.c0));
  };
  unsigned long long entry = 0;   // the fill starts in phase 0 with no outputs
  if (k > 0) {
    if (lane == 0)
      *(volatile unsigned long long*)(st + k) =
          AGG | ((unsigned long long)agg.f << 60) | ((unsigned long long)agg.c0 << 30) | (unsigned long long)agg.c1;
    PMap acc = pm_identity();   // aggregates passed so far, later tiles outermost
    long long j = (long long)k - 1;
    unsigned long long spins = 0;
    for (;;) {
      const long long idx = j - lane;
      const unsigned long long v = idx >= 0 ? ld_volatile(st + idx) : INC;
      const unsigned incm = __ballot_sync(0xffffffffu, (v & INC) != 0);
      const unsigned rdym = __ballot_sync(0xffffffffu, (v & (INC | AGG)) != 0);
      const int fi = incm ? __ffs(incm) - 1 : 32;
      const unsigned need = fi < 32 ? (2u << fi) - 1u : 0xffffffffu;
      if ((rdym & need) != need) {
        int stop = 0;
        if (lane == 0) {
          if (ld_volatile(&ctrl->done_tile) < k) stop = 1;
          else if (++spins > smax) { set_err(ctrl, E_TIMEOUT, k); stop = 1; }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) return ~0ull;
        __nanosleep(64);
        continue;
      }
      PMap m = lane < fi ? PMap{(int)((v >> 60) & 3), (int)((v >> 30) & C30), (int)(v & C30)} : pm_identity();
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const PMap other = pm_shfl_down(m, o);
        if (lane + o < 32) m = pm_compose(m, other);   // lane l: tiles j-l (latest) down to j-l-2o+1
      }
      acc = pm_compose(acc, pm_shfl(m, 0));
      if (fi < 32) {
        const unsigned long long inc = __shfl_sync(0xffffffffu, v, fi) & ~(AGG | INC);
        entry = apply(acc, inc);
        break;
      }
      j -= 32;
    }
  }
  if (lane == 0) *(volatile unsigned long long*)(st + k) = INC | apply(agg, entry);
  return entry;
}

// One tile of a phased merge-seam fill (beta, F), one warp per tile.
// Returns false when the fill needs no further tiles (or a device check
// failed): the caller stops.
template <int NT, int C, class E, class S>
__device__ bool merge_tile_ph(const FillArgs& a, u64 k, const E& e, MergeSmem<NT>& sm) {
  static_assert(NT == 32, "one warp per tile");
  constexpr int T = MergeGeom<NT, C>::T;
  const int lane = threadIdx.x;
  const ZigDev& z = g_zig[0];
  double* out = (double*)a.out;
  if (lane == 0) sm.misc[5] = ld_volatile(&a.ctrl->done_tile) < k;
  __syncwarp();
  if (sm.misc[5]) return false;
  // ---------------- pass 1: phased merge point, both walks, next point
  E g = e;
  int sig = 0, surv = 1;   // the fill's first word: phase 0
  bool ok = true;
  if (!(k == 0 && lane == 0)) {
    int nobad = 0;
    sig = seam_search<E, S>(g, C, a.sp, z, &surv, nullptr, &nobad);
    if (sig < 0) ok = false;   // no merge point in this chunk: no segment
  }
  sm.sig[lane] = ok ? sig : -1;
  sm.surv[lane] = surv;
  __syncwarp();
  if (lane == NT - 1) ok = false;   // the next tile's first chunk: looked at, not walked
  // an entry phase that no hypothesis has here cannot occur: take the other
  const int sp0 = (surv & 1) ? 0 : 1, sp1 = (surv & 2) ? 1 : 0;
  PhWalk<S> w;
  w.m[0].reset(sp0);
  w.m[1].reset(sp1);
  w.cnt[0] = sp0 ? -1 : 0;   // entering in phase 1: the first completion is the previous walk's
  w.cnt[1] = sp1 ? -1 : 0;
  w.same = sp0 == sp1;
  int endp[2] = {0, 0}, f = 2, bad = 0;
  if (ok) {
    for (int p = sig; p < C; ++p) w.feed(g.next(), a.sp, z);
    int q = -1, u = 1, dummy = 0;
    for (; u <= kSkipMax; ++u) {
      if (lane + u < NT) {
        // a merge point this tile knows: walk to it
        const int qn = sm.sig[lane + u];
        const int lim = qn < 0 ? C : qn;
        for (int p = 0; p < lim; ++p) w.feed(g.next(), a.sp, z);
        if (qn < 0) continue;      // no merge point in that chunk: the walks cross it
        const int sv = sm.surv[lane + u];
        for (int x = 0; x < 2; ++x) {
          const typename S::L& mx = w.m[w.same ? 0 : x];
          if (!(mx.idle() && ((sv >> mx.phase()) & 1))) bad |= 1 << x;
        }
        q = qn;
        break;
      }
      q = seam_search<E, S>(g, C, a.sp, z, &dummy, &w, &bad);
      if (q != -1) break;       // else: the walks have crossed that chunk; try the next
    }
    if (q == -1) { set_err(a.ctrl, E_NOSYNC, k); ok = false; }
    else {
      // (once the walks have met, m[1] is no longer fed: m[0] stands for both)
      const int p0 = w.m[0].phase(), p1 = w.same ? p0 : w.m[1].phase();
      f = p0 | (p1 << 1);
      // a walk in phase 1 at the seam completes its variate's Y
      for (int x = 0; x < (w.same ? 1 : 2); ++x) {
        int len = 0;
        if ((x ? p1 : p0) == 1) {
          E gx = g;
          bool done = false;
          for (; len < C && !done; ++len) done = w.m[x].feed(gx.next(), a.sp, z) != 0;
          if (!done) { set_err(a.ctrl, E_LANDING, k); ok = false; }
          w.cnt[x] += 1;
          if (w.same) w.cnt[1] += 1;
        }
        endp[x] = u * C + q + len;
      }
      if (w.same) endp[1] = endp[0];
    }
  }
  // ---------------- warp scan of the maps, look-back
  PMap mine = ok ? PMap{f, w.cnt[0], w.cnt[1]} : pm_identity();
  PMap inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const PMap other = pm_shfl_up(inc, o);
    if (lane >= o) inc = pm_compose(inc, other);
  }
  PMap ex = pm_shfl_up(inc, 1);
  if (lane == 0) ex = pm_identity();
  const PMap agg = pm_shfl(inc, 31);
  const unsigned long long ent = lookback_warp_ph(a.tile_status, k, agg, a.ctrl, a.spin_max, a.stall_tile1);
  if (ent == ~0ull) return false;
  const int ph_in = (int)((ent >> 61) & 1);
  const u64 base = ent & ((1ull << 61) - 1);
  const int ph = (ex.f >> ph_in) & 1;                       // this thread's entry phase
  const bool missed = ok && ((bad >> ph) & 1);
  if (__any_sync(0xffffffffu, missed)) {
    // the true chain is a walk that missed the seam: the seam rule's premise
    // (a gamma variate overhangs a chunk by less than kE words) failed
    if (missed) set_err(a.ctrl, E_LANDING, k);
    return false;
  }
  const int off = ph_in ? ex.c1 : ex.c0;
  const int cnt = ok ? (ph ? w.cnt[1] : w.cnt[0]) : 0;
  const u64 total = (u64)(ph_in ? agg.c1 : agg.c0);
  const u64 chunk0 = k * (u64)T + (u64)lane * C;
  if (k + 1 == a.n_tiles && base + total < a.n) {
    // ran out of tiles: the tile's last walk ends where the chain continues,
    // at a variate boundary
    u64 np = ok ? chunk0 + (u64)endp[ph] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const u64 y = __shfl_xor_sync(0xffffffffu, np, o);
      np = y > np ? y : np;
    }
    if (lane == 0) {
      a.ctrl->total = base + total;
      a.ctrl->next_pos = np;
      a.ctrl->last_tile = k;
    }
  }
  // ---------------- pass 2: regenerate, stage records, evaluate while writing
  if (base < a.n) {
    g = e;
    for (int q = 0; q < sig; ++q) (void)g.next();
    typename S::M m;
    const int st = ph ? sp1 : sp0;
    m.reset(st);
    bool skip = st == 1;
    const u64 my0 = base + (u64)off;
    int emitted = 0;
    int p = sig;
    bool active = ok && cnt > 0;
    u64* myrow = &sm.stage[0][lane * (kRecS + 1) * kRecW];
    while (__any_sync(0xffffffffu, active)) {
      int ns = 0;
      while (active && ns < kRecS) {
        u64 u = g.next();
        ++p;
        if (!m.feed(u, a.sp, z)) continue;
        if (skip) { skip = false; continue; }
        u64* r = myrow + ns * kRecW;
        m.record(r);
        const u64 gi = my0 + emitted + ns;
        r[7] = 0;
        if (S::needs_tail(r) && gi < a.n) {
          unsigned long long qi = atomicAdd(a.tail_count, 1ull);
          if (qi < a.tail_cap) {
            TailEntry te;
            te.g = a.tail_abs ? (u64)(out + gi) : gi;
            te.w0 = r[0];
            te.w1 = (u64)a.req;
            for (int j = 0; j < 6; ++j) te.x[j] = r[1 + j];
            a.tailq[qi] = te;
            r[7] = 1;
          }
        }
        ++ns;
        if (gi == a.n - 1) {
          a.ctrl->next_pos = chunk0 + (u64)p;
          atomicMin(&a.ctrl->done_tile, k);
        }
        if (emitted + ns == cnt) active = false;
      }
      __syncwarp();
      const u64 dst = my0 + emitted;
      for (int it = 0; it < kRecS; ++it) {
        int ent2 = it * 32 + lane;
        int rr = ent2 / kRecS, col = ent2 % kRecS;
        u64 d = __shfl_sync(0xffffffffu, dst, rr);
        int c = __shfl_sync(0xffffffffu, ns, rr);
        if (col < c && d + col < a.n) {
          const u64* r = &sm.stage[0][(rr * (kRecS + 1) + col) * kRecW];
          if (!r[7]) S::store(out, d + col, r, a.sp, z);
        }
      }
      __syncwarp();
      emitted += ns;
    }
  }
  __syncwarp();
  return true;
}

template <int NT, int C, class E, class S>
__global__ void __launch_bounds__(NT, 512 / NT) k_merge(FillArgs a) {
  __shared__ MergeSmem<NT> sm;
  E e;
  e.init_tile(a.eng, blockIdx.x, threadIdx.x, sm.sh4);
  for (u64 k = blockIdx.x; k < a.n_tiles; k += gridDim.x) {
    bool more;
    if constexpr (S::kPhased) more = merge_tile_ph<NT, C, E, S>(a, k, e, sm);
    else more = merge_tile<NT, C, E, S>(a, k, e, sm);
    if (!more) break;
    e.advance(a.eng);
  }
}

template <int NT, int C, class E>
__global__ void __launch_bounds__(NT) k_onepw_batch(BatchArgs b) {
  __shared__ __align__(16) u64 stage[NT / 32][32 * kRowW];
  __shared__ u64 sh4[4];
  __shared__ FillArgs fa;
  __shared__ unsigned long long slot;
  const int wid = threadIdx.x >> 5;
  BatchItem bi;
  while (batch_claim(b, fa, bi, &slot)) {
    E e;
    e.init_tile(fa.eng, bi.tile, threadIdx.x, sh4);
    if (fa.dist == D_U64) onepw_tile<NT, E, SampU64>(fa, bi.tile, e, stage[wid], C);
    else if (fa.dist == D_UNIFORM52) onepw_tile<NT, E, SampUniform52>(fa, bi.tile, e, stage[wid], C);
    else onepw_tile<NT, E, SampUniform>(fa, bi.tile, e, stage[wid], C);
  }
}

template <int NT, int C, class E>
__global__ void __launch_bounds__(NT, 512 / NT) k_merge_batch(BatchArgs b) {
  __shared__ MergeSmem<NT> sm;
  __shared__ FillArgs fa;
  __shared__ unsigned long long slot;
  BatchItem bi;
  while (batch_claim(b, fa, bi, &slot)) {
    E e;
    e.init_tile(fa.eng, bi.tile, threadIdx.x, sm.sh4);
    if (fa.dist == D_GAMMA) merge_tile<NT, C, E, SampGamma>(fa, bi.tile, e, sm);
    else merge_tile_ph<NT, C, E, SampBeta>(fa, bi.tile, e, sm);
  }
}

template <class S>
__global__ void k_tails_rec(FillArgs a) {
  const ZigDev& z = g_zig[0];
  unsigned long long n = ld_volatile(a.tail_count);
  if (n > a.tail_cap) n = a.tail_cap;
  double* out = (double*)a.out;
  for (unsigned long long i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    TailEntry te = a.tailq[i];
    u64 r[8] = {te.w0, te.x[0], te.x[1], te.x[2], te.x[3], te.x[4], te.x[5], 0};
    if constexpr (S::kPhased) S::store(out, te.g, r, a.sp, z);   // beta: keeps the gamma pair when asked
    else out[te.g] = S::value(r, a.sp, z);
  }
}

template <class S>
__global__ void k_tails(FillArgs a) {
  const ZigDev& z = g_zig[(a.dist == D_EXP || a.dist == D_EXPF) ? 1 : 0];
  unsigned long long n = ld_volatile(a.tail_count);
  if (n > a.tail_cap) n = a.tail_cap;
  typedef typename S::out_t OT;
  OT* out = (OT*)a.out;
  for (unsigned long long i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    TailEntry te = a.tailq[i];
    double v = S::tail_value(te.w0, te.w1, z);
    if (a.sp.epi) v = epi_value(v, a.sp);
    out[te.g] = (OT)v;
  }
}

// Adds this translation unit's fallback counts to out[DBG_N]; reset: zero them.
inline int dbg_read(unsigned long long* out, int reset) {
  unsigned long long h[DBG_N];
  int e = (int)cudaMemcpyFromSymbol(h, g_dbg, sizeof(h));
  if (e) return e;
  for (int i = 0; i < DBG_N; ++i) out[i] += h[i];
  if (reset) {
    for (int i = 0; i < DBG_N; ++i) h[i] = 0;
    e = (int)cudaMemcpyToSymbol(g_dbg, h, sizeof(h));
  }
  return e;
}

// ------------------------------------------------------------------ per-engine entry
constexpr int NT_ = 128;
constexpr int C_ = 384;     // chunk words of the one-word and ziggurat fills (measured best of 256, 384, 512)
constexpr int CM_ = 2048;   // chunk words of the merge-seam samplers in batches (single fills: S::kChunk)
constexpr int NTM_ = 32;    // threads per CTA of the merge-seam samplers
constexpr int CR_ = 256;    // chunk words of the one-pass bounded fill with rejections

template <class E, class S>
int launch_merge(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  if (occ) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_merge<NTM_, S::kChunk, E, S>, NTM_, 0);
    return 0;
  }
  k_merge<NTM_, S::kChunk, E, S><<<grid, NTM_, 0, s>>>(a);
  return (int)cudaGetLastError();
}

template <class E, class S>
int launch_es(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  if constexpr (std::is_same<E, PhiloxDev>::value) {
    if (occ) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_onepw_ctr<NT_, S>, NT_, 0);
      return 0;
    }
    k_onepw_ctr<NT_, S><<<grid, NT_, 0, s>>>(a);
    return (int)cudaGetLastError();
  }
  if (occ) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_onepw<NT_, E, S>, NT_, 0);
    return 0;
  }
  k_onepw<NT_, E, S><<<grid, NT_, 0, s>>>(a);
  return (int)cudaGetLastError();
}

template <class E>
int launch_fold(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  if (occ) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_fold<NT_, E>, NT_, 0);
  k_fold<NT_, E><<<grid, NT_, 0, s>>>(a);
  return (int)cudaGetLastError();
}

template <class E>
int launch_rej(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  if (occ) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_rej<NT_, CR_, E>, NT_, 0);
    return 0;
  }
  k_rej<NT_, CR_, E><<<grid, NT_, 0, s>>>(a);
  return (int)cudaGetLastError();
}

template <class E, class S>
int launch_lean(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  if (occ) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_lean<NT_, C_, E, S>, NT_, 0);
    return 0;
  }
  k_lean<NT_, C_, E, S><<<grid, NT_, 0, s>>>(a);
  return (int)cudaGetLastError();
}

// Batched classes: grid <= 0 reports the occupancy in *occ.
template <class E, int CB>
int launch_batch_c(int cls, const BatchArgs& b, int grid, cudaStream_t s, int* occ) {
  if (cls == BC_ONEPW) {
    if (grid <= 0) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_onepw_batch<NT_, CB, E>, NT_, 0);
    k_onepw_batch<NT_, CB, E><<<grid, NT_, 0, s>>>(b);
  } else if (cls == BC_LEAN) {
    if (grid <= 0) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_lean_batch<NT_, CB, E>, NT_, 0);
    k_lean_batch<NT_, CB, E><<<grid, NT_, 0, s>>>(b);
  } else {
    if (grid <= 0) return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_merge_batch<NTM_, CM_, E>, NTM_, 0);
    k_merge_batch<NTM_, CM_, E><<<grid, NTM_, 0, s>>>(b);
  }
  return (int)cudaGetLastError();
}

template <class E>
int launch_batch_cls(int cls, int cvar, const BatchArgs& b, int grid, cudaStream_t s, int* occ) {
  if (cvar == 1 && cls != BC_MERGE) return launch_batch_c<E, 128>(cls, b, grid, s, occ);
  return launch_batch_c<E, C_>(cls, b, grid, s, occ);
}

template <class E>
int dispatch_dist(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  switch (a.dist) {
    case D_U64: return launch_es<E, SampU64>(a, grid, s, occ);
    case D_UNIFORM: return a.sp.epi ? launch_es<E, SampUniformE>(a, grid, s, occ) : launch_es<E, SampUniform>(a, grid, s, occ);
    case D_BOUNDED: return launch_rej<E>(a, grid, s, occ);
    case D_BOUNDED_ONE:
      return (a.sp.m >> 32) ? launch_es<E, SampBoundedOne>(a, grid, s, occ) : launch_es<E, SampBoundedOne32>(a, grid, s, occ);
    case D_UNIFORM52: return launch_es<E, SampUniform52>(a, grid, s, occ);
    case D_FOLD: return launch_fold<E>(a, grid, s, occ);
    case D_UNIFORMF2: return launch_es<E, SampUniformF2>(a, grid, s, occ);
    case D_NORMALF: return launch_lean<HalfWords<E>, LeanNormalF>(a, grid, s, occ);
    case D_EXPF: return launch_lean<HalfWords<E>, LeanExpF>(a, grid, s, occ);
    case D_NORMAL: return a.sp.epi ? launch_lean<E, LeanNormalE>(a, grid, s, occ) : launch_lean<E, LeanNormal>(a, grid, s, occ);
    case D_EXP: return a.sp.epi ? launch_lean<E, LeanExpE>(a, grid, s, occ) : launch_lean<E, LeanExp>(a, grid, s, occ);
    case D_GAMMA: return a.sp.ga.boost ? launch_merge<E, SampGammaBoost>(a, grid, s, occ) : launch_merge<E, SampGamma>(a, grid, s, occ);
    case D_BETA: return launch_merge<E, SampBeta>(a, grid, s, occ);
    case D_T: return launch_merge<E, SampT>(a, grid, s, occ);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace rp

// Defines the entry points of one engine's translation unit.
#define RP_ENGINE_TU(NAME, ENGINE)                                                              \
  namespace rp {                                                                               \
  int dispatch_##NAME(const FillArgs& a, int grid, void* s, int* occ) {                        \
    return dispatch_dist<ENGINE>(a, grid, (cudaStream_t)s, occ);                               \
  }                                                                                            \
  int batch_##NAME(int cls, int cvar, const BatchArgs& b, int grid, void* s, int* occ) {      \
    return launch_batch_cls<ENGINE>(cls, cvar, b, grid, (cudaStream_t)s, occ);                 \
  }                                                                                            \
  int upload_zig_##NAME(const void* host2) {                                                   \
    return (int)cudaMemcpyToSymbol(g_zig, host2, 2 * sizeof(ZigDev));                          \
  }                                                                                            \
  int dbg_##NAME(unsigned long long* out, int reset) {                                         \
    return dbg_read(out, reset);                                                               \
  }                                                                                            \
  }
