// Fill kernels of librp (sm_103a), included once per engine translation unit.
//
// A stream is cut into tiles of T = NT*C consecutive words.  Persistent CTAs
// take tiles round-robin (tile k by CTA k mod grid); thread t of a tile owns
// chunk t (C consecutive words) and reaches its chunk in the next tile by one
// constant jump of its engine state, so each thread generates long runs of
// its stream with one jump per C words.
//
// One word per variate (raw words, uniforms): the output index of a word is
// known, so every thread streams its chunk out through a per-warp staging
// buffer that turns the chunk-contiguous runs into coalesced 128-byte lines.
//
// Rejection samplers: each thread runs the serial sampler as a state machine
// fed one word at a time.  The parallel parse (chains of candidates across
// chunk seams) uses sync points:
//   * len(q) is the number of words a candidate starting at word q would
//     consume (evaluated speculatively for any q);
//   * the sync point of a chunk is the first s in [G, G+S) (relative to the
//     chunk) such that every candidate starting in [0, s) ends by s.  The
//     true chain, which enters the chunk from the previous one, then passes
//     through s unless a candidate longer than G straddles the seam;
//   * thread t runs the sampler from its sync point to the next chunk's sync
//     point, which it evaluates itself from the same words with the same
//     rule, and checks that the chain lands on it (E_LANDING otherwise).
// Pass 1 counts the outputs of each segment; a block scan and a decoupled
// look-back over tile counts give every thread its first output index; pass
// 2 regenerates the chunk and writes the values through the staging buffer.
// Outputs whose value needs FP64 libm (ziggurat tails, ~3e-4 of outputs) are
// queued and evaluated by full warps in a second kernel.
#pragma once
#include <cuda_runtime.h>

#include "rp_device.cuh"
#include "rp_internal.h"

namespace rp {

// Each translation unit that includes this file owns its copy of the tables
// (no relocatable device code); upload_zig_tu() fills it.
static __device__ ZigDev g_zig[2];

namespace {

constexpr u64 M52 = (1ull << 52) - 1;
constexpr u64 M53 = (1ull << 53) - 1;
constexpr int kG = 8;                                 // sync window
constexpr int kS = 24;                                // sync search length
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
  // libm logs (one ulp) decide unless the sides are within their effect
  double o1 = __dsub_rn(1.0, u53_bits(w1)), o2 = __dsub_rn(1.0, u53_bits(w2));
  double a = __ddiv_rn(-log(o1), z.R), b = -log(o2);
  double l2 = __dadd_rn(b, b), r2 = __dmul_rn(a, a);
  double mg = (l2 + r2) * 0x1.0p-48;
  if (l2 > r2 + mg) return true;
  if (l2 < r2 - mg) return false;
  a = __ddiv_rn(-cr_log_dev(o1), z.R);
  b = -cr_log_dev(o2);
  return __dadd_rn(b, b) > __dmul_rn(a, a);
}

#include "rp_gamma.cuh"

// ------------------------------------------------------------------ samplers
// Each sampler is a state machine fed one word at a time, run twice over a
// segment.  Pass 1 (feed1) counts outputs and records the accept decisions
// in chain order: wedge tests are queued per lane and evaluated after the
// chunk (all lanes together, instead of one divergent lane at a time), tail
// pair tests are evaluated on the spot (they decide the candidate length).
// Pass 2 (feed2) replays the recorded decisions; feed2 returns OUT_VAL with
// the word whose value is the output, or OUT_TAIL with the two words of a
// tail output (FP64 libm, evaluated later by full warps).
enum { OUT_NONE = 0, OUT_VAL = 1, OUT_TAIL = 2 };
constexpr int kPend = 16;    // wedge tests queued per lane and chunk

struct Rec {
  u64 wbits, tbits;          // wedge / tail-pair decisions in chain order
  int nw, nt, np;            // decisions recorded, pending wedge tests
  int replay;                // 0: pass 2 must re-evaluate decisions
  u64 pu0[kPend], pu1[kPend];
  __device__ __forceinline__ void reset() { wbits = tbits = 0; nw = nt = np = 0; replay = 1; }
  __device__ __forceinline__ void push_tail(bool b) {
    if (nt < 64) tbits |= (u64)b << nt;
    else replay = 0;
    ++nt;
  }
};

struct SampU64 {
  static constexpr bool kOnePerWord = true;
  typedef u64 out_t;
  __device__ static __forceinline__ u64 value1(u64 u, const SampArgs&) { return u; }
};
struct SampUniform {
  static constexpr bool kOnePerWord = true;
  typedef double out_t;
  __device__ static __forceinline__ double value1(u64 u, const SampArgs&) { return u53_bits(u); }
};

// Lemire (Sec. 3.2): one word per attempt; accept when low64(u m) >= 2^64 mod m.
struct SampBounded {
  static constexpr bool kOnePerWord = false;
  static constexpr bool kLen1 = true;
  typedef u64 out_t;
  struct M {
    __device__ __forceinline__ void reset() {}
    __device__ __forceinline__ bool idle() const { return true; }
    __device__ __forceinline__ int feed1(u64 u, const ZigDev&, const SampArgs& a, Rec&) {
      return u * a.m >= a.thresh;
    }
    __device__ __forceinline__ int feed2(u64 u, const ZigDev&, const SampArgs& a, Rec&, u64* ew, u64*, u64*) {
      *ew = u;
      return u * a.m >= a.thresh ? OUT_VAL : OUT_NONE;
    }
  };
  __device__ static __forceinline__ int settle(Rec&, const ZigDev&) { return 0; }
  __device__ static __forceinline__ u64 value(u64 u, const ZigDev&, const SampArgs& a) { return __umul64hi(u, a.m); }
  template <class E>
  __device__ static __forceinline__ int len(u64, const E&, const ZigDev&) { return 1; }
  __device__ static double tail_value(u64, u64, const ZigDev&) { return 0.0; }
};

// Normal ziggurat (Sec. 3.1): bits 0-7 strip i, bit 8 sign, bits 9-60 r.
struct SampNormal {
  static constexpr bool kOnePerWord = false;
  static constexpr bool kLen1 = false;
  typedef double out_t;
  struct M {
    int st;  // 0 idle, 1 wedge waiting for U, 2 tail waiting for U1, 3 tail waiting for U2
    u64 u0, w1;
    __device__ __forceinline__ void reset() { st = 0; }
    __device__ __forceinline__ bool idle() const { return st == 0; }
    __device__ __forceinline__ int feed1(u64 u, const ZigDev& z, const SampArgs&, Rec& rc) {
      if (st == 0) {
        int i = (int)(u & 0xff);
        if (((u >> 9) & M52) < z.k[i]) return 1;
        u0 = u;
        st = i ? 1 : 2;
        return 0;
      }
      if (st == 1) {
        st = 0;
        if (rc.np < kPend) {
          rc.pu0[rc.np] = u0;
          rc.pu1[rc.np] = u;
          ++rc.np;
          return 0;
        }
        rc.replay = 0;  // too many to queue: decide here, pass 2 re-decides
        return wedge_accept<true>((u0 >> 9) & M52, (int)(u0 & 0xff), u, z);
      }
      if (st == 2) { w1 = u; st = 3; return 0; }
      bool ok = tail_pair_accept(w1, u, z);
      rc.push_tail(ok);
      st = ok ? 0 : 2;
      return ok;
    }
    __device__ __forceinline__ int feed2(u64 u, const ZigDev& z, const SampArgs&, Rec& rc, u64* ew, u64* t0,
                                         u64* t1) {
      if (st == 0) {
        int i = (int)(u & 0xff);
        if (((u >> 9) & M52) < z.k[i]) { *ew = u; return OUT_VAL; }
        u0 = u;
        st = i ? 1 : 2;
        return OUT_NONE;
      }
      if (st == 1) {
        st = 0;
        bool ok = rc.replay ? ((rc.wbits >> rc.nw) & 1) : wedge_accept<true>((u0 >> 9) & M52, (int)(u0 & 0xff), u, z);
        ++rc.nw;
        if (!ok) return OUT_NONE;
        *ew = u0;
        return OUT_VAL;
      }
      if (st == 2) { w1 = u; st = 3; return OUT_NONE; }
      bool ok = rc.replay ? ((rc.tbits >> rc.nt) & 1) : tail_pair_accept(w1, u, z);
      ++rc.nt;
      if (!ok) { st = 2; return OUT_NONE; }
      st = 0;
      *t0 = u0;
      *t1 = w1;
      return OUT_TAIL;
    }
  };
  // pass-1 wedge tests queued in the chunk, all lanes together
  __device__ static int settle(Rec& rc, const ZigDev& z) {
    int c = 0;
    for (int j = 0; j < rc.np; ++j) {
      bool ok = wedge_accept<true>((rc.pu0[j] >> 9) & M52, (int)(rc.pu0[j] & 0xff), rc.pu1[j], z);
      rc.wbits |= (u64)ok << j;
      c += ok;
    }
    rc.nw = 0;
    rc.nt = 0;
    return c;
  }
  __device__ static __forceinline__ double value(u64 u, const ZigDev& z, const SampArgs&) {
    int i = (int)(u & 0xff);
    return neg_if(mul_rn_dmul((u >> 9) & M52, z.w[i]), (u >> 8) & 1);
  }
  // speculative candidate length at a word; `g` is the engine positioned
  // right after it (copied, never advanced)
  template <class E>
  __device__ static __forceinline__ int len(u64 u, const E& g, const ZigDev& z) {
    int i = (int)(u & 0xff);
    if (((u >> 9) & M52) < z.k[i]) return 1;
    if (i != 0) return 2;
    E h = g;
    for (int k = 1; k <= kTailPairsMax; ++k) {
      u64 a = h.next(), b = h.next();
      if (tail_pair_accept(a, b, z)) return 1 + 2 * k;
    }
    return 1 << 20;  // longer than any window: no sync point here
  }
  // +-(R + a), a = -log(1-U1)/R of the accepted pair; libm log (within 2 ulp
  // of the correctly rounded value)
  __device__ static double tail_value(u64 u0, u64 w1, const ZigDev& z) {
    double a = __ddiv_rn(-log(__dsub_rn(1.0, u53_bits(w1))), z.R);
    return neg_if(__dadd_rn(z.R, a), (u0 >> 8) & 1);
  }
};

// Exponential ziggurat (Sec. 3.1): bits 0-7 strip i, bits 8-60 r; tail R - log(1-U).
struct SampExp {
  static constexpr bool kOnePerWord = false;
  static constexpr bool kLen1 = false;
  typedef double out_t;
  struct M {
    int st;  // 0 idle, 1 wedge waiting for U, 2 tail waiting for U
    u64 u0;
    __device__ __forceinline__ void reset() { st = 0; }
    __device__ __forceinline__ bool idle() const { return st == 0; }
    __device__ __forceinline__ int feed1(u64 u, const ZigDev& z, const SampArgs&, Rec& rc) {
      if (st == 0) {
        int i = (int)(u & 0xff);
        if (((u >> 8) & M53) < z.k[i]) return 1;
        u0 = u;
        st = i ? 1 : 2;
        return 0;
      }
      int s = st;
      st = 0;
      if (s == 2) return 1;  // the tail always accepts
      if (rc.np < kPend) {
        rc.pu0[rc.np] = u0;
        rc.pu1[rc.np] = u;
        ++rc.np;
        return 0;
      }
      rc.replay = 0;
      return wedge_accept<false>((u0 >> 8) & M53, (int)(u0 & 0xff), u, z);
    }
    __device__ __forceinline__ int feed2(u64 u, const ZigDev& z, const SampArgs&, Rec& rc, u64* ew, u64* t0,
                                         u64* t1) {
      if (st == 0) {
        int i = (int)(u & 0xff);
        if (((u >> 8) & M53) < z.k[i]) { *ew = u; return OUT_VAL; }
        u0 = u;
        st = i ? 1 : 2;
        return OUT_NONE;
      }
      int s = st;
      st = 0;
      if (s == 2) { *t0 = u0; *t1 = u; return OUT_TAIL; }
      bool ok = rc.replay ? ((rc.wbits >> rc.nw) & 1) : wedge_accept<false>((u0 >> 8) & M53, (int)(u0 & 0xff), u, z);
      ++rc.nw;
      if (!ok) return OUT_NONE;
      *ew = u0;
      return OUT_VAL;
    }
  };
  __device__ static int settle(Rec& rc, const ZigDev& z) {
    int c = 0;
    for (int j = 0; j < rc.np; ++j) {
      bool ok = wedge_accept<false>((rc.pu0[j] >> 8) & M53, (int)(rc.pu0[j] & 0xff), rc.pu1[j], z);
      rc.wbits |= (u64)ok << j;
      c += ok;
    }
    rc.nw = 0;
    rc.nt = 0;
    return c;
  }
  __device__ static __forceinline__ double value(u64 u, const ZigDev& z, const SampArgs&) {
    return mul_rn_dmul((u >> 8) & M53, z.w[u & 0xff]);
  }
  template <class E>
  __device__ static __forceinline__ int len(u64 u, const E&, const ZigDev& z) {
    int i = (int)(u & 0xff);
    return ((u >> 8) & M53) < z.k[i] ? 1 : 2;
  }
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
// bit 63 aggregate, bit 62 inclusive, low 62 bits value.  Lane l inspects
// predecessor j - l; the window is consumed up to the nearest inclusive value
// once every entry before it is at least an aggregate.  Returns the tile's
// exclusive prefix in all lanes, or ~0 if the bounded wait ran out or the
// tile became unnecessary.
__device__ unsigned long long lookback_warp(unsigned long long* st, unsigned long long k, unsigned long long cnt,
                                           Ctrl* ctrl) {
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
    long long idx = j - lane;
    unsigned long long v = idx >= 0 ? ld_volatile(st + idx) : INC;
    unsigned inc_mask = __ballot_sync(0xffffffffu, (v & INC) != 0);
    unsigned rdy_mask = __ballot_sync(0xffffffffu, (v & (INC | AGG)) != 0);
    int first = inc_mask ? __ffs(inc_mask) - 1 : 31;
    unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
    if ((rdy_mask & need) != need) {
      int stop = 0;
      if (lane == 0) {
        if (ld_volatile(&ctrl->done_tile) < k) stop = 1;
        else if (++spins > kSpinMax) { set_err(ctrl, E_TIMEOUT, k); stop = 1; }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return ~0ull;
      __nanosleep(64);
      continue;
    }
    unsigned long long c = lane <= first ? (v & VAL) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    excl += c;
    if (inc_mask) break;
    j -= 32;
  }
  if (lane == 0) *(volatile unsigned long long*)(st + k) = INC | (excl + cnt);
  return excl;
}

// ------------------------------------------------------------------ staging
// Lane rows of kStage outputs, flushed by the warp two rows per instruction so
// that each row (a run of consecutive outputs) is written by 16 lanes.
template <class OT>
__device__ __forceinline__ void flush_rows(OT* __restrict__ out, const OT* row_base, u64 dst, int cnt, u64 n) {
  const int lane = threadIdx.x & 31;
  const int half = lane >> 4, col = lane & 15;
#pragma unroll 4
  for (int r = 0; r < 32; r += 2) {
    int rr = r + half;
    u64 d = __shfl_sync(0xffffffffu, dst, rr);
    int c = __shfl_sync(0xffffffffu, cnt, rr);
    if (col < c && d + col < n) out[d + col] = row_base[rr * kRow + col];
  }
}

// ------------------------------------------------------------------ kernels
template <int NT, int C, class E, class S>
__global__ void __launch_bounds__(NT) k_onepw(FillArgs a) {
  // one word per variate: chunk words stream straight to the output
  typedef typename S::out_t OT;
  constexpr int T = NT * C;
  __shared__ __align__(16) OT stage[NT / 32][32 * kRow];
  __shared__ u64 sh4[4];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  OT* out = (OT*)a.out;
  E e;
  e.init_tile(a.eng, blockIdx.x, t, sh4);
  for (u64 k = blockIdx.x; k < a.n_tiles; k += gridDim.x) {
    E g = e;
    u64 base = k * (u64)T + (u64)t * C;
    for (int j0 = 0; j0 < C; j0 += kStage) {
#pragma unroll
      for (int j = 0; j < kStage; ++j) stage[wid][lane * kRow + j] = S::value1(g.next(), a.sp);
      __syncwarp();
      flush_rows<OT>(out, stage[wid], base + j0, kStage, a.n);
      __syncwarp();
    }
    e.advance(a.eng);
  }
}

template <int NT, int C, class E, class S>
__global__ void __launch_bounds__(NT) k_reject(FillArgs a) {
  typedef typename S::out_t OT;
  constexpr int T = NT * C;
  __shared__ __align__(16) OT stage[NT / 32][32 * kRow];
  __shared__ int wsum[32];
  __shared__ int misc[8];
  __shared__ ZigDev zs;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (!S::kLen1) {
    const int which = (a.dist == D_EXP) ? 1 : 0;
    const u64* src = (const u64*)&g_zig[which];
    u64* dst = (u64*)&zs;
    for (int i = t; i < (int)(sizeof(ZigDev) / 8); i += NT) dst[i] = src[i];
    __syncthreads();
  }
  const ZigDev& z = zs;
  OT* out = (OT*)a.out;
  __shared__ u64 sh4[4];
  E e;
  e.init_tile(a.eng, blockIdx.x, t, sh4);

  for (u64 k = blockIdx.x; k < a.n_tiles; k += gridDim.x) {
    if (ld_volatile(&a.ctrl->done_tile) < k) break;
    // ---------------- pass 1: sync point, segment walk, count
    E g = e;
    int sig = 0, cnt = 0, endp = C;
    bool ok = true;
    if (!S::kLen1 && !(k == 0 && t == 0)) {
      // first s in [G, G+S) with every candidate starting in [0, s) ending by s
      int reach = 0;
      sig = -1;
      for (int q = 0; q < kG + kS; ++q) {
        if (q >= kG && reach <= q) { sig = q; break; }
        u64 u = g.next();
        reach = max(reach, q + S::len(u, g, z));
      }
      if (sig < 0) { set_err(a.ctrl, E_NOSYNC, k); ok = false; }
    }
    typename S::M m;
    m.reset();
    Rec rc;
    rc.reset();
    if (ok) {
      for (int p = sig; p < C; ++p) cnt += m.feed1(g.next(), z, a.sp, rc);
      if (!S::kLen1) {
        // the next chunk's sync point, by the same rule, while the chain runs on
        int reach = C;
        endp = -1;
        for (int q = C; q < C + kG + kS; ++q) {
          if (q - C >= kG && reach <= q) {
            endp = q;
            break;
          }
          u64 u = g.next();
          reach = max(reach, q + S::len(u, g, z));
          cnt += m.feed1(u, z, a.sp, rc);
        }
        if (endp < 0) { set_err(a.ctrl, E_NOSYNC, k); ok = false; }
        else if (!m.idle()) { set_err(a.ctrl, E_LANDING, k); ok = false; }
      }
      cnt += S::settle(rc, z);
    }
    // ---------------- offsets
    int off = block_exclusive_scan<NT>(cnt, wsum, &misc[1]);
    if (t < 32) {
      unsigned long long ex = lookback_warp(a.tile_status, k, (unsigned long long)misc[1], a.ctrl);
      if (t == 0) {
        misc[2] = (int)(ex & 0x7fffffff);
        misc[3] = (int)(ex >> 31);
        misc[4] = (ex == ~0ull);
      }
    }
    __syncthreads();
    if (misc[4]) break;
    const u64 base = (u64)(unsigned)misc[2] | ((u64)(unsigned)misc[3] << 31);
    const u64 chunk0 = k * (u64)T + (u64)t * C;   // stream position of the chunk
    if (t == NT - 1 && k + 1 == a.n_tiles && base + (u64)misc[1] < a.n) {
      // ran out of tiles: report where the chain continues
      a.ctrl->total = base + (u64)misc[1];
      a.ctrl->next_pos = chunk0 + (u64)endp;
      a.ctrl->last_tile = k;
    }
    // ---------------- pass 2: regenerate, evaluate, stage, write
    if (base < a.n) {
      g = e;
      for (int q = 0; q < sig; ++q) (void)g.next();
      m.reset();
      const u64 my0 = base + (u64)off;   // first output index of this thread
      int emitted = 0;
      int p = sig;
      bool active = ok && cnt > 0;
      while (__any_sync(0xffffffffu, active)) {
        int ns = 0;
        while (active && ns < kStage) {
          u64 t0 = 0, t1 = 0, ew = 0;
          int r = m.feed2(g.next(), z, a.sp, rc, &ew, &t0, &t1);
          ++p;
          if (r == OUT_NONE) continue;
          const u64 gi = my0 + emitted + ns;
          OT v = S::value(ew, z, a.sp);
          if (r == OUT_TAIL && gi < a.n) {
            unsigned long long qi = atomicAdd(&a.ctrl->n_tail, 1ull);
            if (qi < a.tail_cap) a.tailq[qi] = TailEntry{gi, t0, t1};
            else v = (OT)S::tail_value(t0, t1, z);
          }
          stage[wid][lane * kRow + ns] = v;
          ++ns;
          if (gi == a.n - 1) {
            a.ctrl->next_pos = chunk0 + (u64)p;
            atomicMin(&a.ctrl->done_tile, k);
          }
          if (emitted + ns == cnt) active = false;
        }
        __syncwarp();
        flush_rows<OT>(out, stage[wid], my0 + emitted, ns, a.n);
        __syncwarp();
        emitted += ns;
      }
    }
    __syncthreads();
    e.advance(a.eng);
  }
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
constexpr int kSkipMax = 8;  // chunks a walk may cross to find a merge point
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

template <int NT, int C, class E, class S>
__global__ void __launch_bounds__(NT) k_merge(FillArgs a) {
  constexpr int T = NT * C;
  __shared__ __align__(16) u64 stage[NT / 32][32 * (kRecS + 1) * kRecW];
  __shared__ int wsum[32];
  __shared__ int misc[8];
  __shared__ u64 sh4[4];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const ZigDev& z = g_zig[0];   // read through L1 (keeps shared memory small)
  double* out = (double*)a.out;
  E e;
  e.init_tile(a.eng, blockIdx.x, t, sh4);

  for (u64 k = blockIdx.x; k < a.n_tiles; k += gridDim.x) {
    if (ld_volatile(&a.ctrl->done_tile) < k) break;
    // ---------------- pass 1: merge point, walk, count, next merge point
    E g = e;
    int sig = 0, cnt = 0, endp = -1;
    bool ok = true;
    if (!(k == 0 && t == 0)) {
      sig = merge_search<E, S>(g, C, a.sp, z, nullptr, nullptr);
      if (sig < 0) ok = false;   // no merge point in this chunk: no segment
    }
    typename S::M m;
    m.reset();
    if (ok) {
      for (int p = sig; p < C; ++p) cnt += m.feed(g.next(), a.sp, z);
      int q = -1, u = 1;
      for (; u <= kSkipMax; ++u) {
        q = merge_search<E, S>(g, C, a.sp, z, &m, &cnt);
        if (q != -1) break;       // else: the own chain has crossed that chunk; try the next
      }
      if (q == -1) { set_err(a.ctrl, E_NOSYNC, k); ok = false; }
      else if (q == -2) { set_err(a.ctrl, E_LANDING, k); ok = false; }
      else endp = u * C + q;
    }
    // ---------------- offsets
    int off = block_exclusive_scan<NT>(cnt, wsum, &misc[1]);
    if (t < 32) {
      unsigned long long ex = lookback_warp(a.tile_status, k, (unsigned long long)misc[1], a.ctrl);
      if (t == 0) {
        misc[2] = (int)(ex & 0x7fffffff);
        misc[3] = (int)(ex >> 31);
        misc[4] = (ex == ~0ull);
      }
    }
    __syncthreads();
    if (misc[4]) break;
    const u64 base = (u64)(unsigned)misc[2] | ((u64)(unsigned)misc[3] << 31);
    const u64 chunk0 = k * (u64)T + (u64)t * C;
    if (k + 1 == a.n_tiles && base + (u64)misc[1] < a.n) {
      // ran out of tiles: the last segment of the tile ends where the chain continues
      if (t == 0) sh4[0] = 0;
      __syncthreads();
      if (ok) atomicMax((unsigned long long*)&sh4[0], chunk0 + (u64)endp);
      __syncthreads();
      if (t == 0) {
        a.ctrl->total = base + (u64)misc[1];
        a.ctrl->next_pos = sh4[0];
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
      u64* myrow = &stage[wid][lane * (kRecS + 1) * kRecW];
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
            unsigned long long qi = atomicAdd(&a.ctrl->n_tail, 1ull);
            if (qi < a.tail_cap) {
              TailEntry te;
              te.g = gi; te.w0 = r[0]; te.w1 = 0;
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
            const u64* r = &stage[wid][(rr * (kRecS + 1) + col) * kRecW];
            if (!r[7]) out[d + col] = S::value(r, a.sp, z);
          }
        }
        __syncwarp();
        emitted += ns;
      }
    }
    __syncthreads();
    e.advance(a.eng);
  }
}

template <class S>
__global__ void k_tails_rec(FillArgs a) {
  const ZigDev& z = g_zig[0];
  unsigned long long n = ld_volatile(&a.ctrl->n_tail);
  if (n > a.tail_cap) n = a.tail_cap;
  double* out = (double*)a.out;
  for (unsigned long long i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    TailEntry te = a.tailq[i];
    u64 r[8] = {te.w0, te.x[0], te.x[1], te.x[2], te.x[3], te.x[4], te.x[5], 0};
    out[te.g] = S::value(r, a.sp, z);
  }
}

template <class S>
__global__ void k_tails(FillArgs a) {
  const ZigDev& z = g_zig[a.dist == D_EXP ? 1 : 0];
  unsigned long long n = ld_volatile(&a.ctrl->n_tail);
  if (n > a.tail_cap) n = a.tail_cap;
  typedef typename S::out_t OT;
  OT* out = (OT*)a.out;
  for (unsigned long long i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    TailEntry te = a.tailq[i];
    out[te.g] = (OT)S::tail_value(te.w0, te.w1, z);
  }
}

// ------------------------------------------------------------------ per-engine entry
constexpr int NT_ = 128;
constexpr int C_ = 256;
constexpr int CM_ = 2048;   // chunk words of the merge-seam samplers
constexpr int NTM_ = 32;    // threads per CTA of the merge-seam samplers

template <class E, class S>
int launch_merge(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  if (occ) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_merge<NTM_, CM_, E, S>, NTM_, 0);
    return 0;
  }
  k_merge<NTM_, CM_, E, S><<<grid, NTM_, 0, s>>>(a);
  return (int)cudaGetLastError();
}

template <class E, class S>
int launch_es(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  if constexpr (S::kOnePerWord) {
    if (occ) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_onepw<NT_, C_, E, S>, NT_, 0);
      return 0;
    }
    k_onepw<NT_, C_, E, S><<<grid, NT_, 0, s>>>(a);
  } else {
    if (occ) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_reject<NT_, C_, E, S>, NT_, 0);
      return 0;
    }
    k_reject<NT_, C_, E, S><<<grid, NT_, 0, s>>>(a);
  }
  return (int)cudaGetLastError();
}

template <class E>
int dispatch_dist(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  switch (a.dist) {
    case D_U64: return launch_es<E, SampU64>(a, grid, s, occ);
    case D_UNIFORM: return launch_es<E, SampUniform>(a, grid, s, occ);
    case D_BOUNDED: return launch_es<E, SampBounded>(a, grid, s, occ);
    case D_NORMAL: return launch_es<E, SampNormal>(a, grid, s, occ);
    case D_EXP: return launch_es<E, SampExp>(a, grid, s, occ);
    case D_GAMMA: return launch_merge<E, SampGamma>(a, grid, s, occ);
    case D_BETA: return launch_merge<E, SampBeta>(a, grid, s, occ);
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
  int upload_zig_##NAME(const void* host2) {                                                   \
    return (int)cudaMemcpyToSymbol(g_zig, host2, 2 * sizeof(ZigDev));                          \
  }                                                                                            \
  }
