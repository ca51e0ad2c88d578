// Bitmap two-pass fill for samplers whose candidate length is fixed by the
// candidate's first word: the normal ziggurat (1 word fast, 2 words wedge,
// 1 + 2k words tail), the exponential ziggurat (1 or 2 words) and Lemire's
// bounded integers (1 word).
//
// Tiles, chunks, sync points and the look-back are those of the file header.
// What differs is how the two passes share work:
//   pass 1 walks the chain and records, per thread, a bitmap of the chunk
//          positions whose candidate produced an output (wedge tests are
//          queued in shared memory and decided after the walk, all lanes
//          together; tail outputs go to a per-tile list);
//   pass 2 regenerates the words and turns every marked word into its value,
//          with no parsing at all, writing through the per-warp staging rows.
// The common step (a fast-accept candidate) is one 32-bit compare of the
// word's top significand bits against k_i >> 20 (normal) or >> 21
// (exponential); equal top bits fall back to the full 52/53-bit compare.
//
// Fragment of rp_fill_impl.cuh, included inside its namespace after the
// samplers, scans and staging helpers.

// Out-of-line copies of the rare tests, so that the unrolled walk stays small.
__device__ __noinline__ bool tail_pair_nl(u64 w1, u64 w2, const ZigDev& z) { return tail_pair_accept(w1, w2, z); }
template <bool kNormal>
__device__ __noinline__ bool wedge_nl(u64 r, int i, u64 u2, const ZigDev& z) { return wedge_accept<kNormal>(r, i, u2, z); }

struct LeanTab {
  unsigned khi[256];   // top 32 bits of the 52/53-bit fast-accept bound k_i
  double w[256];       // w_i; the float samplers keep their float w_i's bits in the low word
                       // (read as a float with no conversion on the FP64 pipe)
};

// RN(r w) for 0 <= r < 2^53 with one fused multiply-add: D = 2^52 + (r mod
// 2^52) is exact, and D w - 2^52 w = (r mod 2^52) w exactly, so
// fma(D, w, -2^52 w) rounds the exact product once; for r >= 2^52, D = r and
// the addend is zero.  Same value as the definition's single rounding.
// -2^52 w is formed on the bits of w (positive, normal, far from overflow):
// exponent + 52 and the sign bit, one integer add on the high word.
__device__ __forceinline__ double mul_rn_fma(u64 r, double w) {
  const double D = __longlong_as_double((long long)(0x4330000000000000ull | (r & M52)));
  const double c = __longlong_as_double(__double_as_longlong(w) + (long long)0x8340000000000000ull);
  return __fma_rn(D, w, (r >> 52) ? 0.0 : c);
}

// The walk's view of a word, per sampler:
//   fast_hi   the 32-bit fast-accept test (top significand bits below the
//             bound's), exact unless tie() (equal top bits: fast_exact decides);
//   pack_pos  the wedge queue's second word with the candidate's position in
//             bits the wedge test does not read (pos_of reads it back);
//   tail_pair the normal tail's pair test;   tab_w  the table's w_i.
#define LEAN_WORD_HOOKS                                                                               \
  __device__ static __forceinline__ bool fast_hi(u64 u, const LeanTab& tb) {                          \
    return (unsigned)(u >> 29) < tb.khi[u & 0xff];                                                    \
  }                                                                                                   \
  __device__ static __forceinline__ bool tie(u64 u, const LeanTab& tb) {                              \
    return (unsigned)(u >> 29) == tb.khi[u & 0xff];                                                   \
  }                                                                                                   \
  __device__ static __forceinline__ u64 pack_pos(u64 u1, int pos) { return (u1 & ~0x7ffull) | (u64)pos; } \
  __device__ static __forceinline__ int pos_of(u64 u1) { return (int)(u1 & 0x7ff); }                  \
  __device__ static __forceinline__ bool tail_pair(u64 w1, u64 w2, const ZigDev& z) {                 \
    return tail_pair_nl(w1, w2, z);                                                                   \
  }                                                                                                   \
  __device__ static __forceinline__ double tab_w(double w) { return w; }

// Normal ziggurat (Sec. 3.1): bits 0-7 strip, bit 8 sign, bits 9-60 r.
// kEpi: the base of a derived distribution, each value transformed as written.
template <bool kEpi>
struct LeanNormalT {
  static constexpr bool kSync = true;
  static constexpr int kWhich = 0;
  static constexpr int kKShift = 20;
  // A tail of 1 + 2k words that starts just before a seam overhangs it by up
  // to 2k words, so sync points start at 16: an overhang past 16 needs
  // k >= 9 (probability 0.062^8 per tail), against k >= 5 (1.5e-5) for 8,
  // which a 2^28-variate fill met about once in 170.  kG + kS stays 32: the
  // walk into the next chunk fits the one overhang mask word.
  static constexpr int kG = 16, kS = 16;
  static constexpr bool kTailPairs = true;
  typedef double out_t;
  __device__ static __forceinline__ bool fast_exact(u64 u, const ZigDev& z) { return ((u >> 9) & M52) < z.k[u & 0xff]; }
  __device__ static __forceinline__ bool fast(u64 u, const LeanTab& tb, const ZigDev& z) {
    const unsigned rh = (unsigned)(u >> 29), kh = tb.khi[u & 0xff];
    if (rh != kh) return rh < kh;
    return fast_exact(u, z);
  }
  LEAN_WORD_HOOKS
  __device__ static __forceinline__ double value(u64 u, const LeanTab& tb, const SampArgs& a) {
    const double x = mul_rn_fma((u >> 9) & M52, tb.w[u & 0xff]);
    const double v = __longlong_as_double(__double_as_longlong(x) ^ (long long)((u >> 8 & 1) << 63));
    if constexpr (kEpi) return epi_value(v, a);
    else return v;
  }
  __device__ static __forceinline__ bool wedge(u64 u0, u64 u1, const ZigDev& z) {
    return wedge_nl<true>((u0 >> 9) & M52, (int)(u0 & 0xff), u1, z);
  }
  template <class E>
  __device__ static __forceinline__ int len(u64 u, const E& g, const LeanTab& tb, const ZigDev& z) {
    if (fast(u, tb, z)) return 1;
    if ((u & 0xff) != 0) return 2;
    E h = g;
    for (int k = 1; k <= kTailPairsMax; ++k) {
      u64 a = h.next(), b = h.next();
      if (tail_pair_nl(a, b, z)) return 1 + 2 * k;
    }
    return 1 << 20;
  }
};

using LeanNormal = LeanNormalT<false>;
using LeanNormalE = LeanNormalT<true>;

// Exponential ziggurat (Sec. 3.1): bits 0-7 strip, bits 8-60 r; the tail
// takes one more word and always accepts, so every candidate is 1 or 2 words
// and a sync window of 2 suffices.
template <bool kEpi>
struct LeanExpT {
  static constexpr bool kSync = true;
  static constexpr int kWhich = 1;
  static constexpr int kKShift = 21;
  static constexpr int kG = 2, kS = 24;
  static constexpr bool kTailPairs = false;
  typedef double out_t;
  __device__ static __forceinline__ bool fast_exact(u64 u, const ZigDev& z) { return ((u >> 8) & M53) < z.k[u & 0xff]; }
  __device__ static __forceinline__ bool fast(u64 u, const LeanTab& tb, const ZigDev& z) {
    const unsigned rh = (unsigned)(u >> 29), kh = tb.khi[u & 0xff];
    if (rh != kh) return rh < kh;
    return fast_exact(u, z);
  }
  LEAN_WORD_HOOKS
  __device__ static __forceinline__ double value(u64 u, const LeanTab& tb, const SampArgs& a) {
    const double v = mul_rn_fma((u >> 8) & M53, tb.w[u & 0xff]);
    if constexpr (kEpi) return epi_value(v, a);
    else return v;
  }
  __device__ static __forceinline__ bool wedge(u64 u0, u64 u1, const ZigDev& z) {
    return wedge_nl<false>((u0 >> 8) & M53, (int)(u0 & 0xff), u1, z);
  }
  template <class E>
  __device__ static __forceinline__ int len(u64 u, const E&, const LeanTab& tb, const ZigDev& z) {
    return fast(u, tb, z) ? 1 : 2;
  }
};

using LeanExp = LeanExpT<false>;
using LeanExpE = LeanExpT<true>;

// ------------------------------------------------------------------ float ziggurats
// The float variants (Table "continuous", suffix f) over 32-bit half-words
// (HalfWords: each u holds one in its low 32 bits).  Normal: bits 0-7 strip,
// bit 8 sign, bits 9-31 r (23 bits); exponential: bits 8-31 r (24 bits).
// x = RN_f(r wf_i) with wf_i = RN_f(2^29 w_i); fast accept r < k_i / 2^29
// (integer division); the wedge takes y = RN_f((f_{i-1} - f_i) U + f_i) in
// float operations with f_i = RN_f(F_i) and U = u24 of the next half-word,
// and accepts y < exp(t) (t = -x^2/2 or -x, exact in double) against the
// correctly rounded exp; tails are the double samplers' with U = u24 of the
// next half-words, in double, rounded once to float (k_tails).

// Wedge test of the float samplers: FP32 with the margin of wedge_accept,
// then the exact decision.
template <bool kNormal>
__device__ __noinline__ bool wedge_f(unsigned r, int i, unsigned h1, const ZigDev& z) {
  const float x = __fmul_rn((float)r, __fmul_rn(z.wf[i], 0x1.0p29f));
  const float U = (float)(h1 >> 8) * 0x1.0p-24f;
  const float y = __fadd_rn(__fmul_rn(__fsub_rn(z.ff[i - 1], z.ff[i]), U), z.ff[i]);
  const float tf = kNormal ? __fmul_rn(__fmul_rn(-0.5f, x), x) : -x;
  const float ef = expf(tf);
  const float m = 0x1.0p-19f * (1.0f - tf);
  if (y < ef * (1.0f - m)) return true;
  if (y > ef * (1.0f + m)) return false;
  dbg_count(DBG_WEDGE_FP64);
  const double xd = (double)x;
  const double t = kNormal ? __dmul_rn(-0.5, __dmul_rn(xd, xd)) : -xd;
  return lt_cr_exp((double)y, t);
}

// Normal tail pair over half-words: a = -log(1 - U1)/R, b = -log(1 - U2),
// accept when 2b > a^2; libm logs decide unless within their error, then
// the correctly rounded ones.
__device__ __noinline__ bool tail_pair_f(u64 w1, u64 w2, const ZigDev& z) {
  const double o1 = __dsub_rn(1.0, u24d(w1)), o2 = __dsub_rn(1.0, u24d(w2));
  double a = __ddiv_rn(-log(o1), z.R), b = -log(o2);
  double l2 = __dadd_rn(b, b), r2 = __dmul_rn(a, a);
  const double mg = (l2 + r2) * 0x1.0p-48;
  if (l2 > r2 + mg) return true;
  if (l2 < r2 - mg) return false;
  dbg_count(DBG_TAIL_CR);
  a = __ddiv_rn(-cr_log_nl(o1), z.R);
  b = -cr_log_nl(o2);
  return __dadd_rn(b, b) > __dmul_rn(a, a);
}

#define LEAN_HALF_HOOKS                                                                               \
  __device__ static __forceinline__ bool fast_exact(u64 u, const ZigDev& z) {                         \
    return r_of(u) < (unsigned)(z.k[u & 0xff] >> 29);                                                 \
  }                                                                                                   \
  __device__ static __forceinline__ bool fast(u64 u, const LeanTab& tb, const ZigDev&) {              \
    return r_of(u) < tb.khi[u & 0xff];                                                                \
  }                                                                                                   \
  __device__ static __forceinline__ bool fast_hi(u64 u, const LeanTab& tb) { return r_of(u) < tb.khi[u & 0xff]; } \
  __device__ static __forceinline__ bool tie(u64, const LeanTab&) { return false; }                   \
  __device__ static __forceinline__ u64 pack_pos(u64 u1, int pos) { return (u1 & 0xffffffffull) | ((u64)pos << 32); } \
  __device__ static __forceinline__ int pos_of(u64 u1) { return (int)(u1 >> 32); }                   \
  __device__ static __forceinline__ bool tail_pair(u64 w1, u64 w2, const ZigDev& z) {                 \
    return tail_pair_f(w1, w2, z);                                                                    \
  }                                                                                                   \
  __device__ static __forceinline__ double tab_w(double w) {                                          \
    return __longlong_as_double((long long)__float_as_uint(__fmul_rn(__double2float_rn(w), 0x1.0p29f))); \
  }                                                                                                   \
  __device__ static __forceinline__ float wf_of(const LeanTab& tb, u64 u) {                           \
    return __uint_as_float((unsigned)__double_as_longlong(tb.w[u & 0xff]));                           \
  }

struct LeanNormalF {
  static constexpr bool kSync = true;
  static constexpr int kWhich = 0;
  static constexpr int kKShift = 29;   // k_i >> 29: the 23-bit bound itself
  static constexpr int kG = 16, kS = 16;
  static constexpr bool kTailPairs = true;
  typedef float out_t;
  __device__ static __forceinline__ unsigned r_of(u64 u) { return ((unsigned)u >> 9) & 0x7fffffu; }
  LEAN_HALF_HOOKS
  __device__ static __forceinline__ float value(u64 u, const LeanTab& tb, const SampArgs&) {
    const float x = __fmul_rn((float)r_of(u), wf_of(tb, u));
    return ((u >> 8) & 1) ? -x : x;
  }
  __device__ static __forceinline__ bool wedge(u64 u0, u64 u1, const ZigDev& z) {
    return wedge_f<true>(r_of(u0), (int)(u0 & 0xff), (unsigned)u1, z);
  }
  template <class E>
  __device__ static __forceinline__ int len(u64 u, const E& g, const LeanTab& tb, const ZigDev& z) {
    if (fast(u, tb, z)) return 1;
    if ((u & 0xff) != 0) return 2;
    E h = g;
    for (int k = 1; k <= kTailPairsMax; ++k) {
      u64 a = h.next(), b = h.next();
      if (tail_pair_f(a, b, z)) return 1 + 2 * k;
    }
    return 1 << 20;
  }
};

struct LeanExpF {
  static constexpr bool kSync = true;
  static constexpr int kWhich = 1;
  static constexpr int kKShift = 29;   // k_i >> 29: the 24-bit bound itself
  static constexpr int kG = 2, kS = 24;
  static constexpr bool kTailPairs = false;
  typedef float out_t;
  __device__ static __forceinline__ unsigned r_of(u64 u) { return (unsigned)u >> 8; }
  LEAN_HALF_HOOKS
  __device__ static __forceinline__ float value(u64 u, const LeanTab& tb, const SampArgs&) {
    return __fmul_rn((float)r_of(u), wf_of(tb, u));
  }
  __device__ static __forceinline__ bool wedge(u64 u0, u64 u1, const ZigDev& z) {
    return wedge_f<false>(r_of(u0), (int)(u0 & 0xff), (unsigned)u1, z);
  }
  template <class E>
  __device__ static __forceinline__ int len(u64 u, const E&, const LeanTab& tb, const ZigDev& z) {
    return fast(u, tb, z) ? 1 : 2;
  }
};

// Lemire (Sec. 3.2): one word per attempt, no seams to synchronise.
struct LeanBounded {
  static constexpr bool kSync = false;
  static constexpr int kWhich = 0;
  static constexpr int kKShift = 20;
  static constexpr int kG = 0, kS = 0;
  static constexpr bool kTailPairs = false;
  typedef u64 out_t;
  __device__ static __forceinline__ bool fast_exact(u64, const ZigDev&) { return true; }
  LEAN_WORD_HOOKS
  __device__ static __forceinline__ u64 value(u64 u, const LeanTab&, const SampArgs& a) {
    return __umul64hi(u, a.m);
  }
  template <class E>
  __device__ static __forceinline__ int len(u64, const E&, const LeanTab&, const ZigDev&) { return 1; }
};

constexpr int kLPend = 8;        // queued wedge tests per lane and chunk
constexpr int kTileTails = 64;   // tail records per tile (mean ~14 for the normal at 384-word chunks)

// Chain state of pass 1 for one thread.
struct LeanChain {
  int st;        // 0 expect a candidate, 1 wedge U word, 2/3 normal tail pair words, 4 exponential tail word
  int pp;        // position of the pending candidate's first word
  int np;        // queued wedge tests
  u64 pu0, pw1;  // pending candidate's first word; first word of the current tail pair
};

// The uncommon steps of the pass-1 walk: a candidate that is not a fast
// accept (or whose top bits tie with the bound), and every word inside a
// multi-word candidate.  Output positions are marked in the bitmap (`mw` is
// mask word b, still in a register; earlier words are in shared memory).
template <int NT, class S>
__device__ __forceinline__ void lean_rare(u64 u, int p, int b, unsigned& mw, LeanChain& c, const LeanTab& tb, const ZigDev& z,
                                          unsigned (*msk)[NT], u64* queue, u64 (*tails)[3], int* ntails,
                                          Ctrl* ctrl, u64 k) {
  const int t = threadIdx.x;
  auto mark = [&](int q) {
    if ((q >> 5) == b) mw |= 1u << (q & 31);
    else msk[q >> 5][t] |= 1u << (q & 31);
  };
  auto tail_rec = [&](u64 w1) {
    int slot = atomicAdd(ntails, 1);
    if (slot < kTileTails) {
      tails[slot][0] = c.pu0;
      tails[slot][1] = w1;
      tails[slot][2] = ((u64)t << 32) | (unsigned)c.pp;
    } else {
      set_err(ctrl, E_OVERFLOW, k);
    }
  };
  if (c.st == 0) {
    // a candidate that missed the 32-bit test: only equal top bits need the full compare
    if (S::tie(u, tb) && S::fast_exact(u, z)) { mark(p); return; }
    c.pu0 = u;
    c.pp = p;
    c.st = (u & 0xff) ? 1 : (S::kTailPairs ? 2 : 4);
  } else if (c.st == 1) {
    c.st = 0;
    const u64 u1 = S::pack_pos(u, c.pp);   // the position rides in bits the wedge test does not read
    if (c.np < kLPend) {
      queue[(c.np * NT + t) * 2] = c.pu0;
      queue[(c.np * NT + t) * 2 + 1] = u1;
      ++c.np;
    } else if (S::wedge(c.pu0, u1, z)) {
      mark(c.pp);
    }
  } else if (c.st == 4) {
    c.st = 0;
    mark(c.pp);
    tail_rec(u);
  } else if (c.st == 2) {
    c.pw1 = u;
    c.st = 3;
  } else if (S::tail_pair(c.pw1, u, z)) {
    c.st = 0;
    mark(c.pp);
    tail_rec(c.pw1);
  } else {
    c.st = 2;
  }
}

// One word of the walk: the common case (a fast accept) sets one bit.
template <int NT, class S>
__device__ __forceinline__ void lean_step(u64 u, int p, int b, unsigned& mw, LeanChain& c, const LeanTab& tb,
                                          const ZigDev& z, unsigned (*msk)[NT], u64* queue, u64 (*tails)[3],
                                          int* ntails, Ctrl* ctrl, u64 k) {
  if (c.st == 0 && S::fast_hi(u, tb)) mw |= 1u << (p & 31);
  else lean_rare<NT, S>(u, p, b, mw, c, tb, z, msk, queue, tails, ntails, ctrl, k);
}

// Staged rows -> output: row r of the warp holds lane r's `cnt` (<= 16)
// consecutive outputs starting at tile-relative output `off`; each store
// instruction writes two rows, 16 lanes each.  `lim` = outputs left in the
// fill from the tile's first output.
template <class OT>
__device__ __forceinline__ void flush_rows16(OT* __restrict__ outb, const OT* rows, int off, int cnt, int lim) {
  const int lane = threadIdx.x & 31;
  const int half = lane >> 4, col = lane & 15;
#pragma unroll 4
  for (int r = 0; r < 32; r += 2) {
    const int rr = r + half;
    const int o = __shfl_sync(0xffffffffu, off, rr);
    const int c = min(__shfl_sync(0xffffffffu, cnt, rr), lim - o);
    if (col < c) outb[o + col] = rows[rr * kRow + col];
  }
}

// ------------------------------------------------------------------ bit-parallel chain
// Pass 1 over 16-word half-blocks.  The words sit in shared memory (wb[j NT
// + t]) with one 16-bit mask F: the 32-bit fast test (top significand bits
// below the bound's), exact except where the top bits tie, which the
// half-block step checks at the candidate starts that failed it.  With every
// candidate one or two words long (a tie counted as not fast), the
// positions consumed as second words follow from the non-fast mask N alone:
// position q is consumed when q - 1 is a candidate start that is not fast,
// K(q + 1) = N(q) and not K(q).  Inside each maximal run of N bits starting at
// a candidate start a, the consumed positions are a + 1, a + 3, ...,
// including the position after the run when the run length is odd.  Runs
// starting at even and at odd positions are isolated with one addition each
// (adding the start bit clears exactly that run), and their consumed
// positions are the run shifted by one, masked to odd or even positions.
// Candidate starts are the unconsumed positions.  Only normal tails (more
// than two words) leave the bit-parallel path: the walk goes word by word
// from the tail's first word until the chain is idle, then the bit-parallel
// step resumes.

// Wedge test for a candidate at absolute position pos with words u0, u1.
template <int NT, class S>
__device__ __forceinline__ void lean_push_wedge(u64 u0, u64 u1, int pos, int b, unsigned& mw, LeanChain& c,
                                                const ZigDev& z, unsigned (*msk)[NT], u64* queue) {
  const int t = threadIdx.x;
  const u64 u1p = S::pack_pos(u1, pos);   // the position rides in bits the wedge test does not read
  if (c.np < kLPend) {
    queue[(c.np * NT + t) * 2] = u0;
    queue[(c.np * NT + t) * 2 + 1] = u1p;
    ++c.np;
  } else if (S::wedge(u0, u1p, z)) {
    if ((pos >> 5) == b) mw |= 1u << (pos & 31);
    else msk[pos >> 5][t] |= 1u << (pos & 31);
  }
}

// A tail output at absolute position pos (exponential: always accepted;
// normal: its accepted pair's first word is w1).  The value needs libm, so it
// goes to the tile's tail list.
template <int NT>
__device__ __forceinline__ void lean_exp_tail(u64 u0, u64 w1, int pos, int b, unsigned& mw, unsigned (*msk)[NT],
                                              u64 (*tails)[3], int* ntails, Ctrl* ctrl, u64 k) {
  const int t = threadIdx.x;
  if ((pos >> 5) == b) mw |= 1u << (pos & 31);
  else msk[pos >> 5][t] |= 1u << (pos & 31);
  const int slot = atomicAdd(ntails, 1);
  if (slot < kTileTails) {
    tails[slot][0] = u0;
    tails[slot][1] = w1;
    tails[slot][2] = ((u64)t << 32) | (unsigned)pos;
  } else {
    set_err(ctrl, E_OVERFLOW, k);
  }
}

// One half-block at absolute positions P0 .. P0 + 15, from relative position
// `from` on (earlier positions belong to the previous chain).  The chain
// state c carries a candidate that straddles half-blocks.  F holds the
// 32-bit fast test of every word; everything else is looked up only at the
// candidate starts that failed it (about one word in 85): a tie of the top
// bits (the full compare decides; if it says fast, the chain is recomputed
// from that position), strip 0 (a tail) or a wedge.
template <int NT, class S>
__device__ __forceinline__ void lean_half(int P0, int from, unsigned F, const u64* wb, unsigned& mw, LeanChain& c,
                                          const LeanTab& tb, const ZigDev& z, unsigned (*msk)[NT], u64* queue,
                                          u64 (*tails)[3], int* ntails, Ctrl* ctrl, u64 k) {
  const int t = threadIdx.x;
  const int b = P0 >> 5, sh = P0 & 31;
  unsigned ein = 0;   // position `from` is the second word of a candidate
  if (from == 0 && c.st != 0) {
    if (c.st == 1) {          // wedge started on the previous half-block's last word
      lean_push_wedge<NT, S>(c.pu0, wb[t], c.pp, b, mw, c, z, msk, queue);
      c.st = 0;
      ein = 1;
    } else if (c.st == 4) {   // exponential tail likewise
      lean_exp_tail<NT>(c.pu0, wb[t], c.pp, b, mw, msk, tails, ntails, ctrl, k);
      c.st = 0;
      ein = 1;
    } else {                  // a normal tail in progress: word by word until idle
      int j = 0;
      do {
        lean_step<NT, S>(wb[j * NT + t], P0 + j, b, mw, c, tb, z, msk, queue, tails, ntails, ctrl, k);
        ++j;
      } while (j < 16 && c.st != 0);
      from = j;
    }
  }
  while (from < 16) {
    const unsigned range = (0xffffu << from) & 0xffffu;
    const unsigned N = ~F & range;
    const unsigned R = N & ~(ein << from);
    const unsigned RS = R & ~(R << 1);
    const unsigned Er = R & ~(R + (RS & 0x55555555u));
    const unsigned Or = R & ~(R + (RS & 0xAAAAAAAAu));
    const unsigned K = ((Er << 1) & 0xAAAAAAAAu) | ((Or << 1) & 0x55555555u) | (ein << from);
    const unsigned Sc = ~K & range;   // candidate starts
    // not-fast starts in order; `stop` ends this pass early (a tie that is
    // fast after all, or a normal tail)
    unsigned W = Sc & N;
    int stop = 16;
    bool tie = false;
    while (W) {
      const int j = __ffs(W) - 1;
      W &= W - 1;
      const u64 u0 = wb[j * NT + t];
      if (S::tie(u0, tb) && S::fast_exact(u0, z)) {
        stop = j;
        tie = true;
        break;
      }
      if ((u0 & 0xff) == 0) {
        if constexpr (S::kTailPairs) {   // normal tail: walked below
          stop = j;
          break;
        } else {                          // exponential tail: two words, always accepted
          if (j == 15) { c.st = 4; c.pu0 = u0; c.pp = P0 + 15; }
          else lean_exp_tail<NT>(u0, wb[(j + 1) * NT + t], P0 + j, b, mw, msk, tails, ntails, ctrl, k);
          continue;
        }
      }
      if (j == 15) { c.st = 1; c.pu0 = u0; c.pp = P0 + 15; }
      else lean_push_wedge<NT, S>(u0, wb[(j + 1) * NT + t], P0 + j, b, mw, c, z, msk, queue);
    }
    mw |= (Sc & F & range & ((2u << stop) - 1u) >> 1) << sh;   // fast starts before `stop`
    if (stop == 16) break;
    if (tie) {   // fast after all: the chain from `stop` on changes
      F |= 1u << stop;
      from = stop;
      ein = 0;
      continue;
    }
    // a normal tail at t0 = stop: pairs (t0 + 1, t0 + 2), ... until one is accepted
    const int t0 = stop;
    int q = t0 + 1;
    bool acc = false;
    for (; q + 1 < 16; q += 2) {
      if (S::tail_pair(wb[q * NT + t], wb[(q + 1) * NT + t], z)) {
        lean_exp_tail<NT>(wb[t0 * NT + t], wb[q * NT + t], P0 + t0, b, mw, msk, tails, ntails, ctrl, k);
        acc = true;
        q += 2;
        break;
      }
    }
    if (!acc) {   // the tail runs into the next half-block
      c.pu0 = wb[t0 * NT + t];
      c.pp = P0 + t0;
      if (q < 16) { c.st = 3; c.pw1 = wb[q * NT + t]; }
      else c.st = 2;
      break;
    }
    from = q;
    ein = 0;
  }
}

template <int NT, int C>
struct LeanSmem {
  static constexpr int kMW = C / 32 + 1;   // mask words: the chunk and the overhang into the next one
  static constexpr int kStageW = (NT / 32) * 32 * kRow;
  static constexpr int kQueueW = NT * kLPend * 2;
  static constexpr int kWordsW = NT * 16;   // pass 1: one half-block of words per thread
  static constexpr int kBufW = kStageW > kQueueW + kWordsW ? kStageW : kQueueW + kWordsW;
  __align__(16) u64 sbuf[kBufW];   // pass 1: wedge queue, then the half-block words; pass 2: staging rows
  unsigned msk[kMW][NT];
  u64 tails[kTileTails][3];
  int ntails[2];   // by tile parity: reset one tile after use, behind a barrier
  int wsum[32];
  int misc[8];
  u64 sh4[4];
};

template <class S>
__device__ __forceinline__ void lean_load_tab(LeanTab& tb, int nt) {
  const ZigDev& z = g_zig[S::kWhich];
  for (int i = threadIdx.x; i < 256; i += nt) {
    tb.khi[i] = (unsigned)(z.k[i] >> S::kKShift);
    tb.w[i] = S::tab_w(z.w[i]);
  }
}

// One tile of a bitmap two-pass fill.  `e` is the engine at the thread's
// chunk start, `tb` the sampler's shared table, `par` the tile parity.
// Returns false when the fill needs no further tiles (or a device check
// failed): the caller stops.
template <int NT, int C, class E, class S>
__device__ bool lean_tile(const FillArgs& a, u64 k, const E& e, LeanSmem<NT, C>& sm, const LeanTab& tb, int par) {
  static_assert(C % 32 == 0, "chunks are whole mask words");
  typedef typename S::out_t OT;
  static_assert(sizeof(OT) == 8 || sizeof(OT) == 4, "staging holds 8- or 4-byte outputs");
  constexpr int T = NT * C;
  constexpr int kMW = LeanSmem<NT, C>::kMW;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const ZigDev& z = g_zig[S::kWhich];
  OT* out = (OT*)a.out;
  OT* stage = (OT*)sm.sbuf + wid * 32 * kRow;
  // one reader, so that every thread takes the same branch
  if (t == 0) sm.misc[5] = ld_volatile(&a.ctrl->done_tile) < k;
  __syncthreads();
  if (sm.misc[5]) return false;
    int* nts = &sm.ntails[par];
    // ---------------- pass 1: sync point, chain walk with output bitmap
    int s = (k == 0 && t == 0) ? a.sp.half0 : 0, endp = C;   // half0: a half-word fill resumed mid-word
    bool ok = true;
    if (S::kSync && !(k == 0 && t == 0)) {
      E h = e;
      int reach = 0;
      s = -1;
      for (int q = 0; q < S::kG + S::kS; ++q) {
        if (q >= S::kG && reach <= q) { s = q; break; }
        u64 u = h.next();
        reach = max(reach, q + S::len(u, h, tb, z));
      }
      if (s < 0) { set_err(a.ctrl, E_NOSYNC, k); ok = false; s = 0; }
    }
    LeanChain c;
    c.st = 0; c.pp = 0; c.np = 0; c.pu0 = 0; c.pw1 = 0;
    E g = e;
    if constexpr (!S::kSync) {
      for (int b = 0; b < C / 32; ++b) {
        unsigned mw = 0;
#pragma unroll
        for (int j = 0; j < 32; j += E::kStep) {
          u64 u[E::kStep];
          g.next_step(u);
#pragma unroll
          for (int i = 0; i < E::kStep; ++i) mw |= (unsigned)(u[i] * a.sp.m >= a.sp.thresh) << (j + i);
        }
        sm.msk[b][t] = mw;
      }
      sm.msk[kMW - 1][t] = 0;
    } else {
      // positions [s, C): bit-parallel chain over 16-word half-blocks kept in
      // shared memory (positions before the sync point belong to the previous chain)
      u64* wb = sm.sbuf + LeanSmem<NT, C>::kQueueW;
      for (int b = 0; b < C / 32; ++b) {
        unsigned mw = 0;
        for (int h = 0; h < 2; ++h) {
          const int P0 = b * 32 + h * 16;
          unsigned F = 0;
#pragma unroll
          for (int j = 0; j < 16; j += E::kStep) {
            u64 u[E::kStep];
            g.next_step(u);
#pragma unroll
            for (int i = 0; i < E::kStep; ++i) {
              wb[(j + i) * NT + t] = u[i];
              F |= (unsigned)S::fast_hi(u[i], tb) << (j + i);
            }
          }
          const int from = max(0, min(16, s - P0));
          if (from < 16) lean_half<NT, S>(P0, from, F, wb, mw, c, tb, z, sm.msk, sm.sbuf, sm.tails, nts, a.ctrl, k);
        }
        sm.msk[b][t] = mw;
      }
      // the next chunk's sync point by the same rule, while the chain runs on
      {
        unsigned mw = 0;
        int reach = C;
        endp = -1;
        for (int q = C; q < C + S::kG + S::kS; ++q) {
          if (q - C >= S::kG && reach <= q) { endp = q; break; }
          u64 u = g.next();
          reach = max(reach, q + S::len(u, g, tb, z));
          lean_step<NT, S>(u, q, C / 32, mw, c, tb, z, sm.msk, sm.sbuf, sm.tails, nts, a.ctrl, k);
        }
        sm.msk[kMW - 1][t] = mw;
        if (endp < 0) { set_err(a.ctrl, E_NOSYNC, k); ok = false; endp = C; }
        else if (c.st != 0) { set_err(a.ctrl, E_LANDING, k); ok = false; }
      }
      // queued wedge tests, all lanes together
      for (int j = 0; j < c.np; ++j) {
        const u64 u0 = sm.sbuf[(j * NT + t) * 2], u1 = sm.sbuf[(j * NT + t) * 2 + 1];
        if (S::wedge(u0, u1, z)) {
          const int q = S::pos_of(u1);
          sm.msk[q >> 5][t] |= 1u << (q & 31);
        }
      }
    }
    int cnt = 0;
#pragma unroll
    for (int w = 0; w < kMW; ++w) cnt += __popc(sm.msk[w][t]);
    if (!ok) cnt = 0;
    // ---------------- offsets
    const int off = block_exclusive_scan<NT>(cnt, sm.wsum, &sm.misc[1]);   // also orders the queue reads before staging
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
    if (sm.misc[4]) {
      if (t == 0) *nts = 0;   // nothing reads this tile's tail list any more
      return false;
    }
    const u64 base = (u64)(unsigned)sm.misc[2] | ((u64)(unsigned)sm.misc[3] << 31);
    const u64 chunk0 = k * (u64)T + (u64)t * C;
    const u64 my0 = base + (u64)off;
    if (t == NT - 1 && k + 1 == a.n_tiles && base + (u64)sm.misc[1] < a.n) {
      // ran out of tiles: report where the chain continues
      a.ctrl->total = base + (u64)sm.misc[1];
      a.ctrl->next_pos = chunk0 + (u64)endp;
      a.ctrl->last_tile = k;
    }
    // tail outputs of this thread: output index from the bitmap rank
    const int nt_tile = min(*nts, kTileTails);
    for (int j = 0; j < nt_tile; ++j) {
      const u64 tp = sm.tails[j][2];
      if ((int)(tp >> 32) != t) continue;
      const int p = (int)(unsigned)tp;
      int rank = 0;
      for (int w = 0; w < (p >> 5); ++w) rank += __popc(sm.msk[w][t]);
      rank += __popc(sm.msk[p >> 5][t] & ((1u << (p & 31)) - 1u));
      const u64 gi = my0 + (u64)rank;
      if (gi < a.n) {
        unsigned long long qi = atomicAdd(a.tail_count, 1ull);
        if (qi < a.tail_cap) {
          TailEntry te{};
          te.g = a.tail_abs ? (u64)(out + gi) : gi;
          te.w0 = sm.tails[j][0];
          te.w1 = sm.tails[j][1];
          te.x[0] = (u64)a.dist;
          a.tailq[qi] = te;
        }
        else set_err(a.ctrl, E_OVERFLOW, k);
      }
    }
    // the thread holding output n-1 records where the stream continues
    if (ok && cnt > 0 && my0 <= a.n - 1 && a.n - 1 < my0 + (u64)cnt) {
      int want = (int)(a.n - 1 - my0), p = 0;
      for (int w = 0; w < kMW; ++w) {
        const unsigned m = sm.msk[w][t];
        const int pc = __popc(m);
        if (want < pc) {
          unsigned mm = m;
          for (int r = 0; r < want; ++r) mm &= mm - 1u;
          p = w * 32 + __ffs(mm) - 1;
          break;
        }
        want -= pc;
      }
      E h = e;
      for (int q = 0; q < p; ++q) (void)h.next();
      const u64 u = h.next();
      a.ctrl->next_pos = chunk0 + (u64)(p + S::len(u, h, tb, z));
      atomicMin(&a.ctrl->done_tile, k);
    }
    // ---------------- pass 2: regenerate, evaluate marked words, stage, write
    if (base < a.n) {
      E g2 = e;
      const int nblk = ok ? (endp + 31) >> 5 : 0;
      const int maxblk = __reduce_max_sync(0xffffffffu, nblk);
      OT* outb = out + base;
      const u64 room = a.n - base;
      const int lim = room < (u64)0x7fffffff ? (int)room : 0x7fffffff;
      int myoff = off;
      OT* row = stage + lane * kRow;
      for (int hb = 0; hb < 2 * maxblk; ++hb) {   // half blocks of 16 words
        int ns = 0;
        if ((hb >> 1) < nblk) {
          const unsigned m = sm.msk[hb >> 1][t] >> ((hb & 1) * 16);
#pragma unroll 8 / E::kStep
          for (int j = 0; j < 16; j += E::kStep) {
            u64 u[E::kStep];
            g2.next_step(u);
            // branch-free: every word's value lands in the next free slot
            // (ns <= j <= 15 < kRow), which advances only for marked words
#pragma unroll
            for (int i = 0; i < E::kStep; ++i) {
              row[ns] = S::value(u[i], tb, a.sp);
              ns += (int)((m >> (j + i)) & 1u);
            }
          }
        }
        __syncwarp();
        flush_rows16<OT>(outb, stage, myoff, ns, lim);
        __syncwarp();
        myoff += ns;
      }
    }
    __syncthreads();
    if (t == 0) *nts = 0;   // next used two tiles on, after another barrier
    return true;
}

template <int NT, int C, class E, class S>
__global__ void __launch_bounds__(NT, E::kLeanCtas) k_lean(FillArgs a) {
  __shared__ LeanSmem<NT, C> sm;
  __shared__ LeanTab tb;
  lean_load_tab<S>(tb, NT);
  if (threadIdx.x == 0) { sm.ntails[0] = 0; sm.ntails[1] = 0; }
  __syncthreads();
  E e;
  e.init_tile(a.eng, blockIdx.x, threadIdx.x, sm.sh4);
  int par = 0;
  for (u64 k = blockIdx.x; k < a.n_tiles; k += gridDim.x, par ^= 1) {
    if (!lean_tile<NT, C, E, S>(a, k, e, sm, tb, par)) break;
    e.advance(a.eng);
  }
}

// Batched fills of the ziggurat and bounded samplers: CTAs claim (request,
// tile) items until the list is exhausted; tables for both ziggurats stay in
// shared memory.
template <int NT, int C, class E>
__global__ void __launch_bounds__(NT, 5) k_lean_batch(BatchArgs b) {
  __shared__ LeanSmem<NT, C> sm;
  __shared__ LeanTab tb[2];
  __shared__ FillArgs fa;
  __shared__ unsigned long long slot;
  lean_load_tab<LeanNormal>(tb[0], NT);
  lean_load_tab<LeanExp>(tb[1], NT);
  if (threadIdx.x == 0) { sm.ntails[0] = 0; sm.ntails[1] = 0; }
  __syncthreads();
  int par = 0;
  BatchItem bi;
  while (batch_claim(b, fa, bi, &slot)) {
    E e;
    e.init_tile(fa.eng, bi.tile, threadIdx.x, sm.sh4);
    if (fa.dist == D_NORMAL) lean_tile<NT, C, E, LeanNormal>(fa, bi.tile, e, sm, tb[0], par);
    else if (fa.dist == D_EXP) lean_tile<NT, C, E, LeanExp>(fa, bi.tile, e, sm, tb[1], par);
    else lean_tile<NT, C, E, LeanBounded>(fa, bi.tile, e, sm, tb[0], par);
    par ^= 1;
  }
}
