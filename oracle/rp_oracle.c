/* Serial CPU oracle -- TEST INFRASTRUCTURE ONLY (see rp_oracle.h).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared rp_oracle.c -lm
 *
 * Each function cites the part of Randompack (arXiv 2605.05099) it follows.
 * Where the paper is silent the reading used is stated next to the code.
 */
#include "rp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ziggurat_tables.h"

typedef unsigned __int128 u128;

/* ======================================================================
 * Seeding (Sec. 2.3): seed and spawn key are hashed into a 128-bit entropy
 * pool (four 32-bit words) which is then hashed out to the state words.
 * Reading: NumPy SeedSequence semantics (O'Neill's seed_seq design, which the
 * paper says NumPy also follows); pinned bit-for-bit against NumPy.
 * ==================================================================== */
#define SS_INIT_A 0x43b0d7e5u
#define SS_MULT_A 0x931e8875u
#define SS_INIT_B 0x8b51f9ddu
#define SS_MULT_B 0x58f38dedu
#define SS_MIX_L 0xca01f9ddu
#define SS_MIX_R 0x4973f715u
#define SS_POOL 4

static uint32_t ss_hashmix(uint32_t v, uint32_t* hc) {
  v ^= *hc;
  *hc *= SS_MULT_A;
  v *= *hc;
  v ^= v >> 16;
  return v;
}

static uint32_t ss_mix(uint32_t x, uint32_t y) {
  uint32_t r = SS_MIX_L * x - SS_MIX_R * y;
  r ^= r >> 16;
  return r;
}

void or_seedseq_generate(const uint32_t* ent, int n_ent, uint32_t* out, int n_out) {
  uint32_t pool[SS_POOL];
  uint32_t hc = SS_INIT_A;
  for (int i = 0; i < SS_POOL; ++i) pool[i] = ss_hashmix(i < n_ent ? ent[i] : 0u, &hc);
  for (int src = 0; src < SS_POOL; ++src)
    for (int dst = 0; dst < SS_POOL; ++dst)
      if (src != dst) pool[dst] = ss_mix(pool[dst], ss_hashmix(pool[src], &hc));
  for (int src = SS_POOL; src < n_ent; ++src)
    for (int dst = 0; dst < SS_POOL; ++dst) pool[dst] = ss_mix(pool[dst], ss_hashmix(ent[src], &hc));
  uint32_t hb = SS_INIT_B;
  for (int i = 0; i < n_out; ++i) {
    uint32_t v = pool[i % SS_POOL];
    v ^= hb;
    hb *= SS_MULT_B;
    v *= hb;
    v ^= v >> 16;
    out[i] = v;
  }
}

static int words32(uint64_t x, uint32_t* w) {
  w[0] = (uint32_t)x;
  if (x >> 32) { w[1] = (uint32_t)(x >> 32); return 2; }
  return 1;
}

int or_seedseq_entropy(uint64_t seed, int has_key, uint64_t key, uint32_t* ent) {
  int n = words32(seed, ent);
  if (has_key) {
    while (n < SS_POOL) ent[n++] = 0;  /* run entropy padded to the pool size */
    n += words32(key, ent + n);
  }
  return n;
}

static void seed_words64(uint64_t seed, int has_key, uint64_t key, uint64_t* w, int k) {
  uint32_t ent[8], o[16];
  int n = or_seedseq_entropy(seed, has_key, key, ent);
  or_seedseq_generate(ent, n, o, 2 * k);
  for (int i = 0; i < k; ++i) w[i] = (uint64_t)o[2 * i] | ((uint64_t)o[2 * i + 1] << 32);
}

/* ======================================================================
 * Engines (Sec. 2.2, Table "engines")
 * ==================================================================== */
static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

/* The GF(2)-linear transition shared by xoshiro256++ and xoshiro256**
 * (Blackman & Vigna 2018; Table "engines"): the two engines differ only in
 * the scrambler applied to the state before the step. */
static void xoshiro_step(uint64_t s[4]) {
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
}

/* xoshiro256++: the "++" scrambler, rotl(s0 + s3, 23) + s0, of the current
 * state, then the transition.  Parity unpinned for the scrambler (see
 * rp_oracle.h). */
static uint64_t xoshiro_next(uint64_t s[4]) {
  uint64_t out = rotl64(s[0] + s[3], 23) + s[0];
  xoshiro_step(s);
  return out;
}

/* xoshiro256**: the "**" scrambler, rotl(5 s1, 7) 9, of the current state,
 * then the same transition. */
static uint64_t xoshiro_ss_next(uint64_t s[4]) {
  uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
  xoshiro_step(s);
  return out;
}

/* PCG64-DXSM (O'Neill 2019): 128-bit LCG with the 64-bit "cheap" multiplier;
 * the DXSM output is taken from the state before the step. */
#define PCG_CHEAP_MULT 0xda942042e4dd58b5ull
static inline u128 pcg_state(const uint64_t s[4]) { return ((u128)s[0] << 64) | s[1]; }
static inline u128 pcg_inc(const uint64_t s[4]) { return ((u128)s[2] << 64) | s[3]; }
static inline void pcg_put(uint64_t s[4], u128 st) { s[0] = (uint64_t)(st >> 64); s[1] = (uint64_t)st; }

static uint64_t pcg_next(uint64_t s[4]) {
  uint64_t hi = s[0], lo = s[1] | 1u;
  hi ^= hi >> 32;
  hi *= PCG_CHEAP_MULT;
  hi ^= hi >> 48;
  hi *= lo;
  pcg_put(s, pcg_state(s) * (u128)PCG_CHEAP_MULT + pcg_inc(s));
  return hi;
}

/* Arbitrary-stride LCG advance (Brown 1994): the affine map x -> a x + c
 * raised to the power delta by square-and-multiply. */
void or_pcg_advance(uint64_t s[4], uint64_t d_hi, uint64_t d_lo) {
  u128 delta = ((u128)d_hi << 64) | d_lo;
  u128 cur_a = PCG_CHEAP_MULT, cur_c = pcg_inc(s), acc_a = 1, acc_c = 0;
  while (delta) {
    if (delta & 1) {
      acc_a *= cur_a;
      acc_c = acc_c * cur_a + cur_c;
    }
    cur_c = (cur_a + 1) * cur_c;
    cur_a *= cur_a;
    delta >>= 1;
  }
  pcg_put(s, acc_a * pcg_state(s) + acc_c);
}

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011): ten rounds of two
 * 32x32->64 multiplies with a Weyl-sequence key schedule. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    uint64_t p0 = (uint64_t)PHILOX_M0 * x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Word p of a Philox stream = half (p & 1) of block (counter + p/2); the four
 * 32-bit outputs x0..x3 of a block give words x0 | x1<<32 and x2 | x3<<32
 * (reading: the paper's Philox is 4x64; the packing of 4x32 is ours). */
static uint64_t philox_word(or_gen* g, uint64_t p) {
  uint64_t b = p >> 1;
  if (!g->blk_valid || g->blk_idx != b) {
    u128 c = (((u128)g->s[1] << 64) | g->s[0]) + (u128)b;
    uint32_t ctr[4] = {(uint32_t)c, (uint32_t)(c >> 32), (uint32_t)(c >> 64), (uint32_t)(c >> 96)};
    uint32_t key[2] = {(uint32_t)g->s[2], (uint32_t)(g->s[2] >> 32)};
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    g->blk[0] = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
    g->blk[1] = (uint64_t)o[2] | ((uint64_t)o[3] << 32);
    g->blk_idx = b;
    g->blk_valid = 1;
  }
  return g->blk[p & 1];
}

/* Philox4x64-10 (the paper's Philox; Salmon, Moraes, Dror & Shaw 2011):
 * ten rounds of two 64x64->128 multiplies with a Weyl-sequence key
 * schedule; a block gives four 64-bit words. */
#define PHILOX64_M0 0xD2E7470EE14C6C93ull
#define PHILOX64_M1 0xCA5A826395121157ull
#define PHILOX64_W0 0x9E3779B97F4A7C15ull
#define PHILOX64_W1 0xBB67AE8584CAA73Bull

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += PHILOX64_W0; k1 += PHILOX64_W1; }
    u128 p0 = (u128)PHILOX64_M0 * x0;
    u128 p1 = (u128)PHILOX64_M1 * x2;
    uint64_t y0 = (uint64_t)(p1 >> 64) ^ x1 ^ k0;
    uint64_t y1 = (uint64_t)p1;
    uint64_t y2 = (uint64_t)(p0 >> 64) ^ x3 ^ k1;
    uint64_t y3 = (uint64_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Word p of a Philox4x64 stream = word p mod 4 of block (counter + 1 +
 * p / 4): the counter is incremented before each block, as NumPy's Philox
 * does (the seeded counter itself is never a block). */
static uint64_t philox64_word(or_gen* g, uint64_t p) {
  uint64_t b = p >> 2;
  if (!g->blk_valid || g->blk_idx != b) {
    u128 c = (((u128)g->s[1] << 64) | g->s[0]) + (u128)b + 1u;
    uint64_t ctr[4] = {(uint64_t)c, (uint64_t)(c >> 64), 0, 0};
    uint64_t key[2] = {g->s[2], g->s[3]};
    or_philox4x64_10(ctr, key, g->blk);
    g->blk_idx = b;
    g->blk_valid = 1;
  }
  return g->blk[p & 3];
}

uint64_t or_next(or_gen* g) {
  uint64_t w;
  switch (g->engine) {
    case OR_XOSHIRO256PP: w = xoshiro_next(g->s); break;
    case OR_XOSHIRO256SS: w = xoshiro_ss_next(g->s); break;
    case OR_PCG64DXSM: w = pcg_next(g->s); break;
    case OR_PHILOX4X64_10: w = philox64_word(g, g->pos); break;
    default: w = philox_word(g, g->pos); break;
  }
  g->pos++;
  return w;
}

void or_gen_set(or_gen* g, int engine, const uint64_t s[4]) {
  memset(g, 0, sizeof(*g));
  g->engine = engine;
  memcpy(g->s, s, sizeof(g->s));
}

int or_gen_seed(or_gen* g, int engine, uint64_t seed, int has_key, uint64_t key) {
  uint64_t w[4] = {0, 0, 0, 0};
  memset(g, 0, sizeof(*g));
  g->engine = engine;
  if (engine == OR_XOSHIRO256PP || engine == OR_XOSHIRO256SS) {
    /* both xoshiro engines: four seed-sequence words, as the state */
    seed_words64(seed, has_key, key, w, 4);
    memcpy(g->s, w, sizeof(w));
    if ((w[0] | w[1] | w[2] | w[3]) == 0) return -1;
  } else if (engine == OR_PCG64DXSM) {
    /* NumPy-compatible PCG64DXSM seeding (O'Neill's set-sequence seeding):
     * initstate = w0:w1, initseq = w2:w3, inc = initseq<<1 | 1,
     * state = step(step(0) + initstate), where the two seeding steps use the
     * 128-bit PCG multiplier; generation then uses the cheap multiplier. */
    seed_words64(seed, has_key, key, w, 4);
    const u128 mult128 = ((u128)0x2360ED051FC65DA4ull << 64) | 0x4385DF649FCCF645ull;
    u128 initstate = ((u128)w[0] << 64) | w[1];
    u128 initseq = ((u128)w[2] << 64) | w[3];
    u128 inc = (initseq << 1) | 1u;
    u128 st = inc;             /* step from state 0 */
    st += initstate;
    st = st * mult128 + inc;
    pcg_put(g->s, st);
    g->s[2] = (uint64_t)(inc >> 64);
    g->s[3] = (uint64_t)inc;
  } else if (engine == OR_PHILOX4X64_10) {
    /* NumPy's Philox seeding: key = two words of the seed sequence, counter 0 */
    seed_words64(seed, has_key, key, w, 2);
    g->s[0] = 0;
    g->s[1] = 0;
    g->s[2] = w[0];
    g->s[3] = w[1];
  } else {
    /* Philox: every state word is seeded (Table "stream-select": counter +
     * key).  Reading for 4x32: w0 = counter low, w1 = counter high, w2 = key. */
    seed_words64(seed, has_key, key, w, 3);
    g->s[0] = w[0];
    g->s[1] = w[1];
    g->s[2] = w[2];
  }
  return 0;
}

/* ---------------- xoshiro jumps over GF(2) (Sec. 4.4) ---------------- */
typedef struct { uint64_t w[5]; } poly257;   /* up to degree 256 */

static int poly_deg(const uint64_t* p, int nw) {
  for (int i = nw - 1; i >= 0; --i)
    if (p[i]) return 64 * i + 63 - __builtin_clzll(p[i]);
  return -1;
}

/* Berlekamp-Massey over GF(2) on bit 0 of s[0] along 512 steps from a fixed
 * non-zero state: returns the minimal polynomial of the output sequence,
 * which for xoshiro256 is the degree-256 characteristic polynomial of T. */
static uint64_t g_charpoly[5];
static int g_charpoly_ready = 0;

void or_xoshiro_charpoly(uint64_t out[5]) {
  if (!g_charpoly_ready) {
    enum { NB = 512 };
    uint8_t seq[NB];
    uint64_t s[4] = {0x0123456789abcdefull, 0xfedcba9876543210ull, 0x0f1e2d3c4b5a6978ull, 0x8796a5b4c3d2e1f0ull};
    for (int i = 0; i < NB; ++i) { seq[i] = (uint8_t)(s[0] & 1); xoshiro_step(s); }
    /* connection polynomial C(x) = 1 + c1 x + ... ; sequence satisfies
     * sum_{j=0..L} c_j a_{n-j} = 0 */
    uint8_t C[NB + 1] = {0}, B[NB + 1] = {0}, T[NB + 1];
    C[0] = B[0] = 1;
    int L = 0, m = 1;
    for (int n = 0; n < NB; ++n) {
      int d = seq[n];
      for (int j = 1; j <= L; ++j) d ^= C[j] & seq[n - j];
      if (d) {
        memcpy(T, C, sizeof(T));
        for (int j = 0; j + m <= NB; ++j) C[j + m] ^= B[j];
        if (2 * L <= n) { L = n + 1 - L; memcpy(B, T, sizeof(B)); m = 1; }
        else ++m;
      } else {
        ++m;
      }
    }
    /* characteristic polynomial p(x) = x^L C(1/x): coefficient of x^(L-j) is c_j */
    memset(g_charpoly, 0, sizeof(g_charpoly));
    for (int j = 0; j <= L; ++j)
      if (C[j]) g_charpoly[(L - j) >> 6] |= 1ull << ((L - j) & 63);
    g_charpoly_ready = 1;
  }
  memcpy(out, g_charpoly, sizeof(g_charpoly));
}

/* r = a*b mod p, polynomials over GF(2) of degree < 256, p of degree 256 */
static void polymulmod(const uint64_t a[4], const uint64_t b[4], const uint64_t p[5], uint64_t r[4]) {
  uint64_t prod[9] = {0};
  for (int i = 0; i < 256; ++i) {
    if ((a[i >> 6] >> (i & 63)) & 1) {
      /* prod ^= b << i */
      int ws = i >> 6, bs = i & 63;
      for (int k = 0; k < 4; ++k) {
        prod[k + ws] ^= b[k] << bs;
        if (bs) prod[k + ws + 1] ^= b[k] >> (64 - bs);
      }
    }
  }
  for (int deg = 510; deg >= 256; --deg) {
    if ((prod[deg >> 6] >> (deg & 63)) & 1) {
      int sh = deg - 256, ws = sh >> 6, bs = sh & 63;
      for (int k = 0; k < 5; ++k) {
        if (k + ws < 9) prod[k + ws] ^= p[k] << bs;
        if (bs && k + ws + 1 < 9) prod[k + ws + 1] ^= p[k] >> (64 - bs);
      }
    }
  }
  memcpy(r, prod, 4 * sizeof(uint64_t));
}

void or_xoshiro_jump_poly(uint64_t s[4], const uint64_t* nl, int nlimbs) {
  uint64_t p[5];
  or_xoshiro_charpoly(p);
  /* q = x^N mod p by right-to-left square-and-multiply */
  uint64_t q[4] = {1, 0, 0, 0}, base[4] = {2, 0, 0, 0};
  int top = poly_deg(nl, nlimbs);
  for (int bit = 0; bit <= top; ++bit) {
    if ((nl[bit >> 6] >> (bit & 63)) & 1) polymulmod(q, base, p, q);
    polymulmod(base, base, p, base);
  }
  /* T^N s = q(T) s = sum_k q_k T^k s */
  uint64_t acc[4] = {0, 0, 0, 0}, cur[4];
  memcpy(cur, s, sizeof(cur));
  for (int k = 0; k < 256; ++k) {
    if ((q[k >> 6] >> (k & 63)) & 1)
      for (int j = 0; j < 4; ++j) acc[j] ^= cur[j];
    xoshiro_step(cur);
  }
  memcpy(s, acc, sizeof(acc));
}

/* 256x256 GF(2) matrices stored by column: col[j] = T e_j as 4 words */
typedef struct { uint64_t col[256][4]; } gf2mat;

static void mat_apply(const gf2mat* M, const uint64_t v[4], uint64_t r[4]) {
  uint64_t a[4] = {0, 0, 0, 0};
  for (int j = 0; j < 256; ++j)
    if ((v[j >> 6] >> (j & 63)) & 1)
      for (int k = 0; k < 4; ++k) a[k] ^= M->col[j][k];
  memcpy(r, a, sizeof(a));
}

static void mat_mul(const gf2mat* A, const gf2mat* B, gf2mat* C) {  /* C = A B */
  gf2mat tmp;
  for (int j = 0; j < 256; ++j) mat_apply(A, B->col[j], tmp.col[j]);
  *C = tmp;
}

void or_xoshiro_jump_matrix(uint64_t s[4], const uint64_t* nl, int nlimbs) {
  gf2mat* M = (gf2mat*)malloc(sizeof(gf2mat));
  for (int j = 0; j < 256; ++j) {
    uint64_t e[4] = {0, 0, 0, 0};
    e[j >> 6] = 1ull << (j & 63);
    xoshiro_step(e);
    memcpy(M->col[j], e, sizeof(e));
  }
  uint64_t v[4];
  memcpy(v, s, sizeof(v));
  int top = poly_deg(nl, nlimbs);
  for (int bit = 0; bit <= top; ++bit) {
    if ((nl[bit >> 6] >> (bit & 63)) & 1) mat_apply(M, v, v);
    if (bit < top) mat_mul(M, M, M);
  }
  memcpy(s, v, sizeof(v));
  free(M);
}

void or_jump(or_gen* g, uint64_t n_hi, uint64_t n_lo) {
  if (g->engine == OR_XOSHIRO256PP || g->engine == OR_XOSHIRO256SS) {
    uint64_t nl[2] = {n_lo, n_hi};
    or_xoshiro_jump_poly(g->s, nl, 2);
  } else if (g->engine == OR_PCG64DXSM) {
    or_pcg_advance(g->s, n_hi, n_lo);
  }
  g->pos += n_lo;  /* Philox words are addressed by pos directly */
}

void or_seek(or_gen* g, uint64_t pos) {
  /* from the current position to `pos` (forward, modulo 2^64) */
  uint64_t d = pos - g->pos;
  if (d) or_jump(g, 0, d);
}

void or_substream(or_gen* g, int engine, uint64_t base_seed, uint64_t s) {
  or_gen_seed(g, engine, base_seed, 0, 0);
  if (engine == OR_XOSHIRO256PP || engine == OR_XOSHIRO256SS) {
    /* stream s = base jumped s times by 2^128 (Sec. 2.3, duplicate-and-jump) */
    uint64_t nl[3] = {0, 0, s};
    if (s) or_xoshiro_jump_poly(g->s, nl, 3);
  } else if (engine == OR_PHILOX4X32_10) {
    g->s[2] = s;  /* key := s (stream setter) */
  } else if (engine == OR_PHILOX4X64_10) {
    g->s[2] = s;  /* key word 0 := s (stream setter); key word 1 stays seeded */
  } else {
    /* PCG64: stream selector = increment; inc := 2 s + 1 */
    g->s[2] = (uint64_t)((((u128)s << 1) | 1u) >> 64);
    g->s[3] = (uint64_t)((((u128)s << 1) | 1u));
  }
  g->pos = 0;
  g->blk_valid = 0;
}

/* ======================================================================
 * Double-double arithmetic and correctly rounded exp / log (Sec. 4.2:
 * accept tests must not depend on the platform's libm).  Dekker/Knuth
 * error-free transformations; exp by ln2 reduction, 2^-10 scaling, Taylor
 * series and ten squarings; log by one Newton step on exp.
 * ==================================================================== */
typedef struct { double hi, lo; } dd;

static inline dd two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  dd r = {s, (a - (s - bb)) + (b - bb)};
  return r;
}
static inline dd fast_two_sum(double a, double b) {
  double s = a + b;
  dd r = {s, b - (s - a)};
  return r;
}
static inline dd two_prod(double a, double b) {
  double p = a * b;
  dd r = {p, fma(a, b, -p)};
  return r;
}
static inline dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
static inline dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return fast_two_sum(p.hi, p.lo);
}
static inline dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return fast_two_sum(p.hi, p.lo);
}
static inline dd dd_div_d(dd a, double b) {
  double q1 = a.hi / b;
  dd p = two_prod(q1, b);
  double r = ((a.hi - p.hi) - p.lo + a.lo) / b;
  return fast_two_sum(q1, r);
}

/* ln 2 = LN2_HI + LN2_LO + O(2^-110) (checked against mpmath in the tests) */
static const double LN2_HI = 0x1.62e42fefa39efp-1;
static const double LN2_LO = 0x1.abc9e3b39803fp-56;

static dd dd_exp(double x) {
  double k = nearbyint(x / LN2_HI);
  dd a = two_prod(k, LN2_HI), b = two_prod(k, LN2_LO);
  dd r = dd_add((dd){x, 0.0}, (dd){-a.hi, -a.lo});
  r = dd_add(r, (dd){-b.hi, -b.lo});
  r.hi = ldexp(r.hi, -10);
  r.lo = ldexp(r.lo, -10);
  /* Taylor: 1 + s(1 + s/2(1 + s/3(...))) to degree 10; |s| < 3.4e-4 */
  dd p = {1.0, 0.0};
  for (int j = 10; j >= 1; --j) {
    p = dd_div_d(dd_mul(r, p), (double)j);
    p = dd_add((dd){1.0, 0.0}, p);
  }
  for (int j = 0; j < 10; ++j) p = dd_mul(p, p);
  p.hi = ldexp(p.hi, (int)k);
  p.lo = ldexp(p.lo, (int)k);
  return p;
}

static dd dd_log(double y) {
  if (y > 0.9375 && y < 1.0625) {
    /* near 1 the Newton step below is accurate only to ~2^-100 absolute,
     * not relative: sum the series log(1 + r) = r - r^2/2 + r^3/3 - ...
     * with r = y - 1 exact (Sterbenz), |r| < 2^-4, until the terms fall
     * below 2^-112 |r| */
    dd r = {y - 1.0, 0.0};
    dd pk = r, sum = r;
    for (int k = 2; k < 60; ++k) {
      pk = dd_mul(pk, r);
      dd term = dd_div_d(pk, (double)k);
      if (k % 2 == 0) term = (dd){-term.hi, -term.lo};
      sum = dd_add(sum, term);
      if (fabs(term.hi) < ldexp(fabs(r.hi), -112)) break;
    }
    return sum;
  }
  double y0 = log(y);
  dd t = dd_exp(-y0);
  dd z = dd_mul_d(t, y);
  z = dd_add(z, (dd){-1.0, 0.0});              /* z = y e^{-y0} - 1, |z| ~ 1e-16 */
  dd zz = dd_mul(z, z);
  z = dd_add(z, (dd){-0.5 * zz.hi, -0.5 * zz.lo}); /* log(1+z) = z - z^2/2 + O(z^3) */
  return dd_add((dd){y0, 0.0}, z);
}

static uint64_t g_ambiguous = 0;
uint64_t or_cr_ambiguous(void) { return g_ambiguous; }
void or_cr_reset(void) { g_ambiguous = 0; }

/* Round a double-double value (relative error <= 2^-90) to the nearest double,
 * counting cases where a rounding boundary lies within the error bound. */
static double dd_round(dd v) {
  double hi = v.hi, lo = v.lo;
  if (!isfinite(hi) || hi == 0.0) return hi;
  double up = nextafter(hi, INFINITY) - hi, dn = hi - nextafter(hi, -INFINITY);
  double tol = ldexp(fabs(hi), -90);
  if (fabs(lo - 0.5 * up) <= tol || fabs(lo + 0.5 * dn) <= tol) g_ambiguous++;
  /* v is normalised (hi = RN(hi + lo)), so hi is already RN(v) */
  return hi;
}

double or_cr_exp(double x) {
  if (x != x) return x;
  if (x > 709.0) return INFINITY;
  if (x < -745.0) return 0.0;
  if (x == 0.0) return 1.0;
  if (x < -708.0) return exp(x);  /* subnormal results: not used by the samplers */
  return dd_round(dd_exp(x));
}

double or_cr_log(double x) {
  if (x != x || x < 0.0) return NAN;
  if (x == 0.0) return -INFINITY;
  if (x == 1.0) return 0.0;
  if (isinf(x)) return x;
  return dd_round(dd_log(x));
}

/* ======================================================================
 * Distributions (Sec. 3)
 * ==================================================================== */
/* 53-bit uniform in [0,1): floor(u / 2^11) * 2^-53 (Sec. 3.1, method 1) */
static inline double u53(uint64_t u) { return (double)(u >> 11) * 0x1.0p-53; }

void or_fill_u64(or_gen* g, size_t n, uint64_t* out) {
  for (size_t i = 0; i < n; ++i) out[i] = or_next(g);
}

void or_fill_uniform(or_gen* g, size_t n, double* out) {
  for (size_t i = 0; i < n; ++i) out[i] = u53(or_next(g));
}

/* 52-bit uniform, the paper's default (Sec. 3.1, method 2): the word's top
 * 52 bits as the fraction of a double in [1, 2), minus 1; exactly
 * floor(u / 2^12) 2^-52. */
void or_fill_uniform52(or_gen* g, size_t n, double* out) {
  for (size_t i = 0; i < n; ++i) {
    uint64_t bits = (or_next(g) >> 12) | 0x3ff0000000000000ull;
    double x;
    memcpy(&x, &bits, 8);
    out[i] = x - 1.0;
  }
}

/* Bounded integers in [0, m) by Lemire's multiply-and-reject (Sec. 3.2):
 * p = u m (128-bit); reject while low(p) < 2^64 mod m; return high(p).
 * m = 0 means the full 64-bit range (Table "discrete", b = 0).  Reading: one
 * 64-bit word per attempt for every m. */
void or_fill_bounded(or_gen* g, size_t n, uint64_t m, uint64_t* out, uint64_t* start) {
  if (m == 0) {
    for (size_t i = 0; i < n; ++i) {
      if (start) start[i] = g->pos;
      out[i] = or_next(g);
    }
    return;
  }
  uint64_t t = (0 - m) % m;  /* (2^64 - m) mod m = 2^64 mod m */
  for (size_t i = 0; i < n; ++i) {
    for (;;) {
      uint64_t p0 = g->pos;
      u128 p = (u128)or_next(g) * m;
      if ((uint64_t)p >= t) {
        out[i] = (uint64_t)(p >> 64);
        if (start) start[i] = p0;
        break;
      }
    }
  }
}

/* ---- ziggurat (Sec. 3.1 and the ziggurat figure) ----
 * Normal word layout: bits 0-7 strip i, bit 8 sign, bits 9-60 magnitude r
 * (52 bits), x = RN(r * w_i).  Exponential: bits 0-7 strip, bits 8-60 r
 * (53 bits).  High three bits unused.  Fast accept when r < k_i.  Strip 0
 * falls to the tail, other strips to the wedge test y < f(x) with
 * y = f_i + U (f_{i-1} - f_i).  The McFarland-type tangent/secant shortcuts
 * only skip exp evaluations and never change a decision, so the oracle
 * always evaluates f(x) (correctly rounded) in the wedge. */
static uint64_t g_zc[4];
void or_zig_counts(uint64_t c[4]) { memcpy(c, g_zc, sizeof(g_zc)); }

int or_zig_table(int which, int i, uint64_t* k, double* w, double* f) {
  if (i < 0 || i > 255) return -1;
  if (which == 0) { *k = OR_ZN_K[i]; *w = OR_ZN_W[i]; *f = OR_ZN_F[i]; }
  else { *k = OR_ZE_K[i]; *w = OR_ZE_W[i]; *f = OR_ZE_F[i]; }
  return 0;
}
double or_zig_R(int which) { return which == 0 ? OR_ZN_R : OR_ZE_R; }

double or_zig_normal_x(uint64_t u) {
  int i = (int)(u & 0xff);
  uint64_t r = (u >> 9) & ((1ull << 52) - 1);
  double x = (double)r * OR_ZN_W[i];
  return ((u >> 8) & 1) ? -x : x;
}

static double normal_one(or_gen* g, uint64_t* start) {
  for (;;) {
    uint64_t p0 = g->pos;
    uint64_t u = or_next(g);
    int i = (int)(u & 0xff);
    int neg = (int)((u >> 8) & 1);
    uint64_t r = (u >> 9) & ((1ull << 52) - 1);
    double x = (double)r * OR_ZN_W[i];
    if (neg) x = -x;
    if (r < OR_ZN_K[i]) { g_zc[0]++; if (start) *start = p0; return x; }
    if (i == 0) {
      /* tail beyond R (Marsaglia 1964): a = -log(1-U1)/R, b = -log(1-U2),
       * accept when 2b > a^2; the value is R + a with the word's sign.
       * Reading: U1 then U2, both 53-bit, 1-U exact so log1p(-U) = log(1-U). */
      g_zc[3]++;
      for (;;) {
        double U1 = u53(or_next(g)), U2 = u53(or_next(g));
        double a = -or_cr_log(1.0 - U1) / OR_ZN_R;
        double b = -or_cr_log(1.0 - U2);
        if (b + b > a * a) {
          double v = OR_ZN_R + a;
          if (start) *start = p0;
          return neg ? -v : v;
        }
      }
    }
    g_zc[1]++;
    double U = u53(or_next(g));
    double y = (OR_ZN_F[i - 1] - OR_ZN_F[i]) * U + OR_ZN_F[i];
    double t = -0.5 * (x * x);
    if (y < or_cr_exp(t)) { if (start) *start = p0; return x; }
    g_zc[2]++;
  }
}

void or_fill_normal(or_gen* g, size_t n, double* out, uint64_t* start) {
  memset(g_zc, 0, sizeof(g_zc));
  for (size_t i = 0; i < n; ++i) out[i] = normal_one(g, start ? start + i : NULL);
}

void or_fill_exp(or_gen* g, size_t n, double* out, uint64_t* start) {
  memset(g_zc, 0, sizeof(g_zc));
  for (size_t j = 0; j < n; ++j) {
    for (;;) {
      uint64_t p0 = g->pos;
      if (start) start[j] = p0;
      uint64_t u = or_next(g);
      int i = (int)(u & 0xff);
      uint64_t r = (u >> 8) & ((1ull << 53) - 1);
      double x = (double)r * OR_ZE_W[i];
      if (r < OR_ZE_K[i]) { g_zc[0]++; out[j] = x; break; }
      if (i == 0) {
        /* memoryless tail: R + Exp(1) = R - log(1 - U) */
        g_zc[3]++;
        out[j] = OR_ZE_R - or_cr_log(1.0 - u53(or_next(g)));
        break;
      }
      g_zc[1]++;
      double U = u53(or_next(g));
      double y = (OR_ZE_F[i - 1] - OR_ZE_F[i]) * U + OR_ZE_F[i];
      if (y < or_cr_exp(-x)) { out[j] = x; break; }
      g_zc[2]++;
    }
  }
}

/* ---- float variants (Table "continuous": the functions with suffix f;
 * Sec. 3.1: the engines' bit stream read as 32-bit words; Sec. 4.4: floats
 * save space and time).  Readings:
 * - 32-bit words: each 64-bit stream word gives its low half, then its high
 *   half.  A float fill starts at the low half of word pos.  When it ends
 *   on a low half, the high half is left unused, so the position after a
 *   float fill is the next whole word.
 * - uniformf: the paper's default method with a float: the top 23 bits of
 *   the 32-bit word in the fraction of a float in [1, 2), minus 1, which is
 *   exactly floor(h / 2^9) 2^-23.
 * - u24(h) = floor(h / 2^8) 2^-24 (method 1), the samplers' inner uniform.
 * - normalf: bits 0-7 strip i, bit 8 sign, bits 9-31 r (23 bits).
 *   x = RN_f(r w_i), with w_i = RN_f(2^29 W_i) from the double table's
 *   W_i = x_i 2^-52.  Fast accept when r < k_i / 2^29 (integer division:
 *   floor(2^23 x_{i-1} / x_i)).  The wedge takes y = RN_f((f_{i-1} - f_i) U + f_i)
 *   in float operations, with f_i = RN_f(F_i) and U = u24 of the next word,
 *   and accepts when y < exp(-x^2 / 2), decided in double (x^2 is exact
 *   there) against the correctly rounded exp.  The tail is the double
 *   sampler's with U1, U2 = u24 of the next two words, in double, and the
 *   value RN_f(R + a).
 * - expf: bits 0-7 strip, bits 8-31 r (24 bits); w_i = RN_f(2^29 W_i) with
 *   W_i = x_i 2^-53; fast r < k_i / 2^29; wedge against exp(-x) as above;
 *   tail RN_f(R - log(1 - U)). */
typedef struct { or_gen* g; uint64_t w; int hi; } half_reader;

static uint32_t next32(half_reader* h) {
  if (h->hi) { h->hi = 0; return (uint32_t)(h->w >> 32); }
  h->w = or_next(h->g);
  h->hi = 1;
  return (uint32_t)h->w;
}
/* 32-bit word index (2 * word + half) of the next 32-bit word */
static uint64_t half_pos(const half_reader* h) { return h->hi ? 2 * h->g->pos - 1 : 2 * h->g->pos; }

static inline double u24(uint32_t h) { return (double)(h >> 8) * 0x1.0p-24; }

void or_fill_uniformf(or_gen* g, size_t n, float* out) {
  half_reader h = {g, 0, 0};
  for (size_t i = 0; i < n; ++i) {
    uint32_t bits = (next32(&h) >> 9) | 0x3f800000u;
    float x;
    memcpy(&x, &bits, 4);
    out[i] = x - 1.0f;
  }
}

/* float tables from the double ones: which 0 normal, 1 exponential */
int or_zig_table_f(int which, int i, uint32_t* k, float* w, float* f) {
  if (i < 0 || i > 255) return -1;
  const uint64_t* K = which ? OR_ZE_K : OR_ZN_K;
  const double* W = which ? OR_ZE_W : OR_ZN_W;
  const double* F = which ? OR_ZE_F : OR_ZN_F;
  *k = (uint32_t)(K[i] >> 29);
  *w = (float)(W[i] * 0x1.0p29);
  *f = (float)F[i];
  return 0;
}

void or_fill_normalf(or_gen* g, size_t n, float* out, uint64_t* start) {
  half_reader h = {g, 0, 0};
  memset(g_zc, 0, sizeof(g_zc));
  for (size_t j = 0; j < n; ++j) {
    for (;;) {
      uint64_t p0 = half_pos(&h);
      uint32_t u = next32(&h);
      int i = (int)(u & 0xff);
      int neg = (int)((u >> 8) & 1);
      uint32_t r = u >> 9;
      uint32_t ki; float wi, fi;
      or_zig_table_f(0, i, &ki, &wi, &fi);
      float x = (float)r * wi;
      if (neg) x = -x;
      if (r < ki) { g_zc[0]++; if (start) start[j] = p0; out[j] = x; break; }
      if (i == 0) {
        g_zc[3]++;
        double a, b;
        do {
          double U1 = u24(next32(&h)), U2 = u24(next32(&h));
          a = -or_cr_log(1.0 - U1) / OR_ZN_R;
          b = -or_cr_log(1.0 - U2);
        } while (!(b + b > a * a));
        float v = (float)(OR_ZN_R + a);
        if (start) start[j] = p0;
        out[j] = neg ? -v : v;
        break;
      }
      g_zc[1]++;
      uint32_t k1; float w1, f1;
      or_zig_table_f(0, i - 1, &k1, &w1, &f1);
      float U = (float)u24(next32(&h));
      float y = (f1 - fi) * U + fi;
      double xd = (double)x;
      if ((double)y < or_cr_exp(-0.5 * (xd * xd))) { if (start) start[j] = p0; out[j] = x; break; }
      g_zc[2]++;
    }
  }
}

void or_fill_expf(or_gen* g, size_t n, float* out, uint64_t* start) {
  half_reader h = {g, 0, 0};
  memset(g_zc, 0, sizeof(g_zc));
  for (size_t j = 0; j < n; ++j) {
    for (;;) {
      uint64_t p0 = half_pos(&h);
      uint32_t u = next32(&h);
      int i = (int)(u & 0xff);
      uint32_t r = u >> 8;
      uint32_t ki; float wi, fi;
      or_zig_table_f(1, i, &ki, &wi, &fi);
      float x = (float)r * wi;
      if (r < ki) { g_zc[0]++; if (start) start[j] = p0; out[j] = x; break; }
      if (i == 0) {
        g_zc[3]++;
        if (start) start[j] = p0;
        out[j] = (float)(OR_ZE_R - or_cr_log(1.0 - u24(next32(&h))));
        break;
      }
      g_zc[1]++;
      uint32_t k1; float w1, f1;
      or_zig_table_f(1, i - 1, &k1, &w1, &f1);
      float U = (float)u24(next32(&h));
      float y = (f1 - fi) * U + fi;
      if ((double)y < or_cr_exp(-(double)x)) { if (start) start[j] = p0; out[j] = x; break; }
      g_zc[2]++;
    }
  }
}

/* ---- gamma (Marsaglia & Tsang 2000; Sec. 3.1 "Gamma and related") ----
 * alpha >= 1: d = alpha - 1/3, c = 1/sqrt(9d); repeat: x ~ N(0,1) (ziggurat
 * above), v = 1 + c x; if v <= 0 draw again (no uniform consumed);
 * v = v^3, U ~ U53, accept d v if U < 1 - 0.0331 x^4 or
 * log U < x^2/2 + d (1 - v + log v).
 * alpha < 1 (reading): Gamma(alpha) = Gamma(alpha + 1) U^(1/alpha), the boost
 * uniform drawn after the accepted Gamma(alpha+1), evaluated as
 * exp(log(U)/alpha). */
typedef struct { double d, c; } mt_consts;

static mt_consts mt_setup(double a) {
  mt_consts k;
  k.d = a - 1.0 / 3.0;
  k.c = 1.0 / sqrt(9.0 * k.d);
  return k;
}

static double gamma_ge1(or_gen* g, mt_consts k, uint64_t* start) {
  int first = 1;
  for (;;) {
    uint64_t p0 = g->pos;
    double x = normal_one(g, NULL);
    if (first && start) *start = p0;
    first = 0;
    double v = 1.0 + k.c * x;
    if (v <= 0.0) continue;
    v = v * v * v;
    double U = u53(or_next(g));
    double x2 = x * x;
    if (U < 1.0 - 0.0331 * (x2 * x2)) { if (start) *start = p0; return k.d * v; }
    if (or_cr_log(U) < 0.5 * x2 + k.d * ((1.0 - v) + or_cr_log(v))) { if (start) *start = p0; return k.d * v; }
  }
}

static double gamma_one(or_gen* g, double alpha, mt_consts k, uint64_t* start) {
  if (alpha >= 1.0) return gamma_ge1(g, k, start);
  double y = gamma_ge1(g, k, start);
  double U = u53(or_next(g));
  return y * or_cr_exp(or_cr_log(U) / alpha);
}

int or_fill_gamma(or_gen* g, size_t n, double alpha, double* out, uint64_t* start) {
  if (!(alpha > 0.0)) return -1;
  mt_consts k = mt_setup(alpha >= 1.0 ? alpha : alpha + 1.0);
  for (size_t i = 0; i < n; ++i) out[i] = gamma_one(g, alpha, k, start ? start + i : NULL);
  return 0;
}

/* Beta(a, b) = X / (X + Y), X ~ Gamma(a) drawn before Y ~ Gamma(b) (Table
 * "continuous", beta). */
int or_fill_beta(or_gen* g, size_t n, double a, double b, double* out, uint64_t* start) {
  if (!(a > 0.0) || !(b > 0.0)) return -1;
  mt_consts ka = mt_setup(a >= 1.0 ? a : a + 1.0), kb = mt_setup(b >= 1.0 ? b : b + 1.0);
  for (size_t i = 0; i < n; ++i) {
    double X = gamma_one(g, a, ka, start ? start + i : NULL);
    double Y = gamma_one(g, b, kb, NULL);
    out[i] = X / (X + Y);
  }
  return 0;
}

/* ---- derived distributions (Table "continuous"; Sec. 3.1 "Gamma and
 * related distributions", "Extreme value and Weibull distributions") ----
 * Each is a transform of the base samplers above, in the stream order of
 * its draws.  Every arithmetic step is one IEEE operation in the order the
 * formula is written (no contraction); exp, log and pow are correctly
 * rounded.  Readings: unif = a + (b - a) u; normal = mu + sigma z;
 * lognormal = exp(mu + sigma z); Exp(beta) and Gamma(alpha, theta) scale by
 * beta and theta; chi2(nu) = 2 Gamma(nu / 2); Gumbel = mu - beta log(-log u)
 * with u = U53; Pareto = x_m exp(E / alpha); Weibull = lambda pow(E, 1 / k);
 * generalized Pareto from P = Pareto(1, 1 / |xi|) as the paper writes it;
 * F = (X / nu1) / (Y / nu2) with X ~ Gamma(nu1 / 2) drawn before
 * Y ~ Gamma(nu2 / 2); skew normal (Azzalini's representation) from two
 * consecutive normals u0, u1: z = delta |u0| + sqrt(1 - delta^2) u1,
 * delta = alpha / sqrt(1 + alpha^2), x = mu + sigma z; Student t =
 * Z / sqrt(V / nu) with Z ~ N(0, 1) drawn before V ~ chi2_nu. */

/* pow(x, y) for x > 0, correctly rounded: exp(y log x) in double-double */
double or_cr_pow(double x, double y) {
  if (x == 1.0 || y == 0.0) return 1.0;
  if (x == 0.0) return y > 0.0 ? 0.0 : INFINITY;
  if (isinf(x)) return y > 0.0 ? INFINITY : 0.0;
  dd t = dd_mul_d(dd_log(x), y);
  if (t.hi > 709.0) return INFINITY;
  if (t.hi < -708.0) return pow(x, y);   /* subnormal results: not reached by the samplers */
  dd e = dd_exp(t.hi);
  /* exp(hi + lo) = exp(hi) (1 + lo + lo^2 / 2 + ...), |lo| <= 2^-43 */
  dd c = two_sum(1.0, t.lo);
  c = dd_add(c, (dd){0.5 * t.lo * t.lo, 0.0});
  return dd_round(dd_mul(e, c));
}

static double derived_value(int kind, double x, const double* p) {
  switch (kind) {
    case OR_D_UNIF: return p[0] + (p[1] - p[0]) * x;
    case OR_D_NORMAL_MS: return p[0] + p[1] * x;
    case OR_D_LOGNORMAL: return or_cr_exp(p[0] + p[1] * x);
    case OR_D_EXP_SCALE: return p[0] * x;
    case OR_D_GAMMA_SCALE: return p[1] * x;
    case OR_D_CHI2: return 2.0 * x;
    case OR_D_GUMBEL: return p[0] - p[1] * or_cr_log(-or_cr_log(x));
    case OR_D_PARETO: return p[0] * or_cr_exp(x / p[1]);
    case OR_D_WEIBULL: return p[1] * or_cr_pow(x, 1.0 / p[0]);
    case OR_D_GPD: {
      double mu = p[0], sigma = p[1], xi = p[2];
      if (xi == 0.0) return mu + sigma * x;
      double P = 1.0 * or_cr_exp(x / (1.0 / fabs(xi)));
      if (xi > 0.0) return mu + sigma * (P - 1.0) / xi;
      return mu - sigma * (1.0 - 1.0 / P) / xi;
    }
    default: return NAN;
  }
}

int or_fill_derived(or_gen* g, int kind, size_t n, const double* p, double* out, uint64_t* start) {
  switch (kind) {
    case OR_D_UNIF:
    case OR_D_GUMBEL:
      or_fill_uniform(g, n, out);
      if (start) for (size_t i = 0; i < n; ++i) start[i] = g->pos - n + i;
      break;
    case OR_D_NORMAL_MS:
    case OR_D_LOGNORMAL:
      or_fill_normal(g, n, out, start);
      break;
    case OR_D_EXP_SCALE:
    case OR_D_PARETO:
    case OR_D_WEIBULL:
    case OR_D_GPD:
      or_fill_exp(g, n, out, start);
      break;
    case OR_D_GAMMA_SCALE:
      if (or_fill_gamma(g, n, p[0], out, start)) return -1;
      break;
    case OR_D_CHI2:
      if (or_fill_gamma(g, n, 0.5 * p[0], out, start)) return -1;
      break;
    case OR_D_F: {
      double a = 0.5 * p[0], b = 0.5 * p[1];
      if (!(a > 0.0) || !(b > 0.0)) return -1;
      mt_consts ka = mt_setup(a >= 1.0 ? a : a + 1.0), kb = mt_setup(b >= 1.0 ? b : b + 1.0);
      for (size_t i = 0; i < n; ++i) {
        double X = gamma_one(g, a, ka, start ? start + i : NULL);
        double Y = gamma_one(g, b, kb, NULL);
        out[i] = (X / p[0]) / (Y / p[1]);
      }
      return 0;
    }
    case OR_D_T: {
      /* Z / sqrt(V / nu), Z ~ N(0, 1) drawn before V ~ chi2_nu = 2 Gamma(nu / 2) */
      double a = 0.5 * p[0];
      if (!(a > 0.0)) return -1;
      mt_consts k = mt_setup(a >= 1.0 ? a : a + 1.0);
      for (size_t i = 0; i < n; ++i) {
        double z = normal_one(g, start ? start + i : NULL);
        double v = 2.0 * gamma_one(g, a, k, NULL);
        out[i] = z / sqrt(v / p[0]);
      }
      return 0;
    }
    case OR_D_SKEW_NORMAL: {
      double al = p[2];
      double delta = al / sqrt(1.0 + al * al);
      double omega = sqrt(1.0 - delta * delta);
      for (size_t i = 0; i < n; ++i) {
        double u[2];
        or_fill_normal(g, 1, &u[0], start ? start + i : NULL);
        or_fill_normal(g, 1, &u[1], NULL);
        double z = delta * fabs(u[0]) + omega * u[1];
        out[i] = p[0] + p[1] * z;
      }
      return 0;
    }
    default:
      return -1;
  }
  for (size_t i = 0; i < n; ++i) out[i] = derived_value(kind, out[i], p);
  return 0;
}

/* ======================================================================
 * Pathwise gradients.  For z ~ F(.; theta) drawn as z = F^{-1}(u; theta),
 * dz/dtheta = -(dF/dtheta)(z) / f(z).  Written as integrals whose integrand
 * has one sign (no cancellation), evaluated by adaptive tanh-sinh /
 * exp-sinh quadrature (Takahasi & Mori 1974).
 * ==================================================================== */
double or_digamma(double x) {
  /* recurrence psi(x) = psi(x+1) - 1/x up to x >= 12, then the asymptotic
   * series with Bernoulli numbers B2..B14 */
  double acc = 0.0;
  while (x < 12.0) { acc -= 1.0 / x; x += 1.0; }
  double r = 1.0 / (x * x);
  double s = r * (1.0 / 12 - r * (1.0 / 120 - r * (1.0 / 252 - r * (1.0 / 240 - r * (1.0 / 132 - r * (691.0 / 32760 - r * (1.0 / 12)))))));
  return acc + log(x) - 0.5 / x - s;
}

typedef double (*ifun)(double, void*);

/* tanh-sinh on (0,1) for g(u) given u and 1-u separately (no cancellation
 * at the right end).  Level refinement until two levels agree. */
typedef double (*ifun01)(double u, double um, void* ctx);

static double ts01(ifun01 f, void* ctx) {
  const double hpi = 1.5707963267948966;
  double h = 1.0, prev = 0.0, sum = 0.0;
  /* level 0: all nodes with step 1 */
  for (int lev = 0; lev < 12; ++lev) {
    double add = 0.0;
    int step = lev == 0 ? 1 : 2;
    int kstart = lev == 0 ? 0 : 1;
    for (int k = kstart;; k += step) {
      double t = k * h;
      double sh = hpi * sinh(t), ch = cosh(sh);
      double w = hpi * cosh(t) / (ch * ch);
      /* u = (1 + tanh(sh))/2 ; 1 - u = e^{-sh}/(2 ch) ; u for -t: 1/(1+e^{2 sh}) */
      double e2 = exp(-2.0 * sh);
      double um = e2 / (1.0 + e2);     /* 1 - u at +t, u at -t */
      double up = 1.0 / (1.0 + e2);    /* u at +t */
      if (um < 1e-300 || w < 1e-300) break;
      double v = 0.5 * w * (f(up, um, ctx) + (k == 0 ? 0.0 : f(um, up, ctx)));
      add += v;
      if (k > 0 && fabs(v) < 1e-20 * fabs(add + sum) && t > 3.0) break;
    }
    sum += add;                   /* all nodes at the current spacing h */
    double est = sum * h;
    if (lev > 3 && fabs(est - prev) <= 1e-15 * fabs(est)) return est;
    prev = est;
    h *= 0.5;
  }
  return prev;
}

/* exp-sinh on (0, inf) */
static double es0inf(ifun f, void* ctx) {
  const double hpi = 1.5707963267948966;
  double h = 1.0, prev = 0.0, sum = 0.0;
  for (int lev = 0; lev < 12; ++lev) {
    double add = 0.0;
    int step = lev == 0 ? 1 : 2;
    int kstart = lev == 0 ? 0 : 1;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      for (int k = (sgn < 0 ? (lev == 0 ? 1 : kstart) : kstart);; k += step) {
        double t = sgn * k * h;
        double s = exp(hpi * sinh(t));
        double w = hpi * cosh(t) * s;
        if (s > 1e4 || s < 1e-300) break;
        double v = w * f(s, ctx);
        add += v;
        if (k > 2 && fabs(v) < 1e-20 * fabs(add + sum)) break;
      }
    }
    sum += add;
    double est = sum * h;
    if (lev > 3 && fabs(est - prev) <= 1e-15 * fabs(est)) return est;
    prev = est;
    h *= 0.5;
  }
  return prev;
}

/* Gamma(alpha, 1): P(alpha, z) = int_0^z t^{a-1} e^{-t} dt / Gamma(a).
 * dz/dalpha = -int_0^z (ln t - psi(a)) t^{a-1} e^{-t} dt / (z^{a-1} e^{-z})
 *           = +int_z^inf (ln t - psi(a)) t^{a-1} e^{-t} dt / (z^{a-1} e^{-z}).
 * Lower form when ln z < psi(a) (integrand <= 0), upper form otherwise. */
typedef struct { double z, a, psi; } gctx;

static double g_lower(double u, double um, void* c) {
  /* t = z u^{1/a}: t^{a-1} dt = z^a/a du ; divide by z^{a-1} e^{-z} */
  (void)um;
  gctx* k = (gctx*)c;
  if (u <= 0.0) return 0.0;
  double lu = log(u) / k->a;             /* ln(t/z) */
  double t = k->z * exp(lu);
  return (k->z / k->a) * (log(k->z) + lu - k->psi) * exp(k->z - t);
}

static double g_upper(double s, void* c) {
  /* t = z + s */
  gctx* k = (gctx*)c;
  return (log(k->z + s) - k->psi) * exp((k->a - 1.0) * log1p(s / k->z) - s);
}

double or_gamma_dzda(double z, double a) {
  if (!(z > 0.0) || !(a > 0.0)) return 0.0;
  gctx k = {z, a, or_digamma(a)};
  if (log(z) < k.psi) return -ts01(g_lower, &k);
  return es0inf(g_upper, &k);
}

/* Beta(a, b): I_z(a,b); with kappa_a = psi(a) - psi(a+b),
 * dz/da = -int_0^z (ln t - kappa_a) t^{a-1}(1-t)^{b-1} dt / (z^{a-1}(1-z)^{b-1})
 *       = +int_z^1 (ln t - kappa_a) ... ;
 * dz/db: ln(1-t) - kappa_b in place of ln t - kappa_a. */
typedef struct { double z, a, b, ka, kb; int which; } bctx;

static double b_lower(double u, double um, void* c) {
  /* t = z u^{1/a} */
  (void)um;
  bctx* k = (bctx*)c;
  if (u <= 0.0) return 0.0;
  double lr = log(u) / k->a;            /* ln(t/z) */
  double t = k->z * exp(lr);
  double fac = (k->z / k->a) * exp((k->b - 1.0) * (log1p(-t) - log1p(-k->z)));
  double g = k->which == 0 ? (log(k->z) + lr - k->ka) : (log1p(-t) - k->kb);
  return g * fac;
}

static double b_upper(double u, double um, void* c) {
  /* 1 - t = (1 - z) u^{1/b} */
  (void)um;
  bctx* k = (bctx*)c;
  if (u <= 0.0) return 0.0;
  double lr = log(u) / k->b;            /* ln((1-t)/(1-z)) */
  double omt = (1.0 - k->z) * exp(lr);
  double t = 1.0 - omt;
  double fac = ((1.0 - k->z) / k->b) * exp((k->a - 1.0) * (log(t) - log(k->z)));
  double g = k->which == 0 ? (log(t) - k->ka) : (log(1.0 - k->z) + lr - k->kb);
  return g * fac;
}

/* Beta gradient through the gamma composition (the alternative to the
 * implicit beta-CDF derivative): z = X / (X + Y) with X = Gamma(a) and
 * Y = Gamma(b) each reparameterised by its own CDF, so
 *   dz/da = Y / (X + Y)^2 dX/da,   dz/db = -X / (X + Y)^2 dY/db,
 * dX/da and dY/db being the gamma implicit derivatives above. */
void or_beta_dzdab_composed(double x, double y, double a, double b, double* dzda, double* dzdb) {
  double s = x + y;
  double s2 = s * s;
  *dzda = y / s2 * or_gamma_dzda(x, a);
  *dzdb = -x / s2 * or_gamma_dzda(y, b);
}

void or_beta_dzdab(double z, double a, double b, double* dzda, double* dzdb) {
  double pab = or_digamma(a + b);
  bctx k = {z, a, b, or_digamma(a) - pab, or_digamma(b) - pab, 0};
  /* dz/da: integrand ln t - ka <= 0 on (0, z] iff ln z <= ka */
  k.which = 0;
  if (log(z) <= k.ka) *dzda = -ts01(b_lower, &k);
  else *dzda = ts01(b_upper, &k);
  /* dz/db: integrand ln(1-t) - kb is decreasing in t; on [z, 1) it is <= 0
   * iff ln(1-z) <= kb */
  k.which = 1;
  if (log1p(-z) <= k.kb) *dzdb = ts01(b_upper, &k);
  else *dzdb = -ts01(b_lower, &k);
}

/* ======================================================================
 * MVN (Sec. 3.1): x_j = mu + L z_j with Dot2 (Ogita, Rump & Oishi 2005).
 * ==================================================================== */
void or_mvn_apply(int d, size_t n, const double* mu, const double* L, const double* Z, double* X) {
  for (size_t j = 0; j < n; ++j) {
    const double* z = Z + j * (size_t)d;
    for (int i = 0; i < d; ++i) {
      double s = mu[i], c = 0.0;
      for (int k = 0; k <= i; ++k) {
        dd p = two_prod(L[(size_t)i * d + k], z[k]);
        dd q = two_sum(s, p.hi);
        s = q.hi;
        c += p.lo + q.lo;
      }
      X[j * (size_t)d + i] = s + c;
    }
  }
}

void or_mvn_grads(int d, size_t n, const double* G, const double* Z, double* gmu, double* gL) {
  for (int i = 0; i < d; ++i) {
    double s = 0.0, c = 0.0;
    for (size_t j = 0; j < n; ++j) {
      dd q = two_sum(s, G[j * (size_t)d + i]);
      s = q.hi;
      c += q.lo;
    }
    gmu[i] = s + c;
    for (int k = 0; k < d; ++k) {
      if (k > i) { gL[(size_t)i * d + k] = 0.0; continue; }
      double s2 = 0.0, c2 = 0.0;
      for (size_t j = 0; j < n; ++j) {
        dd p = two_prod(G[j * (size_t)d + i], Z[j * (size_t)d + k]);
        dd q = two_sum(s2, p.hi);
        s2 = q.hi;
        c2 += p.lo + q.lo;
      }
      gL[(size_t)i * d + k] = s2 + c2;
    }
  }
}
