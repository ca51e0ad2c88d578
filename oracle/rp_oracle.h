/* Serial CPU oracle for the bulk-fill hot path of Randompack
 * (arXiv 2605.05099).  TEST INFRASTRUCTURE ONLY: only tests/, the smoke check
 * and the CPU-baseline leg of bench.py may load it.  It shares no code with the
 * CUDA path and the CUDA path never calls it.
 *
 * Everything is plain serial C compiled with -ffp-contract=off (Sec. 4.2:
 * bit-identity of the double results needs contraction off).
 *
 * Stream model: a generator is an engine state seeded from (seed, spawn key)
 * (Sec. 2.3) plus a word position `pos`; word p of the stream is the p-th
 * 64-bit engine output after seeding.  A fill consumes exactly the words its
 * variates used and leaves `pos` at the next unconsumed word.
 *
 * Parity unpinned: the output functions of the xoshiro engines.  The
 * xoshiro256++ scrambler, rotl(s0 + s3, 23) + s0, and the constants of the
 * xoshiro256** scrambler (5, 7, 9) are taken from the engines' published
 * definitions, and nothing on this machine gives their outputs (no test
 * vectors; NumPy has no xoshiro).  Their shared transition is pinned by its
 * primitive characteristic polynomial and by jump identities, and the
 * xoshiro256** outputs are tied to that transition's state words (see
 * tests/test_oracle_engines.py).
 */
#ifndef RP_ORACLE_H
#define RP_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_XOSHIRO256PP = 1, OR_PCG64DXSM = 2, OR_PHILOX4X32_10 = 3, OR_PHILOX4X64_10 = 4, OR_XOSHIRO256SS = 5 };

typedef struct {
  int engine;
  /* xoshiro256++ and xoshiro256**: s[0..3].
   * PCG64-DXSM:   s[0]=state hi, s[1]=state lo, s[2]=inc hi, s[3]=inc lo.
   * Philox4x32-10: s[0]=counter lo 64, s[1]=counter hi 64,
   *                s[2]=key (k0 = low 32 bits, k1 = high 32 bits).
   * Philox4x64-10: s[0]=counter lo 64, s[1]=counter hi 64 (counter words
   *                2, 3 are zero), s[2]=k0, s[3]=k1. */
  uint64_t s[4];
  uint64_t pos;          /* words consumed since the seeded state */
  /* Philox block cache (block index relative to the seeded counter) */
  uint64_t blk_idx; int blk_valid; uint64_t blk[4];
} or_gen;

/* ---- seeding (Sec. 2.3; seed_seq_fe128-style mixer, NumPy SeedSequence
 *      semantics) ---- */
/* entropy words -> n_out 32-bit state words (pool of four 32-bit words). */
void or_seedseq_generate(const uint32_t* entropy, int n_entropy, uint32_t* out, int n_out);
/* (seed, spawn key) -> uint32 entropy words; returns count (<= 8). has_key=0: no key */
int or_seedseq_entropy(uint64_t seed, int has_key, uint64_t key, uint32_t* ent);
/* engine state words from (seed, spawn key).  Returns 0, or -1 if the seeded
 * xoshiro state is all zero. */
int or_gen_seed(or_gen* g, int engine, uint64_t seed, int has_key, uint64_t key);
/* raw state assignment (tests) */
void or_gen_set(or_gen* g, int engine, const uint64_t s[4]);

/* ---- engines ---- */
uint64_t or_next(or_gen* g);
/* jump the generator forward by n words (n = n_hi*2^64 + n_lo); pos += n mod 2^64 */
void or_jump(or_gen* g, uint64_t n_hi, uint64_t n_lo);
void or_seek(or_gen* g, uint64_t pos);           /* from the seeded state: jump to pos */
/* xoshiro jump by N given as little-endian 64-bit limbs, two independent
 * constructions (Sec. 4.4): the jump polynomial x^N mod charpoly(T) and
 * repeated squaring of the 256x256 GF(2) matrix. */
void or_xoshiro_jump_poly(uint64_t s[4], const uint64_t* n_limbs, int nl);
void or_xoshiro_jump_matrix(uint64_t s[4], const uint64_t* n_limbs, int nl);
void or_xoshiro_charpoly(uint64_t p[5]);         /* degree-256 polynomial, bit k = coeff of x^k */
/* PCG64-DXSM: advance by delta (128-bit) */
void or_pcg_advance(uint64_t s[4], uint64_t d_hi, uint64_t d_lo);
/* Philox4x32-10 bijection: ctr[4], key[2] -> out[4] */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
void or_fill_uniform52(or_gen* g, size_t n, double* out);

/* ---- correctly rounded elementary functions used in accept tests
 *      (double-double evaluation, rounded once).  Sec. 4.2. ---- */
double or_cr_exp(double x);
double or_cr_log(double x);
/* number of evaluations whose double-double value was too close to a
 * rounding boundary to certify correct rounding (expected: 0). */
uint64_t or_cr_ambiguous(void);
void or_cr_reset(void);

/* ---- distributions (Sec. 3).  `start` (nullable) receives, per output,
 *      the stream position of the word that began the accepted candidate. */
void or_fill_u64(or_gen* g, size_t n, uint64_t* out);
void or_fill_uniform(or_gen* g, size_t n, double* out);                  /* 53-bit */
void or_fill_bounded(or_gen* g, size_t n, uint64_t m, uint64_t* out, uint64_t* start);
void or_fill_normal(or_gen* g, size_t n, double* out, uint64_t* start);
void or_fill_exp(or_gen* g, size_t n, double* out, uint64_t* start);
int  or_fill_gamma(or_gen* g, size_t n, double alpha, double* out, uint64_t* start);
int  or_fill_beta(or_gen* g, size_t n, double a, double b, double* out, uint64_t* start);

/* float variants (suffix f): the stream read as 32-bit words, low half of
 * each word first; `start` receives 32-bit word indices (2 word + half).
 * The position after a fill is the next whole word. */
void or_fill_uniformf(or_gen* g, size_t n, float* out);
void or_fill_normalf(or_gen* g, size_t n, float* out, uint64_t* start);
void or_fill_expf(or_gen* g, size_t n, float* out, uint64_t* start);
int  or_zig_table_f(int which, int i, uint32_t* k, float* w, float* f);

/* derived distributions (Table "continuous"): kinds and parameters p[]
 *   UNIF (a, b), NORMAL_MS (mu, sigma), LOGNORMAL (mu, sigma), EXP_SCALE (beta),
 *   GAMMA_SCALE (alpha, theta), CHI2 (nu), GUMBEL (mu, beta), PARETO (x_m, alpha),
 *   WEIBULL (k, lambda), GPD (mu, sigma, xi), F (nu1, nu2), SKEW_NORMAL (mu, sigma, alpha), T (nu) */
enum { OR_D_UNIF = 1, OR_D_NORMAL_MS = 2, OR_D_LOGNORMAL = 3, OR_D_EXP_SCALE = 4, OR_D_GAMMA_SCALE = 5,
       OR_D_CHI2 = 6, OR_D_GUMBEL = 7, OR_D_PARETO = 8, OR_D_WEIBULL = 9, OR_D_GPD = 10, OR_D_F = 11,
       OR_D_SKEW_NORMAL = 12, OR_D_T = 13 };
int  or_fill_derived(or_gen* g, int kind, size_t n, const double* p, double* out, uint64_t* start);
double or_cr_pow(double x, double y);
/* ziggurat internals for tests */
double or_zig_normal_x(uint64_t u);              /* candidate x = +-RN(r*w_i) */
int    or_zig_table(int which, int i, uint64_t* k, double* w, double* f); /* 0 normal, 1 exp */
double or_zig_R(int which);
/* counters from the last normal/exp fill: fast accepts, wedge tests, rejections, tail */
void or_zig_counts(uint64_t c[4]);

/* ---- pathwise gradients (reparameterisation; implicit derivative of the
 *      CDF at fixed F).  Adaptive tanh-sinh quadrature in double. ---- */
double or_digamma(double x);
double or_gamma_dzda(double z, double alpha);
void   or_beta_dzdab(double z, double a, double b, double* dzda, double* dzdb);
/* the same gradient through the gamma pair (x, y) that made z = x / (x + y) */
void   or_beta_dzdab_composed(double x, double y, double a, double b, double* dzda, double* dzdb);

/* ---- multivariate normal X = mu + L z (Sec. 3.1, mvn).  Row-major n x d
 *      X and Z, L lower-triangular d x d row-major.  Compensated dot
 *      product (Dot2). */
void or_mvn_apply(int d, size_t n, const double* mu, const double* L, const double* Z, double* X);
/* grads: gmu[d] = sum_j G_j ; gL[d*d] = tril(G^T Z) (compensated sums) */
void or_mvn_grads(int d, size_t n, const double* G, const double* Z, double* gmu, double* gL);

/* ---- batched substreams: request r uses substream s (xoshiro: seeded state
 *      jumped by s*2^128; Philox: seeded state with key := s) from word 0. */
void or_substream(or_gen* g, int engine, uint64_t base_seed, uint64_t s);

#ifdef __cplusplus
}
#endif
#endif
