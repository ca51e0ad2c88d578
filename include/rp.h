/* rp.h -- C ABI of the GB300 bulk-fill library (librp.so).
 *
 * Bulk filling of a device array with n variates from one seeded engine
 * stream, after Randompack (arXiv 2605.05099): engines of Sec. 2.2
 * (xoshiro256++, xoshiro256**, PCG64-DXSM, Philox4x32-10 and the paper's
 * Philox4x64-10), seeding and stream control of Sec. 2.3, the distribution
 * algorithms of Sec. 3 and the validation ideas of Sec. 5.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Status: 0 (RP_OK) on success, a negative RP_ERR_* code otherwise; the
 *   message of the last failure on the calling host thread is returned by
 *   rp_last_error() (mirrors the per-RNG last-error string of Sec. 2.1).
 *   No entry point aborts, traps or prints.
 * - Stream model: a stream is an engine state seeded from (seed, spawn key)
 *   (Sec. 2.3); `stream` is the spawn key, or RP_NO_STREAM for none.  Word p
 *   of a stream is the p-th 64-bit engine output after seeding.  `pos` is
 *   read as the first word to use and, on success, set to the next unused
 *   word: a fill consumes exactly the words its variates used, so two fills
 *   in a row give the same values as one fill of the combined length.
 * - Memory: `d_*` pointers are device memory owned by the caller; `h_*`
 *   pointers are host memory owned by the caller.  Output pointers must be
 *   8-byte aligned.  The library owns only immutable tables and an internal
 *   scratch pool that grows on demand and is kept: tile status words, the
 *   tail queue and, for bounded fills with frequent rejections, one parking
 *   area per resident CTA.  Fills drawn as pairs of base variates (beta
 *   and F with equal shapes, the skew normal) also allocate a temporary of
 *   16 min(n, 2^26) bytes for the call and free it before returning.
 * - Streams: `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 *   Fill calls enqueue their kernels on it.  When they return depends on
 *   the fill and on *pos:
 *   - one-word fills (rp_fill_u64, rp_fill_uniform, rp_fill_uniform52,
 *     rp_engine_fold, and rp_fill_uniformf with an even n) consume exactly
 *     n words: *pos is set on the host and the call returns without waiting
 *     for the kernel.  Their only stream operation is the kernel, so once a
 *     call with the same engine and size has set up the jump tables they
 *     can be captured into a CUDA graph (stream capture in relaxed mode)
 *     and replayed;
 *   - the other fills of rp_fill_u64's family and rp_fill_state, when pos
 *     points to host-pinned memory (cudaMallocHost, cudaHostRegister, a
 *     pinned torch tensor), enqueue their kernels, a one-thread kernel that
 *     forms the end position and a copy of it to *pos, and return without
 *     waiting.  *pos is valid once the stream is synchronised; it is
 *     UINT64_MAX if the fill failed on the device, and rp_async_status then
 *     gives the reason.  A later call that reads the same *pos first waits
 *     for the pending write (an event), so fills chained through one pinned
 *     word stay correct, and fills on several streams are ordered on the
 *     device around the library's shared scratch.  Bounded fills take the
 *     exact two-pass path in this mode;
 *   - otherwise (pos in pageable memory, and the fills drawn as pairs of
 *     base variates) the call synchronises the stream once at the end, to
 *     read the consumed-word count and the device status word.
 *   Gradients synchronise their stream to return the reduced sums.
 * - Threading: calls from several host threads are serialised internally;
 *   the lock is held while a call enqueues work, and across its final
 *   synchronisation only in the synchronous cases above.
 * - Devices: the allocating entry points (fills, gradients, batch plans, the
 *   MVN) keep their scratch, jump tables and uploaded tables for the device
 *   that was current at their first call; a later call with another device
 *   current fails with RP_ERR_PARAM before launching anything.  Only
 *   rp_fill_normal_philox_static keeps its state per device.  The library
 *   must not be used across cudaDeviceReset (its cached device pointers and
 *   tables would be stale).
 * - n = 0 is a valid no-op that leaves *pos unchanged (Sec. 5.1, zero
 *   lengths must work).
 */
#ifndef RP_H
#define RP_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RP_XOSHIRO256PP = 1,   /* Blackman & Vigna 2019, 4 x 64-bit state */
  RP_PCG64DXSM = 2,      /* O'Neill 2019, 128-bit LCG + DXSM output */
  RP_PHILOX4X32_10 = 3,  /* Salmon et al. 2011, 128-bit counter, 64-bit key */
  RP_PHILOX4X64_10 = 4,  /* the paper's Philox: 4 x 64-bit words per block, NumPy's Philox seeding */
  RP_XOSHIRO256SS = 5    /* Blackman & Vigna 2018: xoshiro256++'s state, seeding, jumps and
                            substreams, with the "**" scrambler rotl(5 s1, 7) 9 */
} rp_engine;

typedef int rp_status;
#define RP_OK 0
#define RP_ERR_NULL (-1)      /* a required pointer is NULL */
#define RP_ERR_PARAM (-2)     /* invalid distribution parameter or size */
#define RP_ERR_ENGINE (-3)    /* unknown engine id */
#define RP_ERR_CUDA (-4)      /* CUDA runtime error (message has details) */
#define RP_ERR_TIMEOUT (-5)   /* a bounded device wait ran out */
#define RP_ERR_NOMEM (-6)     /* scratch allocation failed */
#define RP_ERR_INTERNAL (-7)  /* device-side consistency check failed */
#define RP_ERR_SEED (-8)      /* seeding produced an all-zero xoshiro state */

#define RP_NO_STREAM UINT64_MAX

/* ---------------------------------------------------------------------
 * Fills.  Common arguments:
 *   engine  rp_engine id
 *   seed    user seed (Sec. 2.3 seeding: seed + spawn key hashed into a
 *           128-bit pool; NumPy SeedSequence semantics)
 *   stream  spawn key, or RP_NO_STREAM
 *   pos     in: first stream word to use; out: next unused word (host ptr;
 *           written asynchronously when it is host-pinned, see Streams)
 *   n       number of variates
 *   d_out   device array of n elements
 * ------------------------------------------------------------------- */

/* Raw 64-bit words (Table "discrete": uint64 with b = 0; raw bitstream). */
rp_status rp_fill_u64(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                      size_t n, uint64_t* d_out, void* cuda_stream);

/* The xor of words pos .. pos + n - 1 of the stream, written to d_fold (one
 * 64-bit device word, owned by the caller); *pos advances by n.  The words
 * are generated as the sequential-engine fills generate them (each thread
 * one contiguous range after one jump, Sec. 4.4 jump-ahead; Philox4x32-10's
 * one-word fills index its blocks directly instead) and folded, and nothing else is
 * computed or stored, so the call's words/s is the engine's throughput
 * ceiling for the fills (Table "engines" lists the paper's CPU rates of the
 * same engines).  Errors as for the fills; n = 0 leaves d_fold untouched. */
rp_status rp_engine_fold(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                         size_t n, uint64_t* d_fold, void* cuda_stream);

/* U[0,1) doubles with 53-bit resolution: floor(u / 2^11) * 2^-53 (Sec. 3.1,
 * method 1), one word per variate, bit-exact. */
rp_status rp_fill_uniform(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                          size_t n, double* d_out, void* cuda_stream);

/* 52-bit uniform in [0, 1), the paper's default (Sec. 3.1, method 2): the
 * word's top 52 bits in the fraction of a double in [1, 2), minus 1, which
 * is exactly floor(u / 2^12) 2^-52.  One word per variate. */
rp_status rp_fill_uniform52(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                            size_t n, double* d_out, void* cuda_stream);

/* Unbiased integers in [0, m) by Lemire's multiply-and-reject (Sec. 3.2):
 * one word per attempt, reject while low64(u m) < 2^64 mod m, output
 * high64(u m).  m = 0 gives the full 64-bit range (raw words). */
rp_status rp_fill_bounded(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                          size_t n, uint64_t m, uint64_t* d_out, void* cuda_stream);

/* Standard normal by the 256-strip ziggurat (Sec. 3.1): low byte = strip,
 * bit 8 = sign, bits 9-60 = magnitude r, x = +-RN(r w_i); fast accept when
 * r < k_i; wedge test y < exp(-x^2/2); tail beyond R by Marsaglia's 1964
 * method.  Accept decisions are exact (correctly rounded exp/log). */
rp_status rp_fill_normal(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                         size_t n, double* d_out, void* cuda_stream);

/* Standard exponential by the 256-strip ziggurat (Sec. 3.1): bits 8-60 =
 * magnitude; memoryless tail R - log(1 - U). */
rp_status rp_fill_exp(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                      size_t n, double* d_out, void* cuda_stream);

/* Float variants (Table "continuous": the functions with suffix f; Sec. 3.1
 * reads the engines' bits as 32-bit words, Sec. 4.4 notes that floats save
 * space and time).  The paper gives no more than "analogous"; the readings:
 * each 64-bit stream word gives two 32-bit words, its low half first; a
 * float fill starts at the low half of word *pos, and when it ends on a low
 * half the high half goes unused, so *pos stays a whole word (the next one).
 *   rp_fill_uniformf  floor(h / 2^9) 2^-23 (the default method in float),
 *                     two outputs per word; d_out must be 8-byte aligned
 *                     (RP_ERR_PARAM otherwise).
 *   rp_fill_normalf   bits 0-7 strip, bit 8 sign, bits 9-31 r (23 bits):
 *                     x = RN_f(r wf_i), wf_i = RN_f(2^29 w_i); fast accept
 *                     r < k_i / 2^29; the wedge y = RN_f((f_{i-1} - f_i) U + f_i)
 *                     in float operations, f_i = RN_f(F_i), U = floor(h / 2^8)
 *                     2^-24 of the next 32-bit word, accepted when
 *                     y < exp(-x^2 / 2) (correctly rounded, in double);
 *                     tails as the double sampler's with those U, in double,
 *                     rounded once to float.
 *   rp_fill_expf      bits 0-7 strip, bits 8-31 r (24 bits), likewise, with
 *                     the tail RN_f(R - log(1 - U)).
 * d_out: n floats (4-byte aligned for normalf and expf).  Errors and the
 * asynchronous *pos as for the double fills. */
rp_status rp_fill_uniformf(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                           size_t n, float* d_out, void* cuda_stream);
rp_status rp_fill_normalf(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                          size_t n, float* d_out, void* cuda_stream);
rp_status rp_fill_expf(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                       size_t n, float* d_out, void* cuda_stream);

/* Gamma(alpha, 1) by Marsaglia & Tsang (Sec. 3.1, gamma); alpha < 1 by the
 * boost Gamma(alpha+1) U^(1/alpha).  alpha > 0. */
rp_status rp_fill_gamma(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                        size_t n, double alpha, double* d_out, void* cuda_stream);

/* Beta(a, b) = X / (X + Y), X ~ Gamma(a) drawn before Y ~ Gamma(b)
 * (Table "continuous", beta).  a, b > 0.  Equal shapes run as a gamma fill
 * of 2n and a pairwise ratio.  Unequal shapes run on phased merge-point
 * seams: a seam is a word after which every chain that can enter the chunk
 * sits at a gamma boundary, in either phase (X or Y next), and each thread
 * carries a map from its entry phase to its exit phase and output count
 * that the scan and the look-back compose.  Shapes whose draws consume
 * words alike (2 and 2.0000001, 30 and 31) therefore need no special case;
 * a chunk without such a point is crossed by the walk before it (up to 64
 * chunks; more fails with RP_ERR_INTERNAL, which no tested shape reaches).
 * The same holds for F (rp_fill_derived) with unequal degrees of freedom. */
rp_status rp_fill_beta(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos,
                       size_t n, double a, double b, double* d_out, void* cuda_stream);

/* rp_fill_beta that also writes each output's gamma pair: d_x[i] = X_i,
 * d_y[i] = Y_i with z_i = X_i / (X_i + Y_i) (the same z as rp_fill_beta,
 * bit for bit), for the composed gradient (rp_beta_grad_composed).  No
 * counterpart in the paper.  d_x, d_y: n doubles each, 8-byte aligned. */
rp_status rp_fill_beta_xy(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, double a,
                          double b, double* d_z, double* d_x, double* d_y, void* cuda_stream);

/* Derived distributions (Table "continuous"; Sec. 3.1 "Gamma and related
 * distributions", "Extreme value and Weibull distributions").  Each output
 * transforms the base sampler's variate as it is written, in the formula's
 * order, one IEEE operation per step:
 *   RP_UNIF         (a, b)          a + (b - a) u, u the 53-bit uniform; a <= b
 *   RP_NORMAL_MS    (mu, sigma)     mu + sigma z, z standard normal
 *   RP_LOGNORMAL    (mu, sigma)     exp(mu + sigma z)
 *   RP_EXP_SCALE    (beta)          beta E, E standard exponential
 *   RP_GAMMA_SCALE  (alpha, theta)  theta Gamma(alpha)
 *   RP_CHI2         (nu)            2 Gamma(nu / 2)
 *   RP_GUMBEL       (mu, beta)      mu - beta log(-log u)
 *   RP_PARETO       (x_m, alpha)    x_m exp(E / alpha)
 *   RP_WEIBULL      (k, lambda)     lambda pow(E, 1 / k)
 *   RP_GPD          (mu, sigma, xi) P = Pareto(1, 1/|xi|): mu + sigma (P - 1) / xi
 *                                   (xi > 0), mu - sigma (1 - 1/P) / xi (xi < 0),
 *                                   mu + sigma E (xi = 0)
 *   RP_F            (nu1, nu2)      (X / nu1) / (Y / nu2), X ~ Gamma(nu1/2) drawn
 *                                   before Y ~ Gamma(nu2/2)
 *   RP_SKEW_NORMAL  (mu, sigma, alpha)  two consecutive normals u0, u1:
 *                                   mu + sigma (delta |u0| + sqrt(1 - delta^2) u1),
 *                                   delta = alpha / sqrt(1 + alpha^2)
 *   RP_T            (nu)            Z / sqrt(V / nu), Z ~ N(0, 1) drawn before
 *                                   V ~ chi2_nu = 2 Gamma(nu / 2)
 * params: 4 doubles (unused ones ignored), host memory.  Scale and shape
 * parameters must be positive and finite, locations finite; otherwise
 * RP_ERR_PARAM before any device work.  exp and pow are CUDA's (one and two
 * ulp), Gumbel's logs correctly rounded; the decisions of the base samplers
 * are exact as in the base fills.  *pos advances by the base words used. */
typedef enum {
  RP_UNIF = 1, RP_NORMAL_MS = 2, RP_LOGNORMAL = 3, RP_EXP_SCALE = 4, RP_GAMMA_SCALE = 5, RP_CHI2 = 6,
  RP_GUMBEL = 7, RP_PARETO = 8, RP_WEIBULL = 9, RP_GPD = 10, RP_F = 11, RP_SKEW_NORMAL = 12, RP_T = 13
} rp_derived;
rp_status rp_fill_derived(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, rp_derived kind,
                          const double* params, size_t n, double* d_out, void* cuda_stream);

/* ---------------------------------------------------------------------
 * Distributions by code, fills from explicit state, substreams and
 * batched fills.
 * ------------------------------------------------------------------- */
typedef enum {
  RP_DIST_U64 = 0,       /* raw words */
  RP_DIST_UNIFORM = 1,   /* 53-bit U[0,1) */
  RP_DIST_BOUNDED = 2,   /* [0, m), m = 0 full range */
  RP_DIST_NORMAL = 3,
  RP_DIST_EXP = 4,
  RP_DIST_GAMMA = 5,     /* alpha = p0 */
  RP_DIST_BETA = 6,      /* a = p0, b = p1 */
  RP_DIST_UNIFORM52 = 7  /* 52-bit U[0,1), the paper's default (rp_fill_uniform52) */
} rp_dist;

/* A fill into host memory, the end-to-end form of rp_fill_state's
 * distributions (dist, p0, p1, m as there): the library fills one of two
 * device staging slots on cuda_stream and copies it to h_out (n 8-byte
 * elements) on its own copy stream, so that a fill overlaps the previous
 * call's copy.  With h_out in pinned memory the call returns once the work
 * is enqueued and h_out is complete after the device is synchronised
 * (cudaDeviceSynchronize, or rp_async_status(NULL)); synchronising
 * cuda_stream alone does not cover the copy.  With h_out in pageable memory
 * the copy completes before the call returns.  *pos as for the fills
 * (written asynchronously when pinned).  Library convenience: the paper's
 * fills write host memory directly. */
rp_status rp_fill_to_host(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, int dist, size_t n,
                          double p0, double p1, uint64_t m, void* h_out, void* cuda_stream);

/* Fill n variates of `dist` from a stream given by its state words (the
 * engine before word 0, layout of rp_seed_state), starting at word *pos;
 * *pos is set to the next unused word.  Same values as the seeded fills of
 * the same stream.  d_out: device array of n 8-byte elements (uint64 for
 * u64/bounded, double otherwise). */
rp_status rp_fill_state(rp_engine engine, const uint64_t* words, uint64_t* pos, int dist, size_t n,
                        double p0, double p1, uint64_t m, void* d_out, void* cuda_stream);

/* State words of substream s of base_seed, the paper's recipe for parallel
 * simulations (Sec. 2.3: copy a base generator, then jump it or set its
 * stream): the
 * base state is seeded from base_seed with no spawn key; the xoshiro engines
 * jump it by s * 2^128 words, Philox sets its (first) key word to s, PCG64-DXSM sets
 * its increment to 2 s + 1.  words must hold 4 entries; *nw receives the
 * count used. */
rp_status rp_substream_state(rp_engine engine, uint64_t base_seed, uint64_t s, uint64_t* words, int* nw);

/* One request of a batch: n variates of `dist` from substream `stream`. */
typedef struct {
  uint64_t stream;   /* substream index s */
  int32_t dist;      /* rp_dist */
  int32_t reserved;  /* must be 0 */
  uint64_t n;        /* variates (0: nothing) */
  double p0, p1;     /* gamma: alpha = p0; beta: a = p0, b = p1 with a != b */
  uint64_t m;        /* bounded: modulus (0: full range) */
  void* d_out;       /* device array of n 8-byte elements, 8-byte aligned */
  uint64_t pos;      /* first word of the substream to use */
} rp_request;

/* A batch plan: every request of a fixed set, served by one CUDA-graph
 * launch of persistent kernels (one per kernel class: one-word, ziggurat and
 * bounded, gamma and beta) that claim (request, tile) work items.  Not in
 * the paper, whose parallel use is one generator object per simulation.
 *   reqs      nreq requests (copied; output pointers must stay valid)
 *   autotune  1: time the schedules (item order, class concurrency, words
 *             per thread) on this request set and keep the fastest;
 *             0: the default schedule
 *   plan      receives the plan (owned by the caller; rp_batch_plan_destroy)
 * Beta requests need a != b (equal shapes: rp_fill_beta or rp_fill_state).
 * Tuning runs the batch several times; outputs are identical each time. */
typedef struct rp_batch_plan rp_batch_plan;
rp_status rp_batch_plan_create(const rp_request* reqs, size_t nreq, rp_engine engine, uint64_t base_seed,
                               int autotune, rp_batch_plan** plan, void* cuda_stream);
/* Runs the plan on cuda_stream and returns after it completed.  Every
 * request is filled from its own start word; next_pos (nullable, nreq
 * entries) receives each request's next unused word. */
rp_status rp_batch_plan_run(rp_batch_plan* plan, uint64_t* next_pos, void* cuda_stream);
/* Schedule chosen (bit 0 item order by size, bit 1 classes serialised,
 * bit 2 128 words per thread), its tuned time in ms (0 if not tuned) and the
 * number of work items. */
rp_status rp_batch_plan_info(const rp_batch_plan* plan, int* schedule, double* tuned_ms, uint64_t* items);
rp_status rp_batch_plan_destroy(rp_batch_plan* plan);
/* One-shot: create (default schedule), run, write each request's next
 * unused word back into reqs[i].pos, destroy. */
rp_status rp_batch_run(rp_request* reqs, size_t nreq, rp_engine engine, uint64_t base_seed, void* cuda_stream);

/* ---------------------------------------------------------------------
 * Normal fill on fixed scratch (Philox4x32-10 only).  Randompack has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory -- code running inside a device allocator's own callbacks
 * (an out-of-memory or pool-trim hook, where allocating would re-enter the
 * allocator), processes whose device memory is all reserved by a caching
 * pool (a fresh cudaMalloc would fail although the pool has room), and
 * loops that cannot take the device-wide synchronisation of cudaFree.
 *
 * Same arguments, stream semantics and output as rp_fill_normal with
 * engine = RP_PHILOX4X32_10, bit for bit.  Its look-back status words,
 * control block and tail queue live in one file-scope device array of the
 * library (about 1.5 MB per device, in place from the moment the library's
 * device code is loaded), so no allocation routine is called.
 *   n        0 .. RP_STATIC_MAX_N; larger n is refused with RP_ERR_PARAM
 *            before any device work (split the call, or use
 *            rp_fill_normal).
 * The first call on each device does a one-time setup with that device
 * current: it looks up the array's address (cudaGetSymbolAddress) and
 * uploads the ziggurat tables; make that first call before any stream
 * capture begins.  Every call on a device uses the same array, so two calls
 * with work in flight at once would race on it; the library's internal
 * lock, held until the call has synchronised its stream, keeps calls from
 * several host threads apart.
 * ------------------------------------------------------------------- */
#define RP_STATIC_MAX_N ((size_t)1 << 22)
rp_status rp_fill_normal_philox_static(uint64_t seed, uint64_t stream, uint64_t* pos, size_t n,
                                       double* d_out, void* cuda_stream);

/* ---------------------------------------------------------------------
 * Pathwise (reparameterisation) gradients.  For z = F^{-1}(u; theta) at
 * fixed u, dz/dtheta = -(dF/dtheta)(z) / f(z): the implicit derivative of the
 * CDF.  Not in the paper (its samplers have no gradients); FP64 throughout.
 *   d_z       device array of n variates (as drawn by rp_fill_gamma/beta)
 *   d_g       device array of n upstream gradients dL/dz, or NULL
 *   d_dz*     device arrays receiving the per-sample dz/dtheta, or NULL
 *   h_grad*   host scalars receiving sum_i g_i dz_i/dtheta (needed when d_g
 *             is given; deterministic fixed-order reduction)
 * The call returns after the kernels have finished.  alpha, a, b > 0.
 * ------------------------------------------------------------------- */
rp_status rp_gamma_grad(const double* d_z, double alpha, const double* d_g, size_t n, double* d_dzda,
                        double* h_grad_alpha, void* cuda_stream);
rp_status rp_beta_grad(const double* d_z, double a, double b, const double* d_g, size_t n, double* d_dzda,
                       double* d_dzdb, double* h_grad_a, double* h_grad_b, void* cuda_stream);

/* Beta gradient through the gamma composition (the alternative to the CDF
 * derivative above; not in the paper): with z = X / (X + Y) and X ~ Gamma(a),
 * Y ~ Gamma(b) each reparameterised by its own CDF,
 *   dz/da = Y / (X + Y)^2 dX/da,   dz/db = -X / (X + Y)^2 dY/db,
 * dX/da and dY/db being rp_gamma_grad's implicit derivatives.  d_x, d_y: the
 * n gamma pairs of the beta draws (rp_fill_beta_xy); other arguments as for
 * rp_beta_grad.  NULL d_dzda/d_dzdb are replaced by temporaries for the call. */
rp_status rp_beta_grad_composed(const double* d_x, const double* d_y, double a, double b, const double* d_g,
                                size_t n, double* d_dzda, double* d_dzdb, double* h_grad_a, double* h_grad_b,
                                void* cuda_stream);

/* ---------------------------------------------------------------------
 * Multivariate normal (Sec. 3.1, multivariate normal): x = mu + L z for n
 * samples of dimension d, z a vector of d standard normals.
 *   d_mu  device, d entries
 *   d_L   device, d x d row-major; only the lower triangle (k <= i) is read
 *   d_Z   device, n x d row-major: receives the n d normals drawn from the
 *         stream (sample j takes normals j d .. j d + d - 1), kept for the
 *         backward pass
 *   d_X   device, n x d row-major: X[j] = mu + L Z[j]
 * The product runs on the FP64 tensor cores; |x - exact| is within 1e-13
 * (|mu| + |L| |z|) componentwise.  1 <= d <= 65536.  Returns after the
 * kernels completed; *pos is set to the next unused word.
 * ------------------------------------------------------------------- */
rp_status rp_mvn(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, int d, size_t n,
                 const double* d_mu, const double* d_L, double* d_Z, double* d_X, void* cuda_stream);
/* Gradients of a loss with upstream d_G = dLoss/dX (n x d): d_gmu (d) =
 * sum_j G[j], d_gL (d x d) = tril(G^T Z) (zero above the diagonal).  Sums
 * are in a fixed order (deterministic).  Not in the paper. */
rp_status rp_mvn_grads(int d, size_t n, const double* d_G, const double* d_Z, double* d_gmu, double* d_gL,
                       void* cuda_stream);

/* ---------------------------------------------------------------------
 * Seeding and stream control (Sec. 2.3), host only.
 * ------------------------------------------------------------------- */
/* Engine state words from (seed, spawn key): xoshiro s0..s3; PCG64 state
 * hi, state lo, inc hi, inc lo; Philox counter lo, counter hi, key.
 * words must hold 4 entries; *nw receives the count used. */
rp_status rp_seed_state(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* words, int* nw);

/* Advance state words (layout as above) by delta = delta_hi 2^64 + delta_lo
 * words: for xoshiro the product of the binary powers T^(2^j) of its GF(2)
 * transition matrix (the same map as the jump polynomial of Sec. 4.4), LCG
 * skip-ahead for PCG64 (Sec. 2.3), counter offset for Philox (delta even). */
rp_status rp_jump_state(rp_engine engine, uint64_t* words, uint64_t delta_hi, uint64_t delta_lo);

/* The library's correctly rounded natural log of n device doubles (d_y[i] =
 * RN(log d_x[i])), the routine behind the gamma boost and the ziggurat tail
 * values (Sec. 4.2 exactness, read as correct rounding).  For checks. */
rp_status rp_log_cr(const double* d_x, double* d_y, size_t n, void* cuda_stream);

/* The library's correctly rounded exp of n device doubles (d_y[i] =
 * RN(exp d_x[i])), the routine that decides the ziggurat wedge tests when
 * y lies within 2^-48 of the libm value (Sec. 3.1 wedges; Sec. 4.2
 * exactness, read as correct rounding).  For checks. */
rp_status rp_exp_cr(const double* d_x, double* d_y, size_t n, void* cuda_stream);

/* How often the exact accept decisions fell back past their fast tests,
 * since the last reset (for checks; Sec. 4.2 exactness): every wedge,
 * normal-tail pair and Marsaglia-Tsang test is decided first in FP32 with a
 * proven margin, then in FP64 with libm and a margin of its error, and only
 * then with the correctly rounded exp/log.  h_counts[6] (host) receives
 *   [0] wedge tests decided past the FP32 margin, [1] of those past the
 *   libm margin (correctly rounded exp), [2], [3] the same for normal tail
 *   pairs (correctly rounded logs), [4], [5] for Marsaglia-Tsang tests.
 * reset != 0 zeroes the counters after reading them.  Reads device memory:
 * call it after the fills it should count have completed. */
rp_status rp_debug_counters(uint64_t* h_counts, int reset);

/* Test hooks of the device error paths (no counterpart in the paper): they
 * make the bounded waits and capacity checks of later fills fail on purpose,
 * without faulting or hanging the GPU.  kind 0 clears every hook; 1: the
 * look-back waits give up after `value` spins (default 2^25) and report
 * RP_ERR_TIMEOUT; 2: tile value - 1 of each launch publishes no count, so
 * its successors' waits run out (0: none); 3: the tail queue holds at most
 * `value` entries (a fill that needs more fails with RP_ERR_INTERNAL);
 * 4: at most `value` tiles per launch for the sampled fills, so that the
 * fill continues over further launches (more than 64 fail with
 * RP_ERR_INTERNAL).  Host state only; returns RP_ERR_PARAM for an unknown
 * kind. */
rp_status rp_debug_faults(int kind, uint64_t value);

/* Failures of asynchronous fills (pinned *pos, see Streams): synchronises
 * cuda_stream (NULL: the whole device), then returns RP_OK if no
 * asynchronous fill has failed since the last call, else RP_ERR_TIMEOUT (a
 * bounded device wait gave up) or RP_ERR_INTERNAL (a device check failed, or
 * the fill needed more tiles than its one launch planned), with the count
 * and the device bits in rp_last_error(), and clears the record.  Library
 * state only; the paper's interface has no counterpart (its fills are
 * synchronous CPU calls). */
rp_status rp_async_status(void* cuda_stream);

/* Message of the last failed call on this host thread ("" if none). */
const char* rp_last_error(void);

/* Library version string. */
const char* rp_version(void);

/* Number of CUDA kernels this library has launched in this process (a
 * diagnostic counter for benchmarks). */
uint64_t rp_kernel_launches(void);

/* Checkpointing (Sec. 4.4, "Thread safety and checkpointing"): a stream's
 * exact state -- engine, the state words before word 0 (as rp_seed_state,
 * rp_substream_state and rp_fill_state use them) and the position -- as an
 * opaque, self-checking buffer of RP_STATE_BYTES bytes, and back.  A fill
 * resumed from a restored state continues the stream exactly.
 *   rp_state_serialize    buf: RP_STATE_BYTES writable host bytes
 *   rp_state_deserialize  refuses (RP_ERR_PARAM) a short buffer, a wrong
 *                         magic or version, an unknown engine, a corrupted
 *                         checksum or an all-zero xoshiro state;
 *                         words receives 4 words. */
#define RP_STATE_BYTES 64
rp_status rp_state_serialize(rp_engine engine, const uint64_t* words, uint64_t pos, uint8_t* buf, size_t buflen);
rp_status rp_state_deserialize(const uint8_t* buf, size_t buflen, rp_engine* engine, uint64_t* words, uint64_t* pos);

/* Engine query: the canonical identifier of engine id (1 ..), or NULL for
 * an unknown id. */
const char* rp_engine_name(int engine);

/* Ziggurat tables used by the kernels (which: 0 normal, 1 exponential):
 * k[256], w[256], f[256] and R.  For inspection and tests. */
rp_status rp_ziggurat_tables(int which, uint64_t* k, double* w, double* f, double* R);

#ifdef __cplusplus
}
#endif
#endif
