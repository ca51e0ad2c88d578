// Internal interface between the host side (rp_host.cpp) and the kernels
// (rp_kernels.cu) of librp.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>

namespace rp {

enum Dist : int { D_U64 = 0, D_UNIFORM = 1, D_BOUNDED = 2, D_NORMAL = 3, D_EXP = 4, D_GAMMA = 5, D_BETA = 6,
                  D_BOUNDED_ONE = 7,   // bounded, one pass that assumes no rejection (records the first one)
                  D_T = 8,             // Student t: a normal, then a gamma (ep[0] = nu)
                  D_UNIFORM52 = 9,     // the paper's default 52-bit uniform
                  D_FOLD = 10,         // xor of the words, no output array (engine-only throughput)
                  D_UNIFORMF2 = 11,    // float uniforms, two per word (the output as 8-byte pairs)
                  D_NORMALF = 12,      // float ziggurat normal over 32-bit half-words
                  D_EXPF = 13 };       // float ziggurat exponential over 32-bit half-words

// Device error bits (ctrl->err)
enum : unsigned {
  E_TIMEOUT = 1u,     // a bounded spin-wait gave up
  E_LANDING = 2u,     // a segment walk jumped over the next sync point
  E_OVERFLOW = 4u,    // a candidate needed words beyond the tile halo
  E_NOSYNC = 8u,      // no tile-start sync point within the search window
  E_INCOMPLETE = 16u, // an asynchronous fill ran out of its planned tiles
};

// Per-launch control block in device memory (scratch).
struct Ctrl {
  unsigned long long done_tile;   // index of the tile that produced output n-1 (init: ~0)
  unsigned long long total;       // outputs produced when the launch ran out of tiles
  unsigned long long next_pos;    // stream position (relative to the launch) after the last output
  unsigned long long last_tile;   // last tile whose exit position was recorded
  unsigned int err;               // E_* bits
  unsigned int pad;
  unsigned long long err_info;
  unsigned long long n_tail;      // entries in the tail queue
  unsigned long long first_reject;   // D_BOUNDED_ONE: first rejected word (relative; init ~0)
};

// Deferred output whose value needs FP64 libm (ziggurat tails): output
// index and the two words that define it.
struct TailEntry {
  unsigned long long g, w0, w1;
  unsigned long long x[6];   // gamma/beta: the record words of the variate
};

// Engine description for one launch.  All word offsets are relative to the
// launch's first word (the caller's *pos).
struct EngineArgs {
  int engine;                   // 1 xoshiro, 2 pcg, 3 philox
  unsigned long long s[4];      // xoshiro: state at the first word; pcg: state hi, lo, inc hi, lo;
                                // philox: counter lo, hi (seeded), key
  unsigned long long word0;     // philox: index of the first word relative to the seeded counter
  // xoshiro: nibble tables (64 chunks x 16 entries x 32 B) of T^(2^j), j = 0..63, and of T^stride
  const void* gf2_pow;
  const void* gf2_stride;
  const void* gf2_thread;   // nibble tables of T^(t C), t < threads per CTA
  const void* gf2_cta;      // nibble tables of T^(T 2^j), j < 16 (T = words per tile)
  // pcg: affine powers (A_j, G_j) for 2^j steps, j = 0..63, as {A hi, A lo, G hi, G lo}
  const unsigned long long* pcg_pow;
  unsigned long long pcg_stride[4];   // (A, G) for the stride
  unsigned long long stride;          // words between a thread's chunks in consecutive tiles
  unsigned long long tile_words;      // words per tile (T)
  unsigned long long chunk_words;     // words per thread chunk (C)
};

// Marsaglia-Tsang constants of one gamma shape: d = s - 1/3, c = 1/sqrt(9 d)
// for s = alpha (alpha >= 1) or s = alpha + 1 with the boost U^(1/alpha).
struct MTParams {
  double d, c, alpha;
  float df, cf;
  int boost;
  int pad;
};

// Output transforms of the derived distributions (Table "continuous"),
// applied to each base variate as it is written.  Parameters ep[]:
//   EPI_AFFINE   ep0 + ep1 x                 unif (a, b - a), normal (mu, sigma)
//   EPI_SCALE    ep0 x                       Exp(beta), Gamma(alpha, theta), chi2 (2)
//   EPI_LOGNORMAL exp(ep0 + ep1 x)           (mu, sigma)
//   EPI_GUMBEL   ep0 - ep1 log(-log x)       (mu, beta), correctly rounded logs
//   EPI_PARETO   ep0 exp(x / ep1)            (x_m, alpha)
//   EPI_WEIBULL  ep1 pow(x, ep0)             (1/k, lambda)
//   EPI_GPD      generalized Pareto          (mu, sigma, xi, 1/|xi|)
//   EPI_F        (X / ep0) / (Y / ep1)       beta record of Gamma(nu1/2), Gamma(nu2/2)
enum Epi : int { EPI_NONE = 0, EPI_AFFINE = 1, EPI_SCALE = 2, EPI_LOGNORMAL = 3, EPI_GUMBEL = 4, EPI_PARETO = 5,
                 EPI_WEIBULL = 6, EPI_GPD = 7, EPI_F = 8 };

struct SampArgs {
  unsigned long long m;       // bounded: modulus (0 = full range)
  unsigned long long thresh;  // bounded: 2^64 mod m
  MTParams ga, gb;            // gamma: ga; beta: X ~ ga, Y ~ gb
  double ep[4];               // output transform parameters
  int epi;                    // output transform (Epi), 0 for the base distributions
  int half0;                  // half-word fills: the first half-word of the launch to use (0 or 1)
  double* outx;               // beta: when not NULL, each output's gamma pair X, Y is also
  double* outy;               //   written here (same index as the output)
};

struct FillArgs {
  EngineArgs eng;
  SampArgs sp;
  int dist;
  unsigned long long n;          // outputs wanted in this launch
  unsigned long long n_tiles;    // tiles available in this launch
  void* out;
  unsigned long long* tile_status;  // n_tiles words (zeroed)
  Ctrl* ctrl;
  TailEntry* tailq;                 // deferred tail outputs
  unsigned long long tail_cap;
  unsigned long long* tail_count;   // entries claimed in tailq (&ctrl->n_tail for one fill)
  int tail_abs;                     // 1: TailEntry.g is the output's address (batches), 0: its index
  int req;                          // request index within a batch
  unsigned long long* park;         // one-pass bounded fill: grid x tile words of parked values
  // test hooks (zero: off): look-back waits give up after spin_max spins
  // instead of kSpinMax; tile stall_tile1 - 1 publishes nothing, so that its
  // successors' waits run out
  unsigned long long spin_max;
  unsigned long long stall_tile1;
};

// Batched fills: one work item is one tile of one request.  Items of a
// request are listed in tile order, so a tile's predecessors are always
// claimed before it (the look-back cannot wait on an unclaimed tile).
struct BatchItem {
  unsigned req, tile;
};
struct BatchArgs {
  const FillArgs* reqs;             // per-request arguments (device)
  const BatchItem* items;           // work list (device)
  unsigned long long n_items;
  unsigned long long* next_item;    // claim counter (zeroed before the launch)
  TailEntry* tailq;                 // tail queue shared by the class
  unsigned long long* tail_count;
  unsigned long long tail_cap;
};

// Kernel classes of a batch (one persistent kernel each).
enum BatchClass : int { BC_ONEPW = 0, BC_LEAN = 1, BC_MERGE = 2 };

// Kernel launchers (rp_kernels.cu).  Return a cudaError_t value.
// Batched launches: grid <= 0 asks for the occupancy (resident CTAs per SM)
// in *occ instead of launching.  cvar selects the words per thread of the
// one-word and bitmap classes: 0 -> 256, 1 -> 128 (merge class: 2048).
int launch_batch(int engine, int cls, int cvar, const BatchArgs& b, int grid, void* stream, int* occ);
int launch_batch_tails(int cls, const BatchArgs& b, void* stream);
struct TileGeom;
TileGeom batch_geom(int cls, int cvar);
int launch_fill(const FillArgs& a, int grid, void* stream);
int launch_tails(const FillArgs& a, void* stream);
// Sets a control block to its initial state on the stream (no host copy: a
// copy from pageable memory would wait for the stream).
int launch_ctrl_reset(Ctrl* ctrl, void* stream);
// Asynchronous fills: writes start + ctrl->next_pos to d_pos (halves: the
// device counted half-words, start + ceil(next_pos / 2); ~0 when the fill failed), and ORs the failure bits into sticky[0], counts failures in
// sticky[1] and keeps the first failure's tile in sticky[2].
int launch_finish(const Ctrl* ctrl, unsigned long long start, unsigned long long* d_pos, unsigned long long* sticky,
                  int halves, void* stream);
// Pairwise outputs from 2m base variates g: mode 0 beta X/(X+Y), 1 F
// (X/p0)/(Y/p1), 2 skew normal p0 + p1 (p2 |u0| + p3 u1).
int launch_pairs(const double* g, double* out, unsigned long long m, int mode, const double* p, void* stream);
// gradients (rp_grad.cu)
int grad_blocks();
// block partials (2 per block), the 2 results, then the gamma gradient's tables
size_t grad_scratch_doubles();
int launch_gamma_grad(const double* z, const double* g, size_t n, double alpha, double* dz, double* part, double* out,
                      void* stream);
int launch_beta_grad(const double* z, const double* g, size_t n, double a, double b, double* dza, double* dzb,
                     double* part, double* out, void* stream);
// Beta gradient through the gamma pair: dzda <- Y/(X+Y)^2 dzda (dX/da on
// entry), dzdb <- -X/(X+Y)^2 dzdb (dY/db on entry), and the two sums with g.
int launch_beta_compose(const double* x, const double* y, const double* g, size_t n, double* dzda, double* dzdb,
                        double* part, double* out, void* stream);
// Beta with equal shapes from 2m consecutive gammas g: z = X/(X+Y), and X, Y kept.
int launch_pairs_xy(const double* g, double* z, double* x, double* y, unsigned long long m, void* stream);
// Fixed scratch of the normal fill that allocates nothing
// (rp_static_scratch.cu).  Sized for at most kStaticMaxN outputs per call:
// a Philox normal fill of n outputs needs at most
// (1.0235 n + 8 sqrt(1.0235 n) + 64) / 32768 + 2 tiles (133 at the maximum)
// and n / 256 + 4096 tail entries, the bounds the allocating path uses.
constexpr unsigned long long kStaticMaxN = 1ull << 22;
constexpr unsigned long long kStaticTiles = 256;
constexpr unsigned long long kStaticTailCap = kStaticMaxN / 256 + 4096;
constexpr size_t kStaticCtrlWords = 32;
constexpr size_t kStaticWords = kStaticCtrlWords + kStaticTiles + kStaticTailCap * (sizeof(TailEntry) / 8);
static_assert(sizeof(Ctrl) <= kStaticCtrlWords * 8, "control block does not fit its slot");
static_assert(sizeof(TailEntry) % 8 == 0, "tail entries must be whole words");
int static_scratch_address(void** p);
int launch_log_cr(const double* x, double* y, unsigned long long n, void* stream);
int launch_exp_cr(const double* x, double* y, unsigned long long n, void* stream);
// Exact-decision fallback counts (rp_kernels.cu), 8 words; reset zeroes them.
int debug_counters(unsigned long long* out, int reset);
// Multivariate normal (rp_mvn.cu).
int launch_mvn_apply(int d, unsigned long long n, const double* mu, const double* L, const double* Z, double* X,
                     void* stream);
int mvn_grad_slices(int d, unsigned long long n, unsigned long long* slice);
int launch_mvn_grads(int d, unsigned long long n, const double* G, const double* Z, double* gmu, double* gL,
                     double* part, void* stream);
// Tile geometry and resources of a (engine, dist) kernel.
struct TileGeom { int nt, c, tile_words, smem_bytes; };
TileGeom tile_geom(int engine, int dist, int gamma_boost);   // gamma_boost: a gamma fill with alpha < 1
int occupancy_blocks(int engine, int dist, int epi);   // resident CTAs per SM
// One-time upload of ziggurat tables into device constant/global memory.
int upload_tables();

}  // namespace rp
