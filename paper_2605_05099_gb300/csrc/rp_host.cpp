// Host side of librp: argument checks, seeding and stream control
// (Randompack Sec. 2.3), jump tables, scratch management and the C ABI
// declared in include/rp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <unordered_map>
#include <mutex>
#include <string>
#include <vector>

#include "rp.h"
#include "rp_internal.h"

namespace rp {
struct ZigDev;
int upload_zig(const void* host2);
}  // namespace rp

namespace {

typedef unsigned long long u64;
typedef unsigned __int128 u128;

thread_local std::string g_err;
std::mutex g_mu;
std::atomic<unsigned long long> g_launches{0};

rp_status fail(rp_status code, const std::string& msg) {
  g_err = msg;
  return code;
}

rp_status cuda_fail(int e, const char* where) {
  return fail(RP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString((cudaError_t)e));
}

// The allocating entry points keep their device state (scratch, jump
// tables, the uploaded ziggurat tables, plans) for one device: the one
// current at their first call.  A call with another device current is
// refused before it launches anything.  Caller holds g_mu.
int g_dev = -1;
rp_status device_guard() {
  int d = 0;
  const int e = (int)cudaGetDevice(&d);
  if (e) return cuda_fail(e, "current device");
  if (g_dev < 0) g_dev = d;
  else if (d != g_dev)
    return fail(RP_ERR_PARAM, "this library's allocating entry points serve one device per process: first used on device " +
                                  std::to_string(g_dev) + ", now called with device " + std::to_string(d) + " current");
  return RP_OK;
}

// Test hooks of the device error paths (rp_debug_faults); zero: off.
struct DebugFaults {
  u64 spin_max = 0;     // look-back waits give up after this many spins
  u64 stall_tile1 = 0;  // tile (value - 1) of each launch publishes nothing
  u64 tail_cap = 0;     // tail queue capacity
  u64 tile_cap = 0;     // tiles per launch of the sampled (non one-word) fills
} g_faults;

// ---------------------------------------------------------------- seeding
// Seed and spawn key are hashed into a pool of four 32-bit words, then
// hashed out to the requested number of state words (Sec. 2.3; NumPy
// SeedSequence semantics, O'Neill's seed_seq design).
struct SeedSeq {
  static constexpr uint32_t kA = 0x43b0d7e5u, kMA = 0x931e8875u, kB = 0x8b51f9ddu, kMB = 0x58f38dedu;
  static constexpr uint32_t kL = 0xca01f9ddu, kR = 0x4973f715u;
  uint32_t pool[4];

  explicit SeedSeq(const std::vector<uint32_t>& ent) {
    uint32_t hc = kA;
    auto hash = [&hc](uint32_t v) {
      v ^= hc;
      hc *= kMA;
      v *= hc;
      return v ^ (v >> 16);
    };
    auto mix = [](uint32_t x, uint32_t y) {
      uint32_t r = kL * x - kR * y;
      return r ^ (r >> 16);
    };
    for (int i = 0; i < 4; ++i) pool[i] = hash(i < (int)ent.size() ? ent[i] : 0u);
    for (int s = 0; s < 4; ++s)
      for (int d = 0; d < 4; ++d)
        if (s != d) pool[d] = mix(pool[d], hash(pool[s]));
    for (size_t s = 4; s < ent.size(); ++s)
      for (int d = 0; d < 4; ++d) pool[d] = mix(pool[d], hash(ent[s]));
  }
  void words64(u64* out, int n) const {
    uint32_t hc = kB;
    for (int i = 0; i < 2 * n; ++i) {
      uint32_t v = pool[i & 3] ^ hc;
      hc *= kMB;
      v *= hc;
      v ^= v >> 16;
      if (i & 1) out[i / 2] |= (u64)v << 32;
      else out[i / 2] = v;
    }
  }
};

void append_u32(std::vector<uint32_t>& v, u64 x) {
  v.push_back((uint32_t)x);
  if (x >> 32) v.push_back((uint32_t)(x >> 32));
}

void seed_words(u64 seed, u64 stream, u64* out, int n) {
  std::vector<uint32_t> ent;
  append_u32(ent, seed);
  if (stream != RP_NO_STREAM) {
    while (ent.size() < 4) ent.push_back(0);
    append_u32(ent, stream);
  }
  SeedSeq(ent).words64(out, n);
}

// ---------------------------------------------------------------- xoshiro GF(2)
// 256x256 matrices over GF(2), column j = image of basis vector e_j.
struct Mat {
  u64 c[256][4];
};

void xo_step(u64 s[4]) {
  u64 t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = (s[3] << 45) | (s[3] >> 19);
}

void mat_vec(const Mat& M, const u64 v[4], u64 r[4]) {
  u64 a[4] = {0, 0, 0, 0};
  for (int w = 0; w < 4; ++w) {
    u64 x = v[w];
    while (x) {
      int b = __builtin_ctzll(x);
      const u64* col = M.c[64 * w + b];
      a[0] ^= col[0]; a[1] ^= col[1]; a[2] ^= col[2]; a[3] ^= col[3];
      x &= x - 1;
    }
  }
  memcpy(r, a, sizeof(a));
}

void mat_mul(const Mat& A, const Mat& B, Mat& out) {  // out = A B
  Mat tmp;
  for (int j = 0; j < 256; ++j) mat_vec(A, B.c[j], tmp.c[j]);
  out = tmp;
}

struct XoTables {
  std::vector<Mat> pow;        // pow[j] = T^(2^j), j < 192
  void* d_pow = nullptr;       // nibble tables of pow[0..63]
  std::map<u64, void*> d_stride;
};
XoTables* g_xo = nullptr;

void nibble_table(const Mat& M, std::vector<u64>& out) {  // 64 x 16 x 4 words
  out.assign(64 * 16 * 4, 0);
  for (int c = 0; c < 64; ++c)
    for (int v = 0; v < 16; ++v)
      for (int b = 0; b < 4; ++b)
        if (v >> b & 1)
          for (int k = 0; k < 4; ++k) out[(c * 16 + v) * 4 + k] ^= M.c[4 * c + b][k];
}

XoTables& xo() {
  if (!g_xo) {
    g_xo = new XoTables;
    g_xo->pow.resize(192);
    for (int j = 0; j < 256; ++j) {
      u64 e[4] = {0, 0, 0, 0};
      e[j >> 6] = 1ull << (j & 63);
      xo_step(e);
      memcpy(g_xo->pow[0].c[j], e, sizeof(e));
    }
    for (int j = 1; j < 192; ++j) mat_mul(g_xo->pow[j - 1], g_xo->pow[j - 1], g_xo->pow[j]);
  }
  return *g_xo;
}

void xo_jump(u64 s[4], u128 n) {
  XoTables& X = xo();
  for (int j = 0; j < 128 && n; ++j, n >>= 1)
    if (n & 1) mat_vec(X.pow[j], s, s);
}

void xo_jump_limbs(u64 s[4], const u64* limbs, int nl) {  // N = sum limbs[i] 2^(64 i), N < 2^192
  XoTables& X = xo();
  for (int i = 0; i < nl && i < 3; ++i)
    for (int b = 0; b < 64; ++b)
      if (limbs[i] >> b & 1) mat_vec(X.pow[64 * i + b], s, s);
}

int xo_device_pow(void** out) {
  XoTables& X = xo();
  if (!X.d_pow) {
    std::vector<u64> all(64 * 64 * 16 * 4), one;
    for (int j = 0; j < 64; ++j) {
      nibble_table(X.pow[j], one);
      memcpy(&all[(size_t)j * one.size()], one.data(), one.size() * 8);
    }
    int e = (int)cudaMalloc(&X.d_pow, all.size() * 8);
    if (e) { X.d_pow = nullptr; return e; }
    e = (int)cudaMemcpy(X.d_pow, all.data(), all.size() * 8, cudaMemcpyHostToDevice);
    if (e) return e;
  }
  *out = X.d_pow;
  return 0;
}

// T^N as a matrix, N < 2^64
void xo_power(u64 N, Mat& M) {
  XoTables& X = xo();
  memset(&M, 0, sizeof(M));
  for (int j = 0; j < 256; ++j) M.c[j][j >> 6] = 1ull << (j & 63);
  for (int j = 0; j < 64; ++j)
    if (N >> j & 1) mat_mul(X.pow[j], M, M);
}

int upload_tables(const std::vector<Mat>& mats, void** out) {
  std::vector<u64> all, one;
  for (const Mat& m : mats) {
    nibble_table(m, one);
    all.insert(all.end(), one.begin(), one.end());
  }
  void* d = nullptr;
  int e = (int)cudaMalloc(&d, all.size() * 8);
  if (e) return e;
  e = (int)cudaMemcpy(d, all.data(), all.size() * 8, cudaMemcpyHostToDevice);
  if (e) { cudaFree(d); return e; }
  *out = d;
  return 0;
}

// Device tables are cached per chunk length; the one-word fills pick their
// chunk length from n, so the caches keep at most kTableCache entries
// (cudaFree waits for the kernels that may still read an evicted table).
constexpr size_t kTableCache = 16;
template <class M>
void evict_one(M& m) {
  if (m.size() < kTableCache) return;
  cudaFree(m.begin()->second);
  m.erase(m.begin());
}

// nibble tables of T^(t C), t < nt (per-thread offsets inside a tile)
std::map<std::pair<u64, int>, void*> g_xo_thread;
int xo_device_thread(u64 C, int nt, void** out) {
  auto key = std::make_pair(C, nt);
  auto it = g_xo_thread.find(key);
  if (it == g_xo_thread.end()) {
    evict_one(g_xo_thread);
    std::vector<Mat> mats(nt);
    xo_power(0, mats[0]);
    Mat step;
    xo_power(C, step);
    for (int t = 1; t < nt; ++t) mat_mul(step, mats[t - 1], mats[t]);
    void* d = nullptr;
    int e = upload_tables(mats, &d);
    if (e) return e;
    it = g_xo_thread.emplace(key, d).first;
  }
  *out = it->second;
  return 0;
}

// nibble tables of T^(T 2^j), j < 16 (per-CTA base offsets)
std::map<u64, void*> g_xo_cta;
int xo_device_cta(u64 T, void** out) {
  auto it = g_xo_cta.find(T);
  if (it == g_xo_cta.end()) {
    evict_one(g_xo_cta);
    std::vector<Mat> mats(16);
    xo_power(T, mats[0]);
    for (int j = 1; j < 16; ++j) mat_mul(mats[j - 1], mats[j - 1], mats[j]);
    void* d = nullptr;
    int e = upload_tables(mats, &d);
    if (e) return e;
    it = g_xo_cta.emplace(T, d).first;
  }
  *out = it->second;
  return 0;
}

int xo_device_stride(u64 D, void** out) {
  XoTables& X = xo();
  auto it = X.d_stride.find(D);
  if (it == X.d_stride.end()) {
    Mat M;
    memset(&M, 0, sizeof(M));
    for (int j = 0; j < 256; ++j) M.c[j][j >> 6] = 1ull << (j & 63);
    for (int j = 0; j < 64; ++j)
      if (D >> j & 1) mat_mul(X.pow[j], M, M);
    std::vector<u64> tab;
    nibble_table(M, tab);
    void* d = nullptr;
    int e = (int)cudaMalloc(&d, tab.size() * 8);
    if (e) return e;
    e = (int)cudaMemcpy(d, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice);
    if (e) return e;
    it = X.d_stride.emplace(D, d).first;
  }
  *out = it->second;
  return 0;
}

// ---------------------------------------------------------------- PCG64 affine powers
constexpr u64 kPcgMult = 0xda942042e4dd58b5ull;
struct Aff {
  u128 A, G;  // x -> A x + G inc
};
Aff aff_pow2(int j) {  // 2^j steps
  Aff r{(u128)kPcgMult, 1};
  for (int i = 0; i < j; ++i) r = Aff{r.A * r.A, r.G * (r.A + 1)};
  return r;
}
Aff aff_steps(u128 n) {
  Aff acc{1, 0};
  Aff cur{(u128)kPcgMult, 1};
  while (n) {
    if (n & 1) acc = Aff{acc.A * cur.A, acc.G * cur.A + cur.G};
    cur = Aff{cur.A * cur.A, cur.G * (cur.A + 1)};
    n >>= 1;
  }
  return acc;
}
u64* g_pcg_pow = nullptr;
int pcg_device_pow(u64** out) {
  if (!g_pcg_pow) {
    std::vector<u64> h(64 * 4);
    for (int j = 0; j < 64; ++j) {
      Aff a = aff_pow2(j);
      h[4 * j] = (u64)(a.A >> 64); h[4 * j + 1] = (u64)a.A;
      h[4 * j + 2] = (u64)(a.G >> 64); h[4 * j + 3] = (u64)a.G;
    }
    int e = (int)cudaMalloc((void**)&g_pcg_pow, h.size() * 8);
    if (e) { g_pcg_pow = nullptr; return e; }
    e = (int)cudaMemcpy(g_pcg_pow, h.data(), h.size() * 8, cudaMemcpyHostToDevice);
    if (e) return e;
  }
  *out = g_pcg_pow;
  return 0;
}

// ---------------------------------------------------------------- engine states
// Counter-based engines address words directly: a fill starts at a word
// offset instead of jumping its state.
bool counter_engine(int engine) { return engine == RP_PHILOX4X32_10 || engine == RP_PHILOX4X64_10; }
// xoshiro256++ and xoshiro256** share the state, the seeding and the jumps.
bool xoshiro_engine(int engine) { return engine == RP_XOSHIRO256PP || engine == RP_XOSHIRO256SS; }

constexpr u128 kPcgMult128 = ((u128)0x2360ED051FC65DA4ull << 64) | 0x4385DF649FCCF645ull;

rp_status seed_state(int engine, u64 seed, u64 stream, u64 s[4]) {
  u64 w[4] = {0, 0, 0, 0};
  if (xoshiro_engine(engine)) {
    seed_words(seed, stream, w, 4);
    if ((w[0] | w[1] | w[2] | w[3]) == 0) return fail(RP_ERR_SEED, "seeding gave an all-zero xoshiro state");
    memcpy(s, w, sizeof(w));
  } else if (engine == RP_PCG64DXSM) {
    seed_words(seed, stream, w, 4);
    u128 initstate = ((u128)w[0] << 64) | w[1], initseq = ((u128)w[2] << 64) | w[3];
    u128 inc = (initseq << 1) | 1u;
    u128 st = inc + initstate;
    st = st * kPcgMult128 + inc;
    s[0] = (u64)(st >> 64); s[1] = (u64)st; s[2] = (u64)(inc >> 64); s[3] = (u64)inc;
  } else if (engine == RP_PHILOX4X32_10) {
    seed_words(seed, stream, w, 3);
    s[0] = w[0]; s[1] = w[1]; s[2] = w[2]; s[3] = 0;
  } else if (engine == RP_PHILOX4X64_10) {
    // NumPy's Philox seeding: key = two seed-sequence words, counter 0
    seed_words(seed, stream, w, 2);
    s[0] = 0; s[1] = 0; s[2] = w[0]; s[3] = w[1];
  } else {
    return fail(RP_ERR_ENGINE, "unknown engine id " + std::to_string(engine));
  }
  return RP_OK;
}

void jump_state(int engine, u64 s[4], u128 delta) {
  if (xoshiro_engine(engine)) {
    xo_jump(s, delta);
  } else if (engine == RP_PCG64DXSM) {
    Aff a = aff_steps(delta);
    u128 st = ((u128)s[0] << 64) | s[1], inc = ((u128)s[2] << 64) | s[3];
    st = a.A * st + a.G * inc;
    s[0] = (u64)(st >> 64); s[1] = (u64)st;
  } else {
    // blocks of two (Philox4x32) or four (Philox4x64) words: a delta that is
    // not a whole number of blocks cannot be expressed in the state words;
    // callers use the word offset instead (rp_fill_* take pos)
    u128 c = (((u128)s[1] << 64) | s[0]) + delta / (engine == RP_PHILOX4X64_10 ? 4 : 2);
    s[0] = (u64)c; s[1] = (u64)(c >> 64);
  }
}

// ---------------------------------------------------------------- ziggurat upload
#include "zig_tables.inc"

struct ZigHost {  // same layout as the device-side ZigDev
  u64 k[256];
  u64 msh[256];
  double f[256];
  int we[256];
  int wtz[256];
  float ff[256];
  float fd[256];
  float wf[256];
  double w[256];    // w_i
  double R;
  float Rf;
  float pad;
};

void fill_zig(ZigHost& z, const unsigned long long* K, const double* W, const double* F, double R) {
  for (int i = 0; i < 256; ++i) {
    z.k[i] = K[i];
    z.f[i] = F[i];
    u64 bits;
    memcpy(&bits, &W[i], 8);
    int be = (int)((bits >> 52) & 0x7ff);
    u64 m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    z.msh[i] = m << 11;
    z.we[i] = be - 1075;
    z.wtz[i] = __builtin_ctzll(m);
    z.ff[i] = (float)F[i];
    z.fd[i] = i ? (float)(F[i - 1] - F[i]) : 0.0f;
    z.wf[i] = (float)W[i];
    z.w[i] = W[i];
  }
  z.R = R;
  z.Rf = (float)R;
  z.pad = 0.0f;
}

bool g_zig_ready = false;
int ensure_zig() {
  if (g_zig_ready) return 0;
  ZigHost z[2];
  fill_zig(z[0], RP_ZIG_N_K, RP_ZIG_N_W, RP_ZIG_N_F, RP_ZIG_N_R);
  fill_zig(z[1], RP_ZIG_E_K, RP_ZIG_E_W, RP_ZIG_E_F, RP_ZIG_E_R);
  int e = rp::upload_zig(z);
  if (!e) g_zig_ready = true;
  return e;
}

// ---------------------------------------------------------------- scratch
struct Scratch {
  unsigned long long* status = nullptr;
  size_t cap = 0;
  rp::Ctrl* ctrl = nullptr;
  rp::Ctrl* h_ctrl = nullptr;  // pinned
  rp::TailEntry* tailq = nullptr;
  size_t tail_cap = 0;
  unsigned long long* park = nullptr;  // one-pass bounded fill: each CTA's parked runs
  size_t park_cap = 0;
};
Scratch g_scr;

// Asynchronous position writes.  A fill whose *pos is host-pinned memory
// enqueues its kernels, a finishing kernel that forms the end position on the
// device, and a copy of it to *pos, and returns without waiting: *pos is
// valid after the stream is synchronised (all ones if the fill failed; then
// rp_async_status gives the reason).  Each such *pos has an event; a later
// call that reads the same *pos first waits for that event, so chaining fills
// through one pinned word stays correct.  The scratch (tile status words,
// control block, tail queue) is shared: a fill on another stream than the
// last user of it waits for that user's event on the device, not on the host.
struct AsyncState {
  u64* dev = nullptr;                       // [0] end position, [1..3] sticky failure bits, count, info
  std::unordered_map<u64*, cudaEvent_t> pending;
  std::vector<cudaEvent_t> free_ev;
  cudaEvent_t scr_ev = nullptr;             // recorded after the last use of the scratch
  void* scr_stream = nullptr;
  bool scr_used = false;
};
AsyncState g_async;
u64* g_f1 = nullptr;   // device scratch word of the float uniform fill's odd last output

cudaEvent_t take_event() {
  if (!g_async.free_ev.empty()) {
    cudaEvent_t e = g_async.free_ev.back();
    g_async.free_ev.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  return e;
}

bool pinned_host(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

// Waits for an asynchronous write still pending on *pos.
int wait_pending_pos(u64* pos) {
  auto it = g_async.pending.find(pos);
  if (it == g_async.pending.end()) return 0;
  const int e = (int)cudaEventSynchronize(it->second);
  g_async.free_ev.push_back(it->second);
  g_async.pending.erase(it);
  return e;
}

// Orders this stream's use of the shared scratch after the previous user's.
int scratch_acquire(void* cstream) {
  if (!g_async.scr_used || g_async.scr_stream == cstream) return 0;
  return (int)cudaStreamWaitEvent((cudaStream_t)cstream, g_async.scr_ev, 0);
}

int scratch_release(void* cstream) {
  if (!g_async.scr_ev) {
    const int e = (int)cudaEventCreateWithFlags(&g_async.scr_ev, cudaEventDisableTiming);
    if (e) return e;
  }
  g_async.scr_stream = cstream;
  g_async.scr_used = true;
  return (int)cudaEventRecord(g_async.scr_ev, (cudaStream_t)cstream);
}

int ensure_async_dev() {
  if (g_async.dev) return 0;
  int e = (int)cudaMalloc((void**)&g_async.dev, 4 * sizeof(u64));
  if (!e) e = (int)cudaMemset(g_async.dev, 0, 4 * sizeof(u64));
  if (e) g_async.dev = nullptr;
  return e;
}

int ensure_park(size_t words) {
  if (words > g_scr.park_cap) {
    if (g_scr.park) cudaFree(g_scr.park);
    int e = (int)cudaMalloc((void**)&g_scr.park, words * 8);
    if (e) { g_scr.park = nullptr; g_scr.park_cap = 0; return e; }
    g_scr.park_cap = words;
  }
  return 0;
}

int ensure_tailq(size_t cap) {
  if (cap > g_scr.tail_cap) {
    if (g_scr.tailq) cudaFree(g_scr.tailq);
    int e = (int)cudaMalloc((void**)&g_scr.tailq, cap * sizeof(rp::TailEntry));
    if (e) { g_scr.tailq = nullptr; g_scr.tail_cap = 0; return e; }
    g_scr.tail_cap = cap;
  }
  return 0;
}

int ensure_scratch(size_t tiles) {
  if (!g_scr.ctrl) {
    int e = (int)cudaMalloc((void**)&g_scr.ctrl, sizeof(rp::Ctrl));
    if (e) return e;
    e = (int)cudaMallocHost((void**)&g_scr.h_ctrl, sizeof(rp::Ctrl));
    if (e) return e;
  }
  if (tiles > g_scr.cap) {
    if (g_scr.status) cudaFree(g_scr.status);
    size_t cap = tiles < 4096 ? 4096 : tiles + tiles / 2;
    int e = (int)cudaMalloc((void**)&g_scr.status, cap * 8);
    if (e) { g_scr.status = nullptr; g_scr.cap = 0; return e; }
    g_scr.cap = cap;
  }
  return 0;
}

int g_sms = 0;
int sm_count() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

std::map<std::pair<int, int>, int> g_occ;

// Marsaglia-Tsang constants (Sec. 3.1, gamma): d = s - 1/3, c = 1/sqrt(9 d),
// s = alpha (alpha >= 1) or alpha + 1 with the boost U^(1/alpha).
rp::MTParams mt_params(double alpha) {
  rp::MTParams p{};
  double s = alpha >= 1.0 ? alpha : alpha + 1.0;
  volatile double third = 1.0 / 3.0;
  p.d = s - third;
  volatile double nine_d = 9.0 * p.d;
  volatile double sq = std::sqrt(nine_d);
  p.c = 1.0 / sq;
  p.alpha = alpha;
  p.df = (float)p.d;
  p.cf = (float)p.c;
  p.boost = alpha < 1.0 ? 1 : 0;
  return p;
}

double gamma_wpv(const rp::MTParams& p) { return p.boost ? 3.2 : 2.15; }

// expected words per variate (upper estimate used to size one launch)
double words_per_variate(int dist, const rp::SampArgs& sp) {
  switch (dist) {
    case rp::D_BOUNDED: return sp.m ? 1.0 / (1.0 - (double)sp.thresh * 0x1.0p-64) : 1.0;
    case rp::D_NORMAL: return 1.0235;
    case rp::D_EXP: return 1.036;
    case rp::D_NORMALF: return 1.0235 / 2;   // half-words: words per variate
    case rp::D_EXPF: return 1.036 / 2;
    case rp::D_GAMMA: return gamma_wpv(sp.ga);
    case rp::D_BETA: return gamma_wpv(sp.ga) + gamma_wpv(sp.gb);
    case rp::D_T: return 1.0235 + gamma_wpv(sp.ga);
    default: return 1.0;
  }
}

// Fill from explicit state words (the engine at word 0 of the stream; *pos
// words in).  Caller holds g_mu.
rp_status run_fill_state_locked(int engine, const u64 s_in[4], u64* pos, size_t n, int dist, const rp::SampArgs& sp,
                                void* d_out, void* cstream, u64* first_reject = nullptr, int async_mode = -1) {
  if (async_mode < 0) {
    // top-level call: an earlier asynchronous write to *pos lands first
    int e = wait_pending_pos(pos);
    if (e) return cuda_fail(e, "pending position write");
    async_mode = pinned_host(pos) ? 1 : 0;
  }
  if (dist == rp::D_BOUNDED && !async_mode && (double)n * ((double)sp.thresh * 0x1.0p-64) < 0.05) {
    // Rejections are unlikely in this fill: one pass writes word p's value
    // at output p and reports the first rejected word q.  Outputs before q
    // are final (the serial sampler gives the same values up to its first
    // rejection); from word q + 1 the exact two-pass fill takes over.
    u64 q = ~0ull, p0 = *pos;
    rp_status st = run_fill_state_locked(engine, s_in, &p0, n, rp::D_BOUNDED_ONE, sp, d_out, cstream, &q, 0);
    if (st) return st;
    if (q >= n) { *pos += n; return RP_OK; }
    u64 p1 = *pos + q + 1;
    st = run_fill_state_locked(engine, s_in, &p1, n - q, rp::D_BOUNDED, sp, (char*)d_out + q * 8, cstream, nullptr, 0);
    if (st) return st;
    *pos = p1;
    return RP_OK;
  }
  u64 s[4] = {s_in[0], s_in[1], s_in[2], s_in[3]};
  rp_status dg = device_guard();
  if (dg) return dg;
  int e = ensure_zig();
  if (e) return cuda_fail(e, "ziggurat table upload");

  rp::FillArgs a;
  memset(&a, 0, sizeof(a));
  a.eng.engine = engine;
  a.dist = dist;
  a.sp = sp;
  rp::TileGeom tg = rp::tile_geom(engine, dist, dist == rp::D_GAMMA && sp.ga.boost);
  const u64 T = (u64)tg.tile_words;
  auto key = std::make_pair(engine, dist | (sp.epi ? 256 : 0));   // transformed fills run other kernels
  if (!g_occ.count(key)) g_occ[key] = rp::occupancy_blocks(engine, dist, sp.epi);
  int occ = g_occ[key] > 0 ? g_occ[key] : 1;
  const bool trivial = (dist == rp::D_U64 || dist == rp::D_UNIFORM || dist == rp::D_BOUNDED_ONE || dist == rp::D_UNIFORMF2 ||
                        dist == rp::D_UNIFORM52 || dist == rp::D_FOLD);
  const bool one_pass_check = dist == rp::D_BOUNDED_ONE;
  if (!trivial || one_pass_check) {
    e = scratch_acquire(cstream);
    if (!e && async_mode) e = ensure_async_dev();
    if (e) return cuda_fail(e, "scratch ordering");
  }

  // Half-word fills (float ziggurats) count positions in half-words on the
  // device; `half` is the first half-word of the next launch within word cur.
  const bool halves = dist == rp::D_NORMALF || dist == rp::D_EXPF;
  int half = 0;
  u64 cur = *pos;
  size_t done = 0;
  const size_t esz = halves ? 4 : 8;
  for (int launch = 0; done < n; ++launch) {
    if (launch > 64) return fail(RP_ERR_INTERNAL, "too many continuation launches");
    size_t left = n - done;
    double wpv = words_per_variate(dist, sp);
    double need = (double)left * wpv + 8.0 * std::sqrt((double)left * (wpv > 1.0 ? wpv : 1.0)) + 64.0;
    u64 C = (u64)tg.c, T = (u64)tg.tile_words;
    u64 tiles, grid;
    if (trivial) {
      // one tile per CTA: each thread streams one contiguous range of at
      // least 64 words (a multiple of 16; of 64 for xoshiro, whose per-thread
      // jump tables are built per chunk length).  Philox4x32-10's kernel
      // strides over blocks instead and uses only the grid.
      const u64 nt = (u64)tg.nt, q = xoshiro_engine(engine) ? 64 : 16;
      grid = std::max<u64>(1, std::min<u64>((u64)sm_count() * occ, (left + nt * 64 - 1) / (nt * 64)));
      C = ((left + grid * nt - 1) / (grid * nt) + q - 1) / q * q;
      T = nt * C;
      tiles = grid;
    } else {
      tiles = (u64)(need / (double)T) + 2;
      if (g_faults.tile_cap && tiles > g_faults.tile_cap) tiles = g_faults.tile_cap;
      grid = std::min<u64>(tiles, (u64)sm_count() * occ);
    }
    // engine at word `cur`
    u64 s0[4];
    memcpy(s0, s, sizeof(s0));
    a.eng.word0 = 0;
    if (counter_engine(engine)) {
      a.eng.word0 = cur;
    } else {
      jump_state(engine, s0, (u128)cur);
    }
    memcpy(a.eng.s, s0, sizeof(s0));
    a.eng.stride = grid * T;
    a.eng.tile_words = T;
    a.eng.chunk_words = C;
    if (grid > 65535) return fail(RP_ERR_INTERNAL, "grid too large for the CTA jump tables");
    if (xoshiro_engine(engine)) {
      e = xo_device_pow((void**)&a.eng.gf2_pow);
      if (!e && !trivial) e = xo_device_stride(a.eng.stride, (void**)&a.eng.gf2_stride);
      if (!e) e = xo_device_thread(C, tg.nt, (void**)&a.eng.gf2_thread);
      if (!e) e = xo_device_cta(T, (void**)&a.eng.gf2_cta);
      if (e) return cuda_fail(e, "jump tables");
    } else if (engine == RP_PCG64DXSM) {
      e = pcg_device_pow((u64**)&a.eng.pcg_pow);
      if (e) return cuda_fail(e, "jump tables");
      Aff d = aff_steps((u128)a.eng.stride);
      a.eng.pcg_stride[0] = (u64)(d.A >> 64); a.eng.pcg_stride[1] = (u64)d.A;
      a.eng.pcg_stride[2] = (u64)(d.G >> 64); a.eng.pcg_stride[3] = (u64)d.G;
    }
    a.n = left;
    a.n_tiles = tiles;
    a.out = (char*)d_out + done * esz;
    a.sp.half0 = half;
    if (sp.outx) {   // beta keeping its gamma pairs: the same output index
      a.sp.outx = sp.outx + done;
      a.sp.outy = sp.outy + done;
    }
    if (!trivial || one_pass_check) {
      e = ensure_scratch(tiles);
      const bool queued = dist == rp::D_NORMAL || dist == rp::D_EXP || dist == rp::D_GAMMA || dist == rp::D_BETA ||
                          dist == rp::D_T || dist == rp::D_NORMALF || dist == rp::D_EXPF;
      if (!e && queued) e = ensure_tailq(left / 256 + 4096);
      if (!e && dist == rp::D_BOUNDED) e = ensure_park((size_t)(grid * T));
      if (e) return fail(RP_ERR_NOMEM, std::string("scratch allocation: ") + cudaGetErrorString((cudaError_t)e));
      a.tile_status = g_scr.status;
      a.ctrl = g_scr.ctrl;
      a.tailq = g_scr.tailq;
      a.tail_cap = queued ? g_scr.tail_cap : 0;
      if (g_faults.tail_cap && a.tail_cap > g_faults.tail_cap) a.tail_cap = g_faults.tail_cap;
      a.tail_count = &g_scr.ctrl->n_tail;
      a.park = g_scr.park;
      a.spin_max = g_faults.spin_max;
      a.stall_tile1 = g_faults.stall_tile1;
      e = (int)cudaMemsetAsync(g_scr.status, 0, tiles * 8, (cudaStream_t)cstream);
      if (!e) e = rp::launch_ctrl_reset(g_scr.ctrl, cstream);
      if (e) return cuda_fail(e, "scratch reset");
      g_launches.fetch_add(1);
    }
    e = rp::launch_fill(a, (int)grid, cstream);
    if (e) return cuda_fail(e, "kernel launch");
    g_launches.fetch_add(1);
    if (a.tail_cap) {
      e = rp::launch_tails(a, cstream);
      if (e) return cuda_fail(e, "tail kernel launch");
      g_launches.fetch_add(1);
    }
    if (trivial) {
      // every word is an output: the end position is known here, and
      // nothing needs to come back (the one-pass bounded check excepted)
      if (one_pass_check) {
        e = (int)cudaMemcpyAsync(g_scr.h_ctrl, g_scr.ctrl, sizeof(rp::Ctrl), cudaMemcpyDeviceToHost, (cudaStream_t)cstream);
        if (!e) e = scratch_release(cstream);
        if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cstream);
        if (e) return cuda_fail(e, "fill");
        if (first_reject) *first_reject = g_scr.h_ctrl->first_reject;
      }
      done = n;
      cur += left;
      break;
    }
    if (async_mode) {
      // one launch, sized above with an eight-sigma margin; the device forms
      // the end position and the copy lands in the pinned *pos
      e = rp::launch_finish(g_scr.ctrl, cur, g_async.dev, g_async.dev + 1, halves ? 1 : 0, cstream);
      if (e) return cuda_fail(e, "finishing kernel launch");
      g_launches.fetch_add(1);
      e = (int)cudaMemcpyAsync(pos, g_async.dev, sizeof(u64), cudaMemcpyDeviceToHost, (cudaStream_t)cstream);
      if (!e) e = scratch_release(cstream);
      cudaEvent_t ev = e ? nullptr : take_event();
      if (!e && !ev) e = (int)cudaErrorMemoryAllocation;
      if (!e) e = (int)cudaEventRecord(ev, (cudaStream_t)cstream);
      if (e) return cuda_fail(e, "asynchronous position write");
      if (g_async.pending.size() >= 256) {
        // positions never read again: recycle the events that have fired
        for (auto it = g_async.pending.begin(); it != g_async.pending.end();) {
          if (cudaEventQuery(it->second) == cudaSuccess) {
            g_async.free_ev.push_back(it->second);
            it = g_async.pending.erase(it);
          } else {
            ++it;
          }
        }
        cudaGetLastError();
      }
      g_async.pending[pos] = ev;
      return RP_OK;
    }
    e = (int)cudaMemcpyAsync(g_scr.h_ctrl, g_scr.ctrl, sizeof(rp::Ctrl), cudaMemcpyDeviceToHost, (cudaStream_t)cstream);
    if (!e) e = scratch_release(cstream);
    if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cstream);
    if (e) return cuda_fail(e, "fill");
    const rp::Ctrl& c = *g_scr.h_ctrl;
    if (c.err) {
      char buf[320];
      const bool merge = dist == rp::D_BETA || dist == rp::D_GAMMA || dist == rp::D_T;
      snprintf(buf, sizeof buf, "device check failed (bits 0x%x, tile %llu)%s", c.err, (unsigned long long)c.err_info,
               (c.err & rp::E_NOSYNC) && merge
                   ? ": no merge point within the 64 chunks a walk may cross; the two gamma shapes of this beta "
                     "or F fill consume words alike too often (shapes nearly equal, or both large and close)"
                   : "");
      return fail(c.err & rp::E_TIMEOUT ? RP_ERR_TIMEOUT : RP_ERR_INTERNAL, buf);
    }
    if (c.total == 0 && c.next_pos == 0 && c.done_tile == ~0ull) return fail(RP_ERR_INTERNAL, "launch produced no output");
    done = c.done_tile != ~0ull ? n : done + c.total;
    if (halves) {
      const u64 h = c.next_pos;   // half-words from the low half of word cur (the launch began at `half`)
      cur += h >> 1;
      half = (int)(h & 1);
    } else {
      cur += c.next_pos;
    }
  }
  // a half-word fill that ends on a low half leaves the high half unused
  *pos = cur + (u64)half;
  return RP_OK;
}

// Output alignment: the element size (4 for the float fills, else 8).
rp_status check_fill_args(int engine, u64* pos, size_t n, void* d_out, int align = 8) {
  if (!pos) return fail(RP_ERR_NULL, "pos is NULL");
  if (n == 0) return RP_OK;
  if (!d_out) return fail(RP_ERR_NULL, "output pointer is NULL");
  if ((uintptr_t)d_out & (uintptr_t)(align - 1))
    return fail(RP_ERR_PARAM, "output pointer must be " + std::to_string(align) + "-byte aligned");
  if (engine < 1 || engine > 5) return fail(RP_ERR_ENGINE, "unknown engine id " + std::to_string(engine));
  return RP_OK;
}

rp_status run_fill(int engine, u64 seed, u64 stream, u64* pos, size_t n, int dist, const rp::SampArgs& sp,
                   void* d_out, void* cstream) {
  rp_status st = check_fill_args(engine, pos, n, d_out, (dist == rp::D_NORMALF || dist == rp::D_EXPF) ? 4 : 8);
  if (st || n == 0) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  u64 s[4] = {0, 0, 0, 0};
  st = seed_state(engine, seed, stream, s);
  if (st) return st;
  return run_fill_state_locked(engine, s, pos, n, dist, sp, d_out, cstream);
}

// Two base variates per output, consecutive in the stream: a base fill of 2n
// (in blocks, to bound the scratch) and the pairwise kernel (launch_pairs).
rp_status pairs_fill(int engine, u64 seed, u64 stream, u64* pos, size_t n, int base, const rp::SampArgs& sb, int mode,
                     const double* q, double* d_out, void* cuda_stream) {
  rp_status st = check_fill_args(engine, pos, n, d_out);
  if (st || n == 0) return st;
  const size_t blk = (size_t)1 << 26;   // pairs per block: 2^27 base variates keep the GPU full (1 GiB scratch)
  double* tmp = nullptr;
  size_t cap = std::min(n, blk);
  int e = (int)cudaMalloc((void**)&tmp, cap * 2 * sizeof(double));
  if (e) return fail(RP_ERR_NOMEM, "pair scratch allocation failed");
  u64 p = *pos;
  for (size_t done = 0; done < n && st == RP_OK; done += cap) {
    size_t m = std::min(cap, n - done);
    st = run_fill(engine, seed, stream, &p, 2 * m, base, sb, tmp, cuda_stream);
    if (st) break;
    e = rp::launch_pairs(tmp, d_out + done, m, mode, q, cuda_stream);
    if (!e) g_launches.fetch_add(1);
    if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e) st = cuda_fail(e, "pairwise outputs");
  }
  cudaFree(tmp);
  if (st == RP_OK) *pos = p;
  return st;
}

}  // namespace

extern "C" {

const char* rp_last_error(void) { return g_err.c_str(); }

rp_status rp_async_status(void* cuda_stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_async.dev) return RP_OK;
  int e = cuda_stream ? (int)cudaStreamSynchronize((cudaStream_t)cuda_stream) : (int)cudaDeviceSynchronize();
  u64 h[4] = {0, 0, 0, 0};
  if (!e) e = (int)cudaMemcpy(h, g_async.dev, sizeof h, cudaMemcpyDeviceToHost);
  if (e) return cuda_fail(e, "asynchronous fill status");
  if (!h[2]) return RP_OK;
  e = (int)cudaMemset(g_async.dev + 1, 0, 3 * sizeof(u64));
  if (e) return cuda_fail(e, "asynchronous fill status reset");
  char buf[256];
  snprintf(buf, sizeof buf, "%llu asynchronous fill(s) failed (device bits 0x%llx%s%s; first at tile %llu)",
           (unsigned long long)h[2], (unsigned long long)h[1], (h[1] & rp::E_TIMEOUT) ? ", a bounded wait gave up" : "",
           (h[1] & rp::E_INCOMPLETE) ? ", ran out of the planned tiles" : "", (unsigned long long)h[3]);
  return fail((h[1] & rp::E_TIMEOUT) ? RP_ERR_TIMEOUT : RP_ERR_INTERNAL, buf);
}
const char* rp_version(void) { return "rp 0.1 (sm_103a)"; }
uint64_t rp_kernel_launches(void) { return g_launches.load(); }

rp_status rp_fill_u64(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, uint64_t* d_out,
                      void* cuda_stream) {
  rp::SampArgs sp{};
  return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_U64, sp, d_out, cuda_stream);
}

rp_status rp_engine_fold(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, uint64_t* d_fold,
                         void* cuda_stream) {
  rp_status st = check_fill_args(engine, (u64*)pos, n, d_fold);
  if (st || n == 0) return st;
  const int e = (int)cudaMemsetAsync(d_fold, 0, sizeof(uint64_t), (cudaStream_t)cuda_stream);
  if (e) return cuda_fail(e, "fold reset");
  rp::SampArgs sp;
  memset(&sp, 0, sizeof(sp));
  return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_FOLD, sp, d_fold, cuda_stream);
}

rp_status rp_fill_uniform(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, double* d_out,
                          void* cuda_stream) {
  rp::SampArgs sp{};
  return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_UNIFORM, sp, d_out, cuda_stream);
}

rp_status rp_fill_uniform52(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, double* d_out,
                            void* cuda_stream) {
  rp::SampArgs sp{};
  return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_UNIFORM52, sp, d_out, cuda_stream);
}

rp_status rp_fill_bounded(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, uint64_t m,
                          uint64_t* d_out, void* cuda_stream) {
  rp::SampArgs sp{};
  sp.m = m;
  if (m == 0) return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_U64, sp, d_out, cuda_stream);
  sp.thresh = (0 - m) % m;
  return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_BOUNDED, sp, d_out, cuda_stream);
}

rp_status rp_fill_normal(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, double* d_out,
                         void* cuda_stream) {
  rp::SampArgs sp{};
  return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_NORMAL, sp, d_out, cuda_stream);
}

rp_status rp_fill_exp(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, double* d_out,
                      void* cuda_stream) {
  rp::SampArgs sp{};
  return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_EXP, sp, d_out, cuda_stream);
}

rp_status rp_fill_normalf(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, float* d_out,
                          void* cuda_stream) {
  rp::SampArgs sp{};
  return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_NORMALF, sp, d_out, cuda_stream);
}

rp_status rp_fill_expf(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, float* d_out,
                       void* cuda_stream) {
  rp::SampArgs sp{};
  return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_EXPF, sp, d_out, cuda_stream);
}

// Float uniforms: two per word, each word's pair written as 8 bytes; an odd
// n takes the low half of one more word, through a one-word fill into a
// scratch word and a 4-byte device copy.
rp_status rp_fill_uniformf(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, float* d_out,
                           void* cuda_stream) {
  rp_status st = check_fill_args(engine, (u64*)pos, n, d_out);
  if (st || n == 0) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  u64 s[4] = {0, 0, 0, 0};
  st = seed_state(engine, seed, stream, s);
  if (st) return st;
  rp::SampArgs sp{};
  const size_t pairs = n / 2;
  if (pairs) {
    st = run_fill_state_locked(engine, s, (u64*)pos, pairs, rp::D_UNIFORMF2, sp, d_out, cuda_stream);
    if (st) return st;
  }
  if (n & 1) {
    if (!g_f1) {
      const int e = (int)cudaMalloc((void**)&g_f1, sizeof(u64));
      if (e) { g_f1 = nullptr; return fail(RP_ERR_NOMEM, "scratch word allocation failed"); }
    }
    // the scratch word is shared: order its use as the fill scratch's
    int e = scratch_acquire(cuda_stream);
    if (e) return cuda_fail(e, "scratch ordering");
    st = run_fill_state_locked(engine, s, (u64*)pos, 1, rp::D_UNIFORMF2, sp, g_f1, cuda_stream);
    if (st) return st;
    e = (int)cudaMemcpyAsync(d_out + (n - 1), g_f1, sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)cuda_stream);
    if (!e) e = scratch_release(cuda_stream);
    if (e) return cuda_fail(e, "float uniform");
  }
  return RP_OK;
}

rp_status rp_fill_gamma(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, double alpha,
                        double* d_out, void* cuda_stream) {
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(RP_ERR_PARAM, "gamma shape must be positive and finite");
  rp::SampArgs sp{};
  sp.ga = mt_params(alpha);
  return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_GAMMA, sp, d_out, cuda_stream);
}

rp_status rp_fill_beta(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, double a, double b,
                       double* d_out, void* cuda_stream) {
  if (!(a > 0.0) || !(b > 0.0) || !std::isfinite(a) || !std::isfinite(b))
    return fail(RP_ERR_PARAM, "beta parameters must be positive and finite");
  rp::SampArgs sp{};
  sp.ga = mt_params(a);
  sp.gb = mt_params(b);
  if (a != b) return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_BETA, sp, d_out, cuda_stream);
  // Equal shapes: X and Y are consecutive Gamma(a) variates of the stream, so
  // the fill is a gamma fill of 2n followed by the pairwise ratio.
  rp::SampArgs sg{};
  sg.ga = sp.ga;
  return pairs_fill(engine, seed, stream, (u64*)pos, n, rp::D_GAMMA, sg, 0, nullptr, d_out, cuda_stream);
}

// Beta(a, b) that also keeps each output's gamma pair (X, Y): unequal shapes
// store them from the merge kernel; equal shapes take a gamma fill of 2n and
// a pairwise kernel, as rp_fill_beta does.
rp_status rp_fill_beta_xy(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, size_t n, double a, double b,
                          double* d_z, double* d_x, double* d_y, void* cuda_stream) {
  if (!(a > 0.0) || !(b > 0.0) || !std::isfinite(a) || !std::isfinite(b))
    return fail(RP_ERR_PARAM, "beta parameters must be positive and finite");
  if (n && (!d_x || !d_y)) return fail(RP_ERR_NULL, "d_x/d_y is NULL");
  if (((uintptr_t)d_x | (uintptr_t)d_y) & 7) return fail(RP_ERR_PARAM, "d_x/d_y must be 8-byte aligned");
  rp::SampArgs sp{};
  sp.ga = mt_params(a);
  sp.gb = mt_params(b);
  if (a != b) {
    sp.outx = d_x;
    sp.outy = d_y;
    return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_BETA, sp, d_z, cuda_stream);
  }
  rp_status st = check_fill_args(engine, (u64*)pos, n, d_z);
  if (st || n == 0) return st;
  const size_t blk = (size_t)1 << 26;
  double* tmp = nullptr;
  const size_t cap = std::min(n, blk);
  int e = (int)cudaMalloc((void**)&tmp, cap * 2 * sizeof(double));
  if (e) return fail(RP_ERR_NOMEM, "beta scratch allocation failed");
  u64 p = *pos;
  rp::SampArgs sg{};
  sg.ga = sp.ga;
  for (size_t done = 0; done < n && st == RP_OK; done += cap) {
    const size_t m = std::min(cap, n - done);
    st = run_fill(engine, seed, stream, &p, 2 * m, rp::D_GAMMA, sg, tmp, cuda_stream);
    if (st) break;
    e = rp::launch_pairs_xy(tmp, d_z + done, d_x + done, d_y + done, m, cuda_stream);
    if (!e) g_launches.fetch_add(1);
    if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e) st = cuda_fail(e, "beta pairs");
  }
  cudaFree(tmp);
  if (st == RP_OK) *pos = p;
  return st;
}

// Derived distributions (Table "continuous"): a base fill whose outputs are
// transformed as they are written (see the Epi codes), or, for two draws of
// one law per output, a base fill of 2n and a pairwise kernel.
rp_status rp_fill_derived(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, rp_derived kind,
                          const double* params, size_t n, double* d_out, void* cuda_stream) {
  if (!params) return fail(RP_ERR_NULL, "params is NULL");
  const double p0 = params[0], p1 = params[1], p2 = params[2];
  auto finite = [](double x) { return std::isfinite(x); };
  auto positive = [](double x) { return x > 0.0 && std::isfinite(x); };
  rp::SampArgs sp{};
  int dist = -1;
  switch (kind) {
    case RP_UNIF:
      if (!finite(p0) || !finite(p1) || !(p0 <= p1) || !finite(p1 - p0)) return fail(RP_ERR_PARAM, "unif needs finite a <= b");
      dist = rp::D_UNIFORM; sp.epi = rp::EPI_AFFINE; sp.ep[0] = p0; sp.ep[1] = p1 - p0;
      break;
    case RP_NORMAL_MS:
    case RP_LOGNORMAL:
      if (!finite(p0) || !positive(p1)) return fail(RP_ERR_PARAM, "needs finite mu and sigma > 0");
      dist = rp::D_NORMAL; sp.epi = kind == RP_NORMAL_MS ? rp::EPI_AFFINE : rp::EPI_LOGNORMAL;
      sp.ep[0] = p0; sp.ep[1] = p1;
      break;
    case RP_EXP_SCALE:
      if (!positive(p0)) return fail(RP_ERR_PARAM, "exponential scale must be positive");
      dist = rp::D_EXP; sp.epi = rp::EPI_SCALE; sp.ep[0] = p0;
      break;
    case RP_GAMMA_SCALE:
      if (!positive(p0) || !positive(p1)) return fail(RP_ERR_PARAM, "gamma shape and scale must be positive");
      dist = rp::D_GAMMA; sp.ga = mt_params(p0); sp.epi = rp::EPI_SCALE; sp.ep[0] = p1;
      break;
    case RP_CHI2:
      if (!positive(p0)) return fail(RP_ERR_PARAM, "chi2 degrees of freedom must be positive");
      dist = rp::D_GAMMA; sp.ga = mt_params(0.5 * p0); sp.epi = rp::EPI_SCALE; sp.ep[0] = 2.0;
      break;
    case RP_GUMBEL:
      if (!finite(p0) || !positive(p1)) return fail(RP_ERR_PARAM, "gumbel needs finite mu and beta > 0");
      dist = rp::D_UNIFORM; sp.epi = rp::EPI_GUMBEL; sp.ep[0] = p0; sp.ep[1] = p1;
      break;
    case RP_PARETO:
      if (!positive(p0) || !positive(p1)) return fail(RP_ERR_PARAM, "pareto x_m and alpha must be positive");
      dist = rp::D_EXP; sp.epi = rp::EPI_PARETO; sp.ep[0] = p0; sp.ep[1] = p1;
      break;
    case RP_WEIBULL:
      if (!positive(p0) || !positive(p1)) return fail(RP_ERR_PARAM, "weibull k and lambda must be positive");
      dist = rp::D_EXP; sp.epi = rp::EPI_WEIBULL; sp.ep[0] = 1.0 / p0; sp.ep[1] = p1;
      break;
    case RP_GPD:
      if (!finite(p0) || !positive(p1) || !finite(p2)) return fail(RP_ERR_PARAM, "gpd needs finite mu, xi and sigma > 0");
      dist = rp::D_EXP; sp.epi = rp::EPI_GPD; sp.ep[0] = p0; sp.ep[1] = p1; sp.ep[2] = p2;
      sp.ep[3] = p2 != 0.0 ? 1.0 / std::fabs(p2) : 0.0;
      break;
    case RP_F: {
      if (!positive(p0) || !positive(p1)) return fail(RP_ERR_PARAM, "F degrees of freedom must be positive");
      sp.ga = mt_params(0.5 * p0);
      sp.gb = mt_params(0.5 * p1);
      sp.epi = rp::EPI_F; sp.ep[0] = p0; sp.ep[1] = p1;
      if (0.5 * p0 != 0.5 * p1) return run_fill(engine, seed, stream, (u64*)pos, n, rp::D_BETA, sp, d_out, cuda_stream);
      rp::SampArgs sg{};
      sg.ga = sp.ga;
      const double q[4] = {p0, p1, 0.0, 0.0};
      return pairs_fill(engine, seed, stream, (u64*)pos, n, rp::D_GAMMA, sg, 1, q, d_out, cuda_stream);
    }
    case RP_T:
      if (!positive(p0)) return fail(RP_ERR_PARAM, "t degrees of freedom must be positive");
      dist = rp::D_T; sp.ga = mt_params(0.5 * p0); sp.ep[0] = p0;
      break;
    case RP_SKEW_NORMAL: {
      if (!finite(p0) || !positive(p1) || !finite(p2)) return fail(RP_ERR_PARAM, "skew normal needs finite mu, alpha and sigma > 0");
      const double delta = p2 / std::sqrt(1.0 + p2 * p2);
      const double q[4] = {p0, p1, delta, std::sqrt(1.0 - delta * delta)};
      rp::SampArgs sn{};
      return pairs_fill(engine, seed, stream, (u64*)pos, n, rp::D_NORMAL, sn, 2, q, d_out, cuda_stream);
    }
    default:
      return fail(RP_ERR_PARAM, "unknown derived distribution " + std::to_string((int)kind));
  }
  return run_fill(engine, seed, stream, (u64*)pos, n, dist, sp, d_out, cuda_stream);
}

namespace {
double* g_grad_part = nullptr;   // device: block partials (2 per block), 2 results, gamma tables
double* g_grad_h = nullptr;      // pinned host copy of the 2 results

int ensure_grad_scratch() {
  if (!g_grad_part) {
    int e = (int)cudaMalloc((void**)&g_grad_part, sizeof(double) * rp::grad_scratch_doubles());
    if (e) { g_grad_part = nullptr; return e; }
    e = (int)cudaMallocHost((void**)&g_grad_h, 2 * sizeof(double));
    if (e) return e;
  }
  return 0;
}
}  // namespace

rp_status rp_gamma_grad(const double* d_z, double alpha, const double* d_g, size_t n, double* d_dzda,
                        double* h_grad_alpha, void* cuda_stream) {
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(RP_ERR_PARAM, "gamma shape must be positive and finite");
  if (n == 0) { if (h_grad_alpha) *h_grad_alpha = 0.0; return RP_OK; }
  if (!d_z) return fail(RP_ERR_NULL, "z is NULL");
  if (d_g && !h_grad_alpha) return fail(RP_ERR_NULL, "h_grad_alpha is NULL while upstream gradients are given");
  if (!d_g && !d_dzda) return fail(RP_ERR_NULL, "nothing to compute: both d_g and d_dzda are NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  if (rp_status dg = device_guard()) return dg;
  int e = ensure_grad_scratch();
  if (e) return fail(RP_ERR_NOMEM, "gradient scratch allocation failed");
  double* out = g_grad_part + 2 * (size_t)rp::grad_blocks();
  e = rp::launch_gamma_grad(d_z, d_g, n, alpha, d_dzda, g_grad_part, out, cuda_stream);
  if (e) return cuda_fail(e, "gamma gradient launch");
  g_launches.fetch_add(3);
  e = (int)cudaMemcpyAsync(g_grad_h, out, sizeof(double), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream);
  if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e) return cuda_fail(e, "gamma gradient");
  if (d_g) *h_grad_alpha = g_grad_h[0];
  return RP_OK;
}

rp_status rp_beta_grad(const double* d_z, double a, double b, const double* d_g, size_t n, double* d_dzda,
                       double* d_dzdb, double* h_grad_a, double* h_grad_b, void* cuda_stream) {
  if (!(a > 0.0) || !(b > 0.0) || !std::isfinite(a) || !std::isfinite(b))
    return fail(RP_ERR_PARAM, "beta parameters must be positive and finite");
  if (n == 0) {
    if (h_grad_a) *h_grad_a = 0.0;
    if (h_grad_b) *h_grad_b = 0.0;
    return RP_OK;
  }
  if (!d_z) return fail(RP_ERR_NULL, "z is NULL");
  if (d_g && (!h_grad_a || !h_grad_b)) return fail(RP_ERR_NULL, "h_grad_a/h_grad_b is NULL while upstream gradients are given");
  if (!d_g && !d_dzda && !d_dzdb) return fail(RP_ERR_NULL, "nothing to compute");
  std::lock_guard<std::mutex> lk(g_mu);
  if (rp_status dg = device_guard()) return dg;
  int e = ensure_grad_scratch();
  if (e) return fail(RP_ERR_NOMEM, "gradient scratch allocation failed");
  double* out = g_grad_part + 2 * (size_t)rp::grad_blocks();
  e = rp::launch_beta_grad(d_z, d_g, n, a, b, d_dzda, d_dzdb, g_grad_part, out, cuda_stream);
  if (e) return cuda_fail(e, "beta gradient launch");
  g_launches.fetch_add(3);
  e = (int)cudaMemcpyAsync(g_grad_h, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream);
  if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e) return cuda_fail(e, "beta gradient");
  if (d_g) { *h_grad_a = g_grad_h[0]; *h_grad_b = g_grad_h[1]; }
  return RP_OK;
}

rp_status rp_beta_grad_composed(const double* d_x, const double* d_y, double a, double b, const double* d_g, size_t n,
                                double* d_dzda, double* d_dzdb, double* h_grad_a, double* h_grad_b, void* cuda_stream) {
  if (!(a > 0.0) || !(b > 0.0) || !std::isfinite(a) || !std::isfinite(b))
    return fail(RP_ERR_PARAM, "beta parameters must be positive and finite");
  if (n == 0) {
    if (h_grad_a) *h_grad_a = 0.0;
    if (h_grad_b) *h_grad_b = 0.0;
    return RP_OK;
  }
  if (!d_x || !d_y) return fail(RP_ERR_NULL, "d_x/d_y is NULL");
  if (d_g && (!h_grad_a || !h_grad_b)) return fail(RP_ERR_NULL, "h_grad_a/h_grad_b is NULL while upstream gradients are given");
  if (!d_g && !d_dzda && !d_dzdb) return fail(RP_ERR_NULL, "nothing to compute");
  std::lock_guard<std::mutex> lk(g_mu);
  if (rp_status dg = device_guard()) return dg;
  int e = ensure_grad_scratch();
  if (e) return fail(RP_ERR_NOMEM, "gradient scratch allocation failed");
  // dX/da and dY/db land in the output arrays (or in temporaries), then the
  // composition rewrites them in place
  double *ta = d_dzda, *tb = d_dzdb, *tmp = nullptr;
  if (!ta || !tb) {
    e = (int)cudaMalloc((void**)&tmp, (size_t)n * sizeof(double) * ((!ta && !tb) ? 2 : 1));
    if (e) return fail(RP_ERR_NOMEM, "gradient temporaries allocation failed");
    if (!ta) ta = tmp;
    if (!tb) tb = tmp + (d_dzda ? 0 : n);
  }
  double* out = g_grad_part + 2 * (size_t)rp::grad_blocks();
  e = rp::launch_gamma_grad(d_x, nullptr, n, a, ta, g_grad_part, out, cuda_stream);
  if (!e) e = rp::launch_gamma_grad(d_y, nullptr, n, b, tb, g_grad_part, out, cuda_stream);
  if (!e) e = rp::launch_beta_compose(d_x, d_y, d_g, n, ta, tb, g_grad_part, out, cuda_stream);
  if (e) {
    if (tmp) cudaFree(tmp);
    return cuda_fail(e, "composed beta gradient launch");
  }
  g_launches.fetch_add(8);
  e = (int)cudaMemcpyAsync(g_grad_h, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream);
  if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (tmp) cudaFree(tmp);
  if (e) return cuda_fail(e, "composed beta gradient");
  if (d_g) { *h_grad_a = g_grad_h[0]; *h_grad_b = g_grad_h[1]; }
  return RP_OK;
}

rp_status rp_seed_state(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* words, int* nw) {
  if (!words || !nw) return fail(RP_ERR_NULL, "words/nw is NULL");
  u64 s[4] = {0, 0, 0, 0};
  rp_status st = seed_state(engine, seed, stream, s);
  if (st) return st;
  memcpy(words, s, sizeof(s));
  *nw = engine == RP_PHILOX4X32_10 ? 3 : 4;
  return RP_OK;
}

rp_status rp_jump_state(rp_engine engine, uint64_t* words, uint64_t delta_hi, uint64_t delta_lo) {
  if (!words) return fail(RP_ERR_NULL, "words is NULL");
  if (engine < 1 || engine > 5) return fail(RP_ERR_ENGINE, "unknown engine id " + std::to_string((int)engine));
  std::lock_guard<std::mutex> lk(g_mu);
  u128 d = ((u128)delta_hi << 64) | delta_lo;
  if (engine == RP_PHILOX4X32_10 && (d & 1)) return fail(RP_ERR_PARAM, "Philox4x32 state jumps must be even (two words per block)");
  if (engine == RP_PHILOX4X64_10 && (d & 3)) return fail(RP_ERR_PARAM, "Philox4x64 state jumps must be multiples of 4 (four words per block)");
  jump_state(engine, (u64*)words, d);
  return RP_OK;
}

// Checkpoint buffer: "RPST", version 1 (u16), engine (u16), four state
// words, the position, eight zero bytes and an FNV-1a 64-bit checksum of
// the first 56 bytes; every integer little-endian, written byte by byte.
namespace {
constexpr uint64_t kFnvOffset = 0xcbf29ce484222325ull, kFnvPrime = 0x100000001b3ull;
uint64_t fnv1a(const uint8_t* p, size_t n) {
  uint64_t h = kFnvOffset;
  for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= kFnvPrime; }
  return h;
}
void put_le(uint8_t* p, uint64_t v, int bytes) {
  for (int i = 0; i < bytes; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
uint64_t get_le(const uint8_t* p, int bytes) {
  uint64_t v = 0;
  for (int i = 0; i < bytes; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}
}  // namespace

rp_status rp_state_serialize(rp_engine engine, const uint64_t* words, uint64_t pos, uint8_t* buf, size_t buflen) {
  if (!words || !buf) return fail(RP_ERR_NULL, "words/buf is NULL");
  if (buflen < RP_STATE_BYTES) return fail(RP_ERR_PARAM, "state buffer shorter than RP_STATE_BYTES");
  if (engine < 1 || engine > 5) return fail(RP_ERR_ENGINE, "unknown engine id " + std::to_string((int)engine));
  memset(buf, 0, RP_STATE_BYTES);
  memcpy(buf, "RPST", 4);
  put_le(buf + 4, 1, 2);
  put_le(buf + 6, (uint64_t)engine, 2);
  for (int i = 0; i < 4; ++i) put_le(buf + 8 + 8 * i, words[i], 8);
  put_le(buf + 40, pos, 8);
  put_le(buf + 56, fnv1a(buf, 56), 8);
  return RP_OK;
}

rp_status rp_state_deserialize(const uint8_t* buf, size_t buflen, rp_engine* engine, uint64_t* words, uint64_t* pos) {
  if (!buf || !engine || !words || !pos) return fail(RP_ERR_NULL, "a pointer is NULL");
  if (buflen < RP_STATE_BYTES) return fail(RP_ERR_PARAM, "state buffer shorter than RP_STATE_BYTES");
  if (memcmp(buf, "RPST", 4) != 0 || get_le(buf + 4, 2) != 1) return fail(RP_ERR_PARAM, "not a version-1 state buffer");
  if (get_le(buf + 56, 8) != fnv1a(buf, 56)) return fail(RP_ERR_PARAM, "state buffer checksum mismatch");
  if (get_le(buf + 48, 8) != 0) return fail(RP_ERR_PARAM, "state buffer reserved bytes are not zero");
  const uint64_t e = get_le(buf + 6, 2);
  if (e < 1 || e > 5) return fail(RP_ERR_PARAM, "state buffer names an unknown engine");
  uint64_t w[4];
  for (int i = 0; i < 4; ++i) w[i] = get_le(buf + 8 + 8 * i, 8);
  if (xoshiro_engine((int)e) && (w[0] | w[1] | w[2] | w[3]) == 0) return fail(RP_ERR_PARAM, "all-zero xoshiro state");
  *engine = (rp_engine)e;
  memcpy(words, w, sizeof(w));
  *pos = get_le(buf + 40, 8);
  return RP_OK;
}

const char* rp_engine_name(int engine) {
  switch (engine) {
    case RP_XOSHIRO256PP: return "xoshiro256pp";
    case RP_PCG64DXSM: return "pcg64dxsm";
    case RP_PHILOX4X32_10: return "philox4x32_10";
    case RP_PHILOX4X64_10: return "philox4x64_10";
    case RP_XOSHIRO256SS: return "xoshiro256ss";
    default: return nullptr;
  }
}

rp_status rp_ziggurat_tables(int which, uint64_t* k, double* w, double* f, double* R) {
  if (!k || !w || !f || !R) return fail(RP_ERR_NULL, "NULL table pointer");
  if (which != 0 && which != 1) return fail(RP_ERR_PARAM, "which must be 0 (normal) or 1 (exponential)");
  const unsigned long long* K = which ? RP_ZIG_E_K : RP_ZIG_N_K;
  const double* W = which ? RP_ZIG_E_W : RP_ZIG_N_W;
  const double* F = which ? RP_ZIG_E_F : RP_ZIG_N_F;
  for (int i = 0; i < 256; ++i) { k[i] = K[i]; w[i] = W[i]; f[i] = F[i]; }
  *R = which ? RP_ZIG_E_R : RP_ZIG_N_R;
  return RP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- normal fill on fixed scratch
// rp_fill_normal_philox_static: the Philox normal fill of rp_fill_normal run
// on the fixed device block of rp_static_scratch.cu instead of scratch from
// cudaMalloc.  Philox is counter-based, so the launch needs no jump tables
// either; nothing on this path calls an allocation routine.
namespace {
static_assert(rp::kStaticMaxN == RP_STATIC_MAX_N, "public and internal scratch limits differ");

constexpr int kStaticMaxDevices = 64;
struct StaticDev {
  bool ready;
  unsigned long long* base;   // the scratch block on this device
  u64 grid_cap;               // SMs x resident CTAs of the fill kernel
};
StaticDev g_static[kStaticMaxDevices];

// One-time setup for the current device `dev`: the scratch address, the
// ziggurat tables in every kernel module, the launch limits.
rp_status static_setup(int dev, StaticDev& D) {
  void* p = nullptr;
  int e = rp::static_scratch_address(&p);
  if (e) return cuda_fail(e, "scratch symbol address");
  if (!p || ((uintptr_t)p & 255)) return fail(RP_ERR_INTERNAL, "scratch symbol is not 256-byte aligned");
  ZigHost z[2];
  fill_zig(z[0], RP_ZIG_N_K, RP_ZIG_N_W, RP_ZIG_N_F, RP_ZIG_N_R);
  fill_zig(z[1], RP_ZIG_E_K, RP_ZIG_E_W, RP_ZIG_E_F, RP_ZIG_E_R);
  e = rp::upload_zig(z);
  if (e) return cuda_fail(e, "ziggurat table upload");
  int sms = 0;
  e = (int)cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e) return cuda_fail(e, "device attribute");
  int occ = rp::occupancy_blocks(RP_PHILOX4X32_10, rp::D_NORMAL, 0);
  D.base = (unsigned long long*)p;
  D.grid_cap = (u64)(sms > 0 ? sms : 1) * (u64)(occ > 0 ? occ : 1);
  D.ready = true;
  return RP_OK;
}
}  // namespace

extern "C" rp_status rp_fill_normal_philox_static(uint64_t seed, uint64_t stream, uint64_t* pos, size_t n,
                                                  double* d_out, void* cuda_stream) {
  if (!pos) return fail(RP_ERR_NULL, "pos is NULL");
  if (n > RP_STATIC_MAX_N)
    return fail(RP_ERR_PARAM, "n = " + std::to_string(n) + " exceeds RP_STATIC_MAX_N = 4194304 (2^22), " +
                                  "the capacity of the fixed scratch; use rp_fill_normal or split the call");
  if (n == 0) return RP_OK;
  if (!d_out) return fail(RP_ERR_NULL, "output pointer is NULL");
  if ((uintptr_t)d_out & 7) return fail(RP_ERR_PARAM, "output pointer must be 8-byte aligned");
  // The lock is held until the stream has been synchronised, so calls from
  // several host threads never have work on the shared block at once.
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  int e = (int)cudaGetDevice(&dev);
  if (e) return cuda_fail(e, "current device");
  if (dev < 0 || dev >= kStaticMaxDevices) return fail(RP_ERR_PARAM, "device ordinal out of range");
  StaticDev& D = g_static[dev];
  if (!D.ready) {
    rp_status st = static_setup(dev, D);
    if (st) return st;
  }
  u64 s[4] = {0, 0, 0, 0};
  rp_status st = seed_state(RP_PHILOX4X32_10, seed, stream, s);
  if (st) return st;

  rp::Ctrl* ctrl = (rp::Ctrl*)D.base;
  unsigned long long* status = D.base + rp::kStaticCtrlWords;
  rp::TailEntry* tailq = (rp::TailEntry*)(D.base + rp::kStaticCtrlWords + rp::kStaticTiles);
  cudaStream_t cs = (cudaStream_t)cuda_stream;

  rp::FillArgs a;
  memset(&a, 0, sizeof(a));
  a.eng.engine = RP_PHILOX4X32_10;
  a.dist = rp::D_NORMAL;
  rp::TileGeom tg = rp::tile_geom(RP_PHILOX4X32_10, rp::D_NORMAL, 0);
  const u64 T = (u64)tg.tile_words;
  memcpy(a.eng.s, s, sizeof(s));
  a.eng.tile_words = T;
  a.eng.chunk_words = (u64)tg.c;
  a.tile_status = status;
  a.ctrl = ctrl;
  a.tailq = tailq;
  a.tail_cap = rp::kStaticTailCap;
  a.tail_count = &ctrl->n_tail;

  u64 cur = *pos;
  size_t done = 0;
  for (int launch = 0; done < n; ++launch) {
    if (launch > 64) return fail(RP_ERR_INTERNAL, "too many continuation launches");
    const size_t left = n - done;
    const double wpv = 1.0235;
    const double need = (double)left * wpv + 8.0 * std::sqrt((double)left * wpv) + 64.0;
    const u64 tiles = (u64)(need / (double)T) + 2;
    if (tiles > rp::kStaticTiles) return fail(RP_ERR_INTERNAL, "tile count exceeds the fixed scratch");
    const u64 grid = std::min<u64>(tiles, D.grid_cap);
    a.eng.word0 = cur;
    a.eng.stride = grid * T;
    a.n = left;
    a.n_tiles = tiles;
    a.out = d_out + done;
    // What must start at zero: the status words of this launch's tiles and
    // the control block (its tail count included), except done_tile and
    // first_reject, which start at all ones as in the allocating path.  Tail
    // entries are written before they are read.
    e = (int)cudaMemsetAsync(status, 0, tiles * 8, cs);
    if (!e) e = (int)cudaMemsetAsync(ctrl, 0, sizeof(rp::Ctrl), cs);
    if (!e) e = (int)cudaMemsetAsync(&ctrl->done_tile, 0xff, sizeof(ctrl->done_tile), cs);
    if (!e) e = (int)cudaMemsetAsync(&ctrl->first_reject, 0xff, sizeof(ctrl->first_reject), cs);
    if (e) return cuda_fail(e, "scratch reset");
    e = rp::launch_fill(a, (int)grid, cuda_stream);
    if (e) return cuda_fail(e, "kernel launch");
    g_launches.fetch_add(1);
    e = rp::launch_tails(a, cuda_stream);
    if (e) return cuda_fail(e, "tail kernel launch");
    g_launches.fetch_add(1);
    rp::Ctrl c;
    e = (int)cudaMemcpyAsync(&c, ctrl, sizeof(c), cudaMemcpyDeviceToHost, cs);
    if (!e) e = (int)cudaStreamSynchronize(cs);
    if (e) return cuda_fail(e, "fill");
    if (c.err) {
      char buf[160];
      snprintf(buf, sizeof buf, "device check failed (bits 0x%x, tile %llu)", c.err, (unsigned long long)c.err_info);
      return fail(c.err & rp::E_TIMEOUT ? RP_ERR_TIMEOUT : RP_ERR_INTERNAL, buf);
    }
    if (c.n_tail > rp::kStaticTailCap) return fail(RP_ERR_INTERNAL, "tail queue of the fixed scratch overflowed");
    if (c.done_tile != ~0ull) {
      cur += c.next_pos;
      done = n;
    } else {
      if (c.total == 0 && c.next_pos == 0) return fail(RP_ERR_INTERNAL, "launch produced no output");
      done += c.total;
      cur += c.next_pos;
    }
  }
  *pos = cur;
  return RP_OK;
}

// ---------------------------------------------------------------- fills from state, substreams
namespace {

// Sampler arguments of (dist, p0, p1, m) with the checks of the seeded fills;
// *dist_out is the kernel distribution (bounded with m = 0 -> raw words).
rp_status make_samp(int dist, double p0, double p1, u64 m, rp::SampArgs& sp, int* dist_out) {
  memset(&sp, 0, sizeof(sp));
  *dist_out = dist;
  switch (dist) {
    case RP_DIST_U64: case RP_DIST_UNIFORM: case RP_DIST_NORMAL: case RP_DIST_EXP: return RP_OK;
    case RP_DIST_UNIFORM52: *dist_out = rp::D_UNIFORM52; return RP_OK;
    case RP_DIST_BOUNDED:
      sp.m = m;
      if (m == 0) { *dist_out = rp::D_U64; return RP_OK; }
      sp.thresh = (0 - m) % m;
      return RP_OK;
    case RP_DIST_GAMMA:
      if (!(p0 > 0.0) || !std::isfinite(p0)) return fail(RP_ERR_PARAM, "gamma shape must be positive and finite");
      sp.ga = mt_params(p0);
      return RP_OK;
    case RP_DIST_BETA:
      if (!(p0 > 0.0) || !(p1 > 0.0) || !std::isfinite(p0) || !std::isfinite(p1))
        return fail(RP_ERR_PARAM, "beta parameters must be positive and finite");
      sp.ga = mt_params(p0);
      sp.gb = mt_params(p1);
      return RP_OK;
    default:
      return fail(RP_ERR_PARAM, "unknown distribution code " + std::to_string(dist));
  }
}

// Beta(a, a) from a state: consecutive Gamma(a) pairs (as rp_fill_beta).
rp_status beta_equal_state_locked(int engine, const u64 s[4], u64* pos, size_t n, const rp::SampArgs& sp,
                                  double* d_out, void* cstream) {
  const size_t blk = (size_t)1 << 26;   // pairs per block: 2^27 base variates keep the GPU full (1 GiB scratch)
  double* tmp = nullptr;
  size_t cap = std::min(n, blk);
  int e = (int)cudaMalloc((void**)&tmp, cap * 2 * sizeof(double));
  if (e) return fail(RP_ERR_NOMEM, "beta scratch allocation failed");
  u64 p = *pos;
  rp_status st = RP_OK;
  for (size_t done = 0; done < n && st == RP_OK; done += cap) {
    size_t m = std::min(cap, n - done);
    rp::SampArgs sg{};
    sg.ga = sp.ga;
    st = run_fill_state_locked(engine, s, &p, 2 * m, rp::D_GAMMA, sg, tmp, cstream);
    if (st) break;
    e = rp::launch_pairs(tmp, d_out + done, m, 0, nullptr, cstream);
    if (!e) g_launches.fetch_add(1);
    if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cstream);
    if (e) st = cuda_fail(e, "beta pairs");
  }
  cudaFree(tmp);
  if (st == RP_OK) *pos = p;
  return st;
}

rp_status substream_words(int engine, u64 base_seed, u64 sidx, u64 w[4]) {
  rp_status st = seed_state(engine, base_seed, RP_NO_STREAM, w);
  if (st) return st;
  if (xoshiro_engine(engine)) {
    const u64 limbs[3] = {0, 0, sidx};   // s * 2^128
    xo_jump_limbs(w, limbs, 3);
  } else if (engine == RP_PHILOX4X32_10 || engine == RP_PHILOX4X64_10) {
    w[2] = sidx;   // (first) key word := s, the stream setter
  } else {
    const u128 inc = ((u128)sidx << 1) | 1u;
    w[2] = (u64)(inc >> 64);
    w[3] = (u64)inc;
  }
  return RP_OK;
}

}  // namespace

extern "C" rp_status rp_fill_state(rp_engine engine, const uint64_t* words, uint64_t* pos, int dist, size_t n,
                                   double p0, double p1, uint64_t m, void* d_out, void* cuda_stream) {
  if (!words) return fail(RP_ERR_NULL, "words is NULL");
  rp_status st = check_fill_args(engine, (u64*)pos, n, d_out);
  if (st || n == 0) return st;
  rp::SampArgs sp;
  int kd = 0;
  st = make_samp(dist, p0, p1, m, sp, &kd);
  if (st) return st;
  u64 s[4] = {words[0], words[1], words[2], engine == RP_PHILOX4X32_10 ? 0 : words[3]};
  std::lock_guard<std::mutex> lk(g_mu);
  if (dist == RP_DIST_BETA && p0 == p1)
    return beta_equal_state_locked(engine, s, (u64*)pos, n, sp, (double*)d_out, cuda_stream);
  return run_fill_state_locked(engine, s, (u64*)pos, n, kd, sp, d_out, cuda_stream);
}

namespace {
// Staging of rp_fill_to_host: two device slots, filled in turn on the
// caller's stream and copied out on the library's copy stream, so that a
// fill overlaps the previous call's copy.
struct HostStage {
  void* slot[2] = {nullptr, nullptr};
  size_t cap = 0;
  cudaEvent_t copied[2] = {nullptr, nullptr};   // the slot's last copy is done
  cudaEvent_t filled = nullptr;
  cudaStream_t copy_stream = nullptr;
  int next = 0;
};
HostStage g_hs;

int host_stage_ensure(size_t bytes) {
  int e = 0;
  if (!g_hs.copy_stream) {
    e = (int)cudaStreamCreateWithFlags(&g_hs.copy_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && !e; ++i) e = (int)cudaEventCreateWithFlags(&g_hs.copied[i], cudaEventDisableTiming);
    if (!e) e = (int)cudaEventCreateWithFlags(&g_hs.filled, cudaEventDisableTiming);
    if (e) return e;
  }
  if (bytes > g_hs.cap) {
    for (int i = 0; i < 2; ++i)
      if (g_hs.slot[i]) cudaFree(g_hs.slot[i]);   // waits for the device (earlier copies) first
    g_hs.slot[0] = g_hs.slot[1] = nullptr;
    g_hs.cap = 0;
    for (int i = 0; i < 2 && !e; ++i) e = (int)cudaMalloc(&g_hs.slot[i], bytes);
    if (e) return e;
    g_hs.cap = bytes;
  }
  return 0;
}
}  // namespace

extern "C" rp_status rp_fill_to_host(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, int dist, size_t n,
                                     double p0, double p1, uint64_t m, void* h_out, void* cuda_stream) {
  if (!pos) return fail(RP_ERR_NULL, "pos is NULL");
  if (n == 0) return RP_OK;
  if (!h_out) return fail(RP_ERR_NULL, "h_out is NULL");
  if (engine < 1 || engine > 5) return fail(RP_ERR_ENGINE, "unknown engine id " + std::to_string((int)engine));
  rp::SampArgs sp;
  int kd = 0;
  rp_status st = make_samp(dist, p0, p1, m, sp, &kd);
  if (st) return st;
  std::lock_guard<std::mutex> lk(g_mu);
  if (rp_status dg = device_guard()) return dg;
  u64 s[4] = {0, 0, 0, 0};
  st = seed_state(engine, seed, stream, s);
  if (st) return st;
  const size_t bytes = n * 8;
  int e = host_stage_ensure(bytes);
  if (e) return fail(RP_ERR_NOMEM, "host staging allocation failed");
  const int k = g_hs.next;
  g_hs.next ^= 1;
  cudaStream_t cs = (cudaStream_t)cuda_stream;
  e = (int)cudaStreamWaitEvent(cs, g_hs.copied[k], 0);   // the slot's previous copy has left it
  if (e) return cuda_fail(e, "staging order");
  if (dist == RP_DIST_BETA && p0 == p1) st = beta_equal_state_locked(engine, s, (u64*)pos, n, sp, (double*)g_hs.slot[k], cuda_stream);
  else st = run_fill_state_locked(engine, s, (u64*)pos, n, kd, sp, g_hs.slot[k], cuda_stream);
  if (st) return st;
  e = (int)cudaEventRecord(g_hs.filled, cs);
  if (!e) e = (int)cudaStreamWaitEvent(g_hs.copy_stream, g_hs.filled, 0);
  if (!e) e = (int)cudaMemcpyAsync(h_out, g_hs.slot[k], bytes, cudaMemcpyDeviceToHost, g_hs.copy_stream);
  if (!e) e = (int)cudaEventRecord(g_hs.copied[k], g_hs.copy_stream);
  if (e) return cuda_fail(e, "copy to host");
  return RP_OK;
}

extern "C" rp_status rp_substream_state(rp_engine engine, uint64_t base_seed, uint64_t s, uint64_t* words, int* nw) {
  if (!words || !nw) return fail(RP_ERR_NULL, "words/nw is NULL");
  if (engine < 1 || engine > 5) return fail(RP_ERR_ENGINE, "unknown engine id " + std::to_string((int)engine));
  std::lock_guard<std::mutex> lk(g_mu);
  u64 w[4] = {0, 0, 0, 0};
  rp_status st = substream_words(engine, base_seed, s, w);
  if (st) return st;
  memcpy(words, w, sizeof(w));
  *nw = engine == RP_PHILOX4X32_10 ? 3 : 4;
  return RP_OK;
}

// ---------------------------------------------------------------- batch plans
// A plan holds, for one request set: each request's substream state, the
// per-request kernel arguments and (request, tile) work lists of the chosen
// schedule, the scratch (tile status words, control blocks, tail queues,
// claim counters) and the instantiated CUDA graph that runs everything.
struct rp_batch_plan {
  int engine = 0;
  u64 base_seed = 0;
  size_t nreq = 0;
  std::vector<rp_request> req;
  std::vector<std::array<u64, 4>> sub;   // substream state (before word 0)
  std::vector<int> cls;                  // kernel class, -1: nothing to do
  std::vector<int> kdist;                // kernel distribution
  std::vector<rp::SampArgs> sp;
  // scratch
  unsigned long long* d_status = nullptr;
  size_t status_cap = 0;
  rp::Ctrl* d_ctrl = nullptr;
  rp::Ctrl* h_ctrl = nullptr;            // pinned
  unsigned long long* d_count = nullptr; // [0..2] claim counters, [3] ziggurat tails, [4] gamma/beta tails
  rp::TailEntry* d_tailq[2] = {nullptr, nullptr};
  u64 tail_cap[2] = {0, 0};
  cudaStream_t cs[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
  // chosen schedule
  int schedule = 0;
  double tuned_ms = 0.0;
  rp::FillArgs* d_fa = nullptr;
  rp::BatchItem* d_items = nullptr;
  u64 n_items_total = 0;
  std::vector<u64> tiles;                // per request, chosen schedule
  cudaGraphExec_t exec = nullptr;
};

namespace {

int batch_class(int kdist) {
  if (kdist == rp::D_U64 || kdist == rp::D_UNIFORM || kdist == rp::D_UNIFORM52) return rp::BC_ONEPW;
  if (kdist == rp::D_GAMMA || kdist == rp::D_BETA) return rp::BC_MERGE;
  return rp::BC_LEAN;
}

struct BatchBuild {
  rp::FillArgs* d_fa = nullptr;
  rp::BatchItem* d_items = nullptr;
  u64 n_items[3] = {0, 0, 0}, item_off[3] = {0, 0, 0};
  std::vector<u64> tiles;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (d_fa) cudaFree(d_fa);
    if (d_items) cudaFree(d_items);
    exec = nullptr; graph = nullptr; d_fa = nullptr; d_items = nullptr;
  }
};

// Builds the device work lists and the graph of one schedule.
// schedule bit 0: items of larger requests first; bit 1: classes one after
// another instead of concurrently; bit 2: 128 words per thread.
rp_status batch_build(rp_batch_plan& P, int schedule, BatchBuild& B) {
  const int cvar = (schedule >> 2) & 1;
  const size_t R = P.nreq;
  std::vector<rp::FillArgs> fa(R);
  B.tiles.assign(R, 0);
  u64 status_off = 0;
  int e = 0;
  void *gpow = nullptr, *gthr[3] = {nullptr, nullptr, nullptr}, *gcta[3] = {nullptr, nullptr, nullptr};
  u64* ppow = nullptr;
  if (xoshiro_engine(P.engine)) {
    e = xo_device_pow(&gpow);
    for (int c = 0; c < 3 && !e; ++c) {
      rp::TileGeom tg = rp::batch_geom(c, cvar);
      e = xo_device_thread((u64)tg.c, tg.nt, &gthr[c]);
      if (!e) e = xo_device_cta((u64)tg.tile_words, &gcta[c]);
    }
  } else if (P.engine == RP_PCG64DXSM) {
    e = pcg_device_pow(&ppow);
  }
  if (e) return cuda_fail(e, "jump tables");
  for (size_t r = 0; r < R; ++r) {
    const int c = P.cls[r];
    if (c < 0) continue;
    rp::FillArgs& a = fa[r];
    memset(&a, 0, sizeof(a));
    const rp::TileGeom tg = rp::batch_geom(c, cvar);
    const u64 T = (u64)tg.tile_words, n = P.req[r].n;
    u64 tiles;
    if (c == rp::BC_ONEPW) {
      tiles = (n + T - 1) / T;
    } else {
      const double wpv = words_per_variate(P.kdist[r], P.sp[r]);
      const double need = (double)n * wpv + 8.0 * std::sqrt((double)n * (wpv > 1.0 ? wpv : 1.0)) + 64.0;
      tiles = (u64)(need / (double)T) + 2;
    }
    if (tiles >= 65536) return fail(RP_ERR_PARAM, "request " + std::to_string(r) + " is too large for a batch");
    B.tiles[r] = tiles;
    a.eng.engine = P.engine;
    u64 s0[4];
    memcpy(s0, P.sub[r].data(), sizeof(s0));
    if (counter_engine(P.engine)) a.eng.word0 = P.req[r].pos;
    else jump_state(P.engine, s0, (u128)P.req[r].pos);
    memcpy(a.eng.s, s0, sizeof(s0));
    a.eng.gf2_pow = gpow;
    a.eng.gf2_thread = gthr[c];
    a.eng.gf2_cta = gcta[c];
    a.eng.pcg_pow = ppow;
    a.eng.tile_words = T;
    a.eng.chunk_words = (u64)tg.c;
    a.sp = P.sp[r];
    a.dist = P.kdist[r];
    a.n = n;
    a.n_tiles = tiles;
    a.out = P.req[r].d_out;
    a.tile_status = P.d_status + status_off;
    a.ctrl = P.d_ctrl + r;
    const int q = c == rp::BC_MERGE ? 1 : 0;
    a.tailq = c == rp::BC_ONEPW ? nullptr : P.d_tailq[q];
    a.tail_cap = c == rp::BC_ONEPW ? 0 : P.tail_cap[q];
    a.tail_count = P.d_count + 3 + q;
    a.tail_abs = 1;
    a.req = (int)r;
    status_off += tiles;
  }
  if (status_off > P.status_cap) return fail(RP_ERR_INTERNAL, "batch status words exceed the plan's scratch");
  // work lists: per class, requests in the schedule's order, tiles ascending
  std::vector<size_t> order(R);
  for (size_t r = 0; r < R; ++r) order[r] = r;
  if (schedule & 1)
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return P.req[x].n > P.req[y].n; });
  std::vector<rp::BatchItem> items;
  for (int c = 0; c < 3; ++c) {
    B.item_off[c] = items.size();
    for (size_t r : order)
      if (P.cls[r] == c)
        for (u64 k = 0; k < B.tiles[r]; ++k) items.push_back(rp::BatchItem{(unsigned)r, (unsigned)k});
    B.n_items[c] = items.size() - B.item_off[c];
  }
  e = (int)cudaMalloc((void**)&B.d_fa, std::max<size_t>(R, 1) * sizeof(rp::FillArgs));
  if (!e) e = (int)cudaMalloc((void**)&B.d_items, std::max<size_t>(items.size(), 1) * sizeof(rp::BatchItem));
  if (e) { B.release(); return fail(RP_ERR_NOMEM, "batch work-list allocation failed"); }
  e = (int)cudaMemcpy(B.d_fa, fa.data(), R * sizeof(rp::FillArgs), cudaMemcpyHostToDevice);
  if (!e && !items.empty())
    e = (int)cudaMemcpy(B.d_items, items.data(), items.size() * sizeof(rp::BatchItem), cudaMemcpyHostToDevice);
  if (e) { B.release(); return cuda_fail(e, "batch upload"); }
  // class kernel arguments and grids
  rp::BatchArgs ba[3];
  int grid[3] = {0, 0, 0};
  const int sms = sm_count();
  for (int c = 0; c < 3; ++c) {
    ba[c].reqs = B.d_fa;
    ba[c].items = B.d_items + B.item_off[c];
    ba[c].n_items = B.n_items[c];
    ba[c].next_item = P.d_count + c;
    const int q = c == rp::BC_MERGE ? 1 : 0;
    ba[c].tailq = P.d_tailq[q];
    ba[c].tail_count = P.d_count + 3 + q;
    ba[c].tail_cap = P.tail_cap[q];
    int occ = 0;
    e = rp::launch_batch(P.engine, c, cvar, ba[c], 0, nullptr, &occ);
    if (e) { B.release(); return cuda_fail(e, "batch occupancy"); }
    const u64 g = (u64)sms * (u64)(occ > 0 ? occ : 1);
    grid[c] = (int)std::min<u64>(g, std::max<u64>(B.n_items[c], 1));
  }
  // capture: reset scratch, run the classes (concurrently or in turn), tails
  cudaStream_t ps = P.cs[0];
  e = (int)cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal);
  if (e) { B.release(); return cuda_fail(e, "graph capture"); }
  int ce = (int)cudaMemsetAsync(P.d_status, 0, std::max<u64>(status_off, 1) * 8, ps);
  if (!ce) ce = (int)cudaMemsetAsync(P.d_ctrl, 0, R * sizeof(rp::Ctrl), ps);
  if (!ce) ce = (int)cudaMemset2DAsync(P.d_ctrl, sizeof(rp::Ctrl), 0xff, sizeof(unsigned long long), R, ps);
  if (!ce) ce = (int)cudaMemsetAsync(P.d_count, 0, 5 * sizeof(unsigned long long), ps);
  const bool serial = (schedule >> 1) & 1;
  if (!ce && !serial) ce = (int)cudaEventRecord(P.ev_fork, ps);
  for (int c = 0; c < 3 && !ce; ++c) {
    if (!B.n_items[c]) continue;
    cudaStream_t s = serial ? ps : P.cs[c];
    if (!serial && c != 0) ce = (int)cudaStreamWaitEvent(s, P.ev_fork, 0);
    if (!ce) ce = rp::launch_batch(P.engine, c, cvar, ba[c], grid[c], s, nullptr);
    if (!ce) ce = rp::launch_batch_tails(c, ba[c], s);
    if (!ce && !serial && c != 0) {
      ce = (int)cudaEventRecord(P.ev_join[c], s);
      if (!ce) ce = (int)cudaStreamWaitEvent(ps, P.ev_join[c], 0);
    }
  }
  e = (int)cudaStreamEndCapture(ps, &B.graph);
  if (ce || e) { B.release(); return cuda_fail(ce ? ce : e, "graph capture"); }
  e = (int)cudaGraphInstantiate(&B.exec, B.graph, 0);
  if (e) { B.release(); return cuda_fail(e, "graph instantiate"); }
  return RP_OK;
}

// Reads the control blocks after a run: device checks, and requests whose
// tile estimate fell short are completed by a plain fill from where their
// chain stopped.  next_pos (nullable) receives each request's next word.
rp_status batch_finish(rp_batch_plan& P, const std::vector<u64>& tiles, u64* next_pos, void* cstream) {
  for (size_t r = 0; r < P.nreq; ++r) {
    const u64 pos0 = P.req[r].pos;
    if (P.cls[r] < 0) { if (next_pos) next_pos[r] = pos0; continue; }
    const rp::Ctrl& c = P.h_ctrl[r];
    if (c.err) {
      char buf[200];
      snprintf(buf, sizeof buf, "batch request %zu: device check failed (bits 0x%x, tile %llu)", r, c.err,
               (unsigned long long)c.err_info);
      return fail(c.err & rp::E_TIMEOUT ? RP_ERR_TIMEOUT : RP_ERR_INTERNAL, buf);
    }
    const u64 n = P.req[r].n;
    if (P.cls[r] == rp::BC_ONEPW) {
      if (next_pos) next_pos[r] = pos0 + n;
      continue;
    }
    if (c.done_tile != ~0ull) {
      if (next_pos) next_pos[r] = pos0 + c.next_pos;
      continue;
    }
    if (c.total >= n || (c.total == 0 && c.next_pos == 0))
      return fail(RP_ERR_INTERNAL, "batch request " + std::to_string(r) + " produced no usable output");
    (void)tiles;
    u64 p = pos0 + c.next_pos;
    u64 s[4];
    memcpy(s, P.sub[r].data(), sizeof(s));
    rp_status st = run_fill_state_locked(P.engine, s, &p, n - c.total, P.kdist[r], P.sp[r],
                                         (char*)P.req[r].d_out + c.total * 8, cstream);
    if (st) return st;
    if (next_pos) next_pos[r] = p;
  }
  return RP_OK;
}

rp_status batch_launch(rp_batch_plan& P, cudaGraphExec_t exec, void* cstream) {
  cudaStream_t s = (cudaStream_t)cstream;
  int e = (int)cudaGraphLaunch(exec, s);
  if (!e && P.nreq) e = (int)cudaMemcpyAsync(P.h_ctrl, P.d_ctrl, P.nreq * sizeof(rp::Ctrl), cudaMemcpyDeviceToHost, s);
  if (!e) e = (int)cudaStreamSynchronize(s);
  if (e) return cuda_fail(e, "batch run");
  g_launches.fetch_add(1);
  return RP_OK;
}

void plan_free(rp_batch_plan* P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->d_fa) cudaFree(P->d_fa);
  if (P->d_items) cudaFree(P->d_items);
  if (P->d_status) cudaFree(P->d_status);
  if (P->d_ctrl) cudaFree(P->d_ctrl);
  if (P->h_ctrl) cudaFreeHost(P->h_ctrl);
  if (P->d_count) cudaFree(P->d_count);
  for (int q = 0; q < 2; ++q)
    if (P->d_tailq[q]) cudaFree(P->d_tailq[q]);
  for (int c = 0; c < 3; ++c) {
    if (P->cs[c]) cudaStreamDestroy(P->cs[c]);
    if (P->ev_join[c]) cudaEventDestroy(P->ev_join[c]);
  }
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  delete P;
}

}  // namespace

extern "C" rp_status rp_batch_plan_create(const rp_request* reqs, size_t nreq, rp_engine engine, uint64_t base_seed,
                                          int autotune, rp_batch_plan** plan, void* cuda_stream) {
  if (!plan) return fail(RP_ERR_NULL, "plan is NULL");
  *plan = nullptr;
  if (nreq && !reqs) return fail(RP_ERR_NULL, "reqs is NULL");
  if (engine < 1 || engine > 5) return fail(RP_ERR_ENGINE, "unknown engine id " + std::to_string((int)engine));
  std::lock_guard<std::mutex> lk(g_mu);
  if (rp_status dg = device_guard()) return dg;
  int e = ensure_zig();
  if (e) return cuda_fail(e, "ziggurat table upload");
  rp_batch_plan* P = new rp_batch_plan();
  P->engine = engine;
  P->base_seed = base_seed;
  P->nreq = nreq;
  P->req.assign(reqs, reqs + nreq);
  P->sub.resize(nreq);
  P->cls.assign(nreq, -1);
  P->kdist.assign(nreq, 0);
  P->sp.resize(nreq);
  u64 tail_need[2] = {4096, 4096}, max_tiles = 0;
  for (size_t r = 0; r < nreq; ++r) {
    const rp_request& q = P->req[r];
    if (q.reserved != 0) { plan_free(P); return fail(RP_ERR_PARAM, "rp_request.reserved must be 0"); }
    int kd = 0;
    rp_status st = make_samp(q.dist, q.p0, q.p1, q.m, P->sp[r], &kd);
    if (st) { plan_free(P); return st; }
    if (q.dist == RP_DIST_BETA && q.p0 == q.p1) {
      plan_free(P);
      return fail(RP_ERR_PARAM, "batched beta requests need a != b (use rp_fill_state for equal shapes)");
    }
    std::array<u64, 4> w{};
    st = substream_words(engine, base_seed, q.stream, w.data());
    if (st) { plan_free(P); return st; }
    P->sub[r] = w;
    P->kdist[r] = kd;
    if (q.n == 0) continue;
    if (!q.d_out) { plan_free(P); return fail(RP_ERR_NULL, "request " + std::to_string(r) + " has no output"); }
    if ((uintptr_t)q.d_out & 7) { plan_free(P); return fail(RP_ERR_PARAM, "request outputs must be 8-byte aligned"); }
    const int c = batch_class(kd);
    P->cls[r] = c;
    if (c != rp::BC_ONEPW) tail_need[c == rp::BC_MERGE ? 1 : 0] += q.n / 1024 + 64;
    // status words: bound over the schedules (the smallest tiles)
    const rp::TileGeom tg = rp::batch_geom(c, 1);
    const double wpv = c == rp::BC_ONEPW ? 1.0 : words_per_variate(kd, P->sp[r]);
    max_tiles += (u64)(((double)q.n * wpv + 8.0 * std::sqrt((double)q.n * std::max(wpv, 1.0)) + 64.0) /
                       (double)tg.tile_words) + 3;
  }
  P->status_cap = max_tiles + 1;
  e = (int)cudaMalloc((void**)&P->d_status, P->status_cap * 8);
  if (!e) e = (int)cudaMalloc((void**)&P->d_ctrl, std::max<size_t>(nreq, 1) * sizeof(rp::Ctrl));
  if (!e) e = (int)cudaMallocHost((void**)&P->h_ctrl, std::max<size_t>(nreq, 1) * sizeof(rp::Ctrl));
  if (!e) e = (int)cudaMalloc((void**)&P->d_count, 8 * sizeof(unsigned long long));
  for (int q = 0; q < 2 && !e; ++q) {
    P->tail_cap[q] = tail_need[q];
    e = (int)cudaMalloc((void**)&P->d_tailq[q], tail_need[q] * sizeof(rp::TailEntry));
  }
  for (int c = 0; c < 3 && !e; ++c) {
    e = (int)cudaStreamCreateWithFlags(&P->cs[c], cudaStreamNonBlocking);
    if (!e) e = (int)cudaEventCreateWithFlags(&P->ev_join[c], cudaEventDisableTiming);
  }
  if (!e) e = (int)cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming);
  if (e) { plan_free(P); return fail(RP_ERR_NOMEM, std::string("batch scratch: ") + cudaGetErrorString((cudaError_t)e)); }
  // schedules: the default one, or the fastest of all when tuning
  const int n_sched = autotune ? 8 : 1;
  BatchBuild best;
  float best_ms = 0.0f;
  int best_s = -1;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (autotune) {
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
  }
  for (int sched = 0; sched < n_sched; ++sched) {
    BatchBuild B;
    rp_status st = batch_build(*P, sched, B);
    if (st) { best.release(); plan_free(P); return st; }
    if (autotune) {
      float ms = 0.0f;
      st = batch_launch(*P, B.exec, cuda_stream);   // warm
      if (!st) st = batch_finish(*P, B.tiles, nullptr, cuda_stream);
      if (!st) {
        cudaEventRecord(t0, (cudaStream_t)cuda_stream);
        e = (int)cudaGraphLaunch(B.exec, (cudaStream_t)cuda_stream);
        cudaEventRecord(t1, (cudaStream_t)cuda_stream);
        if (!e) e = (int)cudaEventSynchronize(t1);
        if (e) st = cuda_fail(e, "batch tuning");
        else cudaEventElapsedTime(&ms, t0, t1);
      }
      if (st) { B.release(); best.release(); plan_free(P); return st; }
      if (best_s < 0 || ms < best_ms) {
        best.release();
        best = B;
        best_ms = ms;
        best_s = sched;
      } else {
        B.release();
      }
    } else {
      best = B;
      best_s = sched;
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (best.graph) { cudaGraphDestroy(best.graph); best.graph = nullptr; }
  P->schedule = best_s;
  P->tuned_ms = autotune ? best_ms : 0.0;
  P->d_fa = best.d_fa;
  P->d_items = best.d_items;
  P->exec = best.exec;
  P->tiles = best.tiles;
  P->n_items_total = best.n_items[0] + best.n_items[1] + best.n_items[2];
  *plan = P;
  return RP_OK;
}

extern "C" rp_status rp_batch_plan_run(rp_batch_plan* plan, uint64_t* next_pos, void* cuda_stream) {
  if (!plan) return fail(RP_ERR_NULL, "plan is NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  if (rp_status dg = device_guard()) return dg;
  rp_status st = batch_launch(*plan, plan->exec, cuda_stream);
  if (st) return st;
  return batch_finish(*plan, plan->tiles, (u64*)next_pos, cuda_stream);
}

extern "C" rp_status rp_batch_plan_info(const rp_batch_plan* plan, int* schedule, double* tuned_ms, uint64_t* items) {
  if (!plan) return fail(RP_ERR_NULL, "plan is NULL");
  if (schedule) *schedule = plan->schedule;
  if (tuned_ms) *tuned_ms = plan->tuned_ms;
  if (items) *items = plan->n_items_total;
  return RP_OK;
}

extern "C" rp_status rp_batch_plan_destroy(rp_batch_plan* plan) {
  std::lock_guard<std::mutex> lk(g_mu);
  plan_free(plan);
  return RP_OK;
}

extern "C" rp_status rp_batch_run(rp_request* reqs, size_t nreq, rp_engine engine, uint64_t base_seed,
                                  void* cuda_stream) {
  rp_batch_plan* P = nullptr;
  rp_status st = rp_batch_plan_create(reqs, nreq, engine, base_seed, 0, &P, cuda_stream);
  if (st) return st;
  std::vector<uint64_t> np(nreq);
  st = rp_batch_plan_run(P, np.data(), cuda_stream);
  if (!st)
    for (size_t r = 0; r < nreq; ++r) reqs[r].pos = np[r];
  rp_batch_plan_destroy(P);
  return st;
}

// ---------------------------------------------------------------- multivariate normal
namespace {
double* g_mvn_part = nullptr;   // backward partial tiles (grown on demand)
size_t g_mvn_cap = 0;

rp_status mvn_check(int d, size_t n) {
  if (d < 1 || d > (1 << 16)) return fail(RP_ERR_PARAM, "d must be in [1, 65536]");
  if (n > ((size_t)1 << 62) / (size_t)d) return fail(RP_ERR_PARAM, "n * d overflows");
  return RP_OK;
}
}  // namespace

extern "C" rp_status rp_mvn(rp_engine engine, uint64_t seed, uint64_t stream, uint64_t* pos, int d, size_t n,
                            const double* d_mu, const double* d_L, double* d_Z, double* d_X, void* cuda_stream) {
  rp_status st = mvn_check(d, n);
  if (st) return st;
  if (!pos) return fail(RP_ERR_NULL, "pos is NULL");
  if (n == 0) return RP_OK;
  if (!d_mu || !d_L || !d_Z || !d_X) return fail(RP_ERR_NULL, "NULL device pointer");
  st = rp_fill_normal(engine, seed, stream, pos, n * (size_t)d, d_Z, cuda_stream);
  if (st) return st;
  int e = rp::launch_mvn_apply(d, n, d_mu, d_L, d_Z, d_X, cuda_stream);
  if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e) return cuda_fail(e, "mvn apply");
  g_launches.fetch_add(1);
  return RP_OK;
}

extern "C" rp_status rp_mvn_grads(int d, size_t n, const double* d_G, const double* d_Z, double* d_gmu, double* d_gL,
                                  void* cuda_stream) {
  rp_status st = mvn_check(d, n);
  if (st) return st;
  if (!d_gmu || !d_gL) return fail(RP_ERR_NULL, "NULL device pointer");
  if (n && (!d_G || !d_Z)) return fail(RP_ERR_NULL, "NULL device pointer");
  std::lock_guard<std::mutex> lk(g_mu);
  if (rp_status dg = device_guard()) return dg;
  if (n == 0) {
    int e = (int)cudaMemsetAsync(d_gmu, 0, (size_t)d * 8, (cudaStream_t)cuda_stream);
    if (!e) e = (int)cudaMemsetAsync(d_gL, 0, (size_t)d * d * 8, (cudaStream_t)cuda_stream);
    if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cuda_stream);
    return e ? cuda_fail(e, "mvn grads") : RP_OK;
  }
  unsigned long long slice = 0;
  const size_t slices = (size_t)rp::mvn_grad_slices(d, n, &slice);
  const size_t need = slices * (size_t)d * (size_t)d;
  if (need > g_mvn_cap) {
    if (g_mvn_part) cudaFree(g_mvn_part);
    g_mvn_part = nullptr;
    g_mvn_cap = 0;
    int e = (int)cudaMalloc((void**)&g_mvn_part, need * sizeof(double));
    if (e) return fail(RP_ERR_NOMEM, "mvn gradient scratch allocation failed");
    g_mvn_cap = need;
  }
  int e = rp::launch_mvn_grads(d, n, d_G, d_Z, d_gmu, d_gL, g_mvn_part, cuda_stream);
  if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e) return cuda_fail(e, "mvn grads");
  g_launches.fetch_add(4);
  return RP_OK;
}

extern "C" rp_status rp_debug_faults(int kind, uint64_t value) {
  std::lock_guard<std::mutex> lk(g_mu);
  switch (kind) {
    case 0: g_faults = DebugFaults(); return RP_OK;
    case 1: g_faults.spin_max = value; return RP_OK;
    case 2: g_faults.stall_tile1 = value; return RP_OK;
    case 3: g_faults.tail_cap = value; return RP_OK;
    case 4: g_faults.tile_cap = value; return RP_OK;
    default: return fail(RP_ERR_PARAM, "unknown debug fault kind " + std::to_string(kind));
  }
}

extern "C" rp_status rp_debug_counters(uint64_t* h_counts, int reset) {
  if (!h_counts) return fail(RP_ERR_NULL, "NULL counts pointer");
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long c[8];
  const int e = rp::debug_counters(c, reset);
  if (e) return cuda_fail(e, "debug counters");
  for (int i = 0; i < 6; ++i) h_counts[i] = c[i];
  return RP_OK;
}

extern "C" rp_status rp_exp_cr(const double* d_x, double* d_y, size_t n, void* cuda_stream) {
  if (n && (!d_x || !d_y)) return fail(RP_ERR_NULL, "NULL device pointer");
  int e = rp::launch_exp_cr(d_x, d_y, n, cuda_stream);
  if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e) return cuda_fail(e, "exp");
  g_launches.fetch_add(1);
  return RP_OK;
}

extern "C" rp_status rp_log_cr(const double* d_x, double* d_y, size_t n, void* cuda_stream) {
  if (n && (!d_x || !d_y)) return fail(RP_ERR_NULL, "NULL device pointer");
  int e = rp::launch_log_cr(d_x, d_y, n, cuda_stream);
  if (!e) e = (int)cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e) return cuda_fail(e, "log");
  g_launches.fetch_add(1);
  return RP_OK;
}
