// Kernel dispatch of librp: engine translation units, the tail-value and
// beta-pair kernels.
#include "rp_fill_impl.cuh"

namespace rp {
int dispatch_xo(const FillArgs& a, int grid, void* s, int* occ);
int dispatch_pcg(const FillArgs& a, int grid, void* s, int* occ);
int dispatch_ph(const FillArgs& a, int grid, void* s, int* occ);
int dispatch_ph64(const FillArgs& a, int grid, void* s, int* occ);
int dispatch_xss(const FillArgs& a, int grid, void* s, int* occ);
int upload_zig_xo(const void* host2);
int batch_xo(int cls, int cvar, const BatchArgs& b, int grid, void* s, int* occ);
int batch_pcg(int cls, int cvar, const BatchArgs& b, int grid, void* s, int* occ);
int batch_ph(int cls, int cvar, const BatchArgs& b, int grid, void* s, int* occ);
int batch_ph64(int cls, int cvar, const BatchArgs& b, int grid, void* s, int* occ);
int batch_xss(int cls, int cvar, const BatchArgs& b, int grid, void* s, int* occ);
int upload_zig_pcg(const void* host2);
int upload_zig_ph(const void* host2);
int upload_zig_ph64(const void* host2);
int upload_zig_xss(const void* host2);
int dbg_xo(unsigned long long* out, int reset);
int dbg_pcg(unsigned long long* out, int reset);
int dbg_ph(unsigned long long* out, int reset);
int dbg_ph64(unsigned long long* out, int reset);
int dbg_xss(unsigned long long* out, int reset);

// Fallback counts summed over the translation units that decide (the engine
// ones and this one); reset zeroes them.
int debug_counters(unsigned long long* out, int reset) {
  for (int i = 0; i < DBG_N; ++i) out[i] = 0;
  int e = dbg_xo(out, reset);
  if (!e) e = dbg_pcg(out, reset);
  if (!e) e = dbg_ph(out, reset);
  if (!e) e = dbg_ph64(out, reset);
  if (!e) e = dbg_xss(out, reset);
  if (!e) e = dbg_read(out, reset);
  return e;
}

namespace {
int dispatch(const FillArgs& a, int grid, void* s, int* occ) {
  switch (a.eng.engine) {
    case 1: return dispatch_xo(a, grid, s, occ);
    case 2: return dispatch_pcg(a, grid, s, occ);
    case 3: return dispatch_ph(a, grid, s, occ);
    case 4: return dispatch_ph64(a, grid, s, occ);
    case 5: return dispatch_xss(a, grid, s, occ);
    default: return (int)cudaErrorInvalidValue;
  }
}
}  // namespace

int launch_fill(const FillArgs& a, int grid, void* stream) { return dispatch(a, grid, stream, nullptr); }

int launch_batch(int engine, int cls, int cvar, const BatchArgs& b, int grid, void* stream, int* occ) {
  switch (engine) {
    case 1: return batch_xo(cls, cvar, b, grid, stream, occ);
    case 2: return batch_pcg(cls, cvar, b, grid, stream, occ);
    case 3: return batch_ph(cls, cvar, b, grid, stream, occ);
    case 4: return batch_ph64(cls, cvar, b, grid, stream, occ);
    case 5: return batch_xss(cls, cvar, b, grid, stream, occ);
    default: return (int)cudaErrorInvalidValue;
  }
}

// Tail values of a batch: TailEntry.g holds the output's address.  Ziggurat
// entries carry their distribution in x[0]; gamma/beta records carry the
// request index in w1 (for its shape parameters).
__global__ void k_tails_lean_batch(BatchArgs b) {
  unsigned long long n = ld_volatile(b.tail_count);
  if (n > b.tail_cap) n = b.tail_cap;
  for (unsigned long long i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    const TailEntry te = b.tailq[i];
    const bool ex = te.x[0] == (u64)D_EXP;
    const double v = ex ? SampExp::tail_value(te.w0, te.w1, g_zig[1]) : SampNormal::tail_value(te.w0, te.w1, g_zig[0]);
    *(double*)te.g = v;
  }
}

__global__ void k_tails_rec_batch(BatchArgs b) {
  unsigned long long n = ld_volatile(b.tail_count);
  if (n > b.tail_cap) n = b.tail_cap;
  for (unsigned long long i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    const TailEntry te = b.tailq[i];
    const FillArgs& a = b.reqs[te.w1];
    const u64 r[8] = {te.w0, te.x[0], te.x[1], te.x[2], te.x[3], te.x[4], te.x[5], 0};
    const double v = a.dist == D_BETA ? SampBeta::value(r, a.sp, g_zig[0]) : SampGamma::value(r, a.sp, g_zig[0]);
    *(double*)te.g = v;
  }
}

int launch_batch_tails(int cls, const BatchArgs& b, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (cls == BC_LEAN) k_tails_lean_batch<<<304, 256, 0, s>>>(b);
  else if (cls == BC_MERGE) k_tails_rec_batch<<<304, 256, 0, s>>>(b);
  else return 0;
  return (int)cudaGetLastError();
}

TileGeom batch_geom(int cls, int cvar) {
  if (cls == BC_MERGE) return TileGeom{NTM_, CM_, MergeGeom<NTM_, CM_>::T, 0};
  const int c = cvar == 1 ? 128 : C_;
  return TileGeom{NT_, c, NT_ * c, 0};
}

__global__ void k_ctrl_reset(Ctrl* __restrict__ c) {
  Ctrl c0;
  memset(&c0, 0, sizeof(c0));
  c0.done_tile = ~0ull;
  c0.first_reject = ~0ull;
  *c = c0;
}

int launch_ctrl_reset(Ctrl* ctrl, void* stream) {
  k_ctrl_reset<<<1, 1, 0, (cudaStream_t)stream>>>(ctrl);
  return (int)cudaGetLastError();
}

__global__ void k_finish(const Ctrl* __restrict__ c, u64 start, u64* __restrict__ d_pos, u64* __restrict__ sticky,
                         int halves) {
  const unsigned err = c->err | (c->done_tile == ~0ull ? E_INCOMPLETE : 0u);
  if (err) {
    atomicOr(sticky, (u64)err);
    if (atomicAdd(sticky + 1, 1ull) == 0) sticky[2] = c->err_info;
    *d_pos = ~0ull;
  } else {
    *d_pos = start + (halves ? (c->next_pos + 1) / 2 : c->next_pos);
  }
}

int launch_finish(const Ctrl* ctrl, unsigned long long start, unsigned long long* d_pos, unsigned long long* sticky,
                  int halves, void* stream) {
  k_finish<<<1, 1, 0, (cudaStream_t)stream>>>(ctrl, start, d_pos, sticky, halves);
  return (int)cudaGetLastError();
}

int launch_tails(const FillArgs& a, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (a.dist == D_NORMAL) k_tails<SampNormal><<<304, 256, 0, s>>>(a);
  else if (a.dist == D_EXP) k_tails<SampExp><<<304, 256, 0, s>>>(a);
  else if (a.dist == D_NORMALF) k_tails<SampNormalF><<<304, 256, 0, s>>>(a);
  else if (a.dist == D_EXPF) k_tails<SampExpF><<<304, 256, 0, s>>>(a);
  else if (a.dist == D_GAMMA) k_tails_rec<SampGamma><<<304, 256, 0, s>>>(a);
  else if (a.dist == D_BETA) k_tails_rec<SampBeta><<<304, 256, 0, s>>>(a);
  else if (a.dist == D_T) k_tails_rec<SampT><<<304, 256, 0, s>>>(a);
  else return 0;
  return (int)cudaGetLastError();
}

// Beta(a, a) from consecutive Gamma(a) draws: out[j] = X / (X + Y) with
// Outputs from consecutive pairs of base variates, u0 = g[2j], u1 = g[2j+1]
// (the serial definitions draw them in this order from one stream):
//   mode 0  beta with equal shapes, X / (X + Y);
//   mode 1  F with equal degrees of freedom, (X / p0) / (Y / p1);
//   mode 2  skew normal, p0 + p1 (p2 |u0| + p3 u1), p2 = delta, p3 = sqrt(1 - delta^2).
__global__ void k_pairs(const double* __restrict__ g, double* __restrict__ out, u64 m, int mode, double p0,
                        double p1, double p2, double p3) {
  for (u64 j = blockIdx.x * (u64)blockDim.x + threadIdx.x; j < m; j += (u64)gridDim.x * blockDim.x) {
    const double2 xy = reinterpret_cast<const double2*>(g)[j];
    double v;
    if (mode == 0) v = __ddiv_rn(xy.x, __dadd_rn(xy.x, xy.y));
    else if (mode == 1) v = __ddiv_rn(__ddiv_rn(xy.x, p0), __ddiv_rn(xy.y, p1));
    else v = __dadd_rn(p0, __dmul_rn(p1, __dadd_rn(__dmul_rn(p2, fabs(xy.x)), __dmul_rn(p3, xy.y))));
    out[j] = v;
  }
}

// Beta with equal shapes, keeping each output's gamma pair.
__global__ void k_pairs_xy(const double* __restrict__ g, double* __restrict__ z, double* __restrict__ x,
                           double* __restrict__ y, u64 m) {
  for (u64 j = blockIdx.x * (u64)blockDim.x + threadIdx.x; j < m; j += (u64)gridDim.x * blockDim.x) {
    const double2 xy = reinterpret_cast<const double2*>(g)[j];
    z[j] = __ddiv_rn(xy.x, __dadd_rn(xy.x, xy.y));
    x[j] = xy.x;
    y[j] = xy.y;
  }
}

int launch_pairs_xy(const double* g, double* z, double* x, double* y, unsigned long long m, void* stream) {
  if (m == 0) return 0;
  const unsigned long long blocks = (m + 255) / 256;
  k_pairs_xy<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(g, z, x, y, m);
  return (int)cudaGetLastError();
}

int launch_pairs(const double* g, double* out, unsigned long long m, int mode, const double* p, void* stream) {
  if (!m) return 0;
  const double q[4] = {p ? p[0] : 0.0, p ? p[1] : 0.0, p ? p[2] : 0.0, p ? p[3] : 0.0};
  k_pairs<<<608, 256, 0, (cudaStream_t)stream>>>(g, out, m, mode, q[0], q[1], q[2], q[3]);
  return (int)cudaGetLastError();
}

// The library's correctly rounded log, element-wise (a check of the value
// path used by the gamma boost and the normal tails).
__global__ void k_log_cr(const double* __restrict__ x, double* __restrict__ y, unsigned long long n) {
  for (unsigned long long i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    y[i] = cr_log_fast(x[i]);
}

int launch_log_cr(const double* x, double* y, unsigned long long n, void* stream) {
  if (!n) return 0;
  k_log_cr<<<608, 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return (int)cudaGetLastError();
}

__global__ void k_exp_cr(const double* __restrict__ x, double* __restrict__ y, unsigned long long n) {
  for (unsigned long long i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    y[i] = cr_exp_dev(x[i]);
}

int launch_exp_cr(const double* x, double* y, unsigned long long n, void* stream) {
  if (!n) return 0;
  k_exp_cr<<<608, 256, 0, (cudaStream_t)stream>>>(x, y, n);
  return (int)cudaGetLastError();
}

int occupancy_blocks(int engine, int dist, int epi) {
  FillArgs a{};
  a.eng.engine = engine;
  a.dist = dist;
  a.sp.epi = epi;
  int occ = 0;
  dispatch(a, 0, 0, &occ);
  return occ;
}

TileGeom tile_geom(int engine, int dist, int gamma_boost) {
  (void)engine;
  if (dist == D_GAMMA && gamma_boost)
    return TileGeom{NTM_, SampGammaBoost::kChunk, MergeGeom<NTM_, SampGammaBoost::kChunk>::T, 0};
  if (dist == D_GAMMA) return TileGeom{NTM_, SampGamma::kChunk, MergeGeom<NTM_, SampGamma::kChunk>::T, 0};
  if (dist == D_BETA) return TileGeom{NTM_, SampBeta::kChunk, MergeGeom<NTM_, SampBeta::kChunk>::T, 0};
  if (dist == D_T) return TileGeom{NTM_, SampT::kChunk, MergeGeom<NTM_, SampT::kChunk>::T, 0};
  // half-word fills: the kernel's chunk of C_ half-words is C_ / 2 words
  if (dist == D_NORMALF || dist == D_EXPF) return TileGeom{NT_, C_ / 2, NT_ * C_ / 2, 0};
  if (dist == D_BOUNDED) return TileGeom{NT_, CR_, NT_ * CR_, 0};
  return TileGeom{NT_, C_, NT_ * C_, 0};
}

int upload_zig(const void* host2) {
  int e = (int)cudaMemcpyToSymbol(g_zig, host2, 2 * sizeof(ZigDev));
  if (!e) e = upload_zig_xo(host2);
  if (!e) e = upload_zig_pcg(host2);
  if (!e) e = upload_zig_ph(host2);
  if (!e) e = upload_zig_ph64(host2);
  if (!e) e = upload_zig_xss(host2);
  return e;
}

}  // namespace rp
