// Fill kernels of librp (sm_103a).
//
// One stream is cut into tiles of T = NT*C consecutive words.  Persistent
// CTAs take tiles round-robin (tile k by CTA k mod grid); inside a tile
// thread t generates the C words of chunk t (its engine state reaches the
// next tile's chunk by one constant jump) into shared memory.
//
// Samplers that consume one word per variate write the tile straight out.
// Rejection samplers run the speculative parse (Sec. 3 samplers, parallel
// form of this library):
//   1. every position p can compute len(p), the words a candidate starting at
//      p would consume; reach(p) = p + len(p);
//   2. a position s is a sync point when no candidate starting in the G
//      positions before s reaches beyond s, so any chain of candidates that
//      enters that window passes through s.  Thread t takes the first sync
//      point of its chunk; the tile start is the first sync point in
//      [G, G+S) of the tile, computed identically by the previous tile from
//      its halo words;
//   3. each thread walks the true chain from its sync point to the next one,
//      checks that it lands exactly on it (otherwise a candidate longer than
//      the window existed: the launch reports E_LANDING and the host retries
//      with a wider window) and records the positions of accepted candidates;
//   4. a block scan gives in-tile output offsets; a decoupled look-back over
//      tile counts gives the tile's first output index;
//   5. outputs are evaluated and written with consecutive threads on
//      consecutive indices (coalesced).
#include <cuda_runtime.h>

#include <cstdio>

#include "rp_device.cuh"
#include "rp_internal.h"

namespace rp {

__device__ ZigDev g_zig[2];

namespace {

constexpr u64 M52 = (1ull << 52) - 1;
constexpr u64 M53 = (1ull << 53) - 1;
constexpr int kG = 8;        // look-back window of a sync point
constexpr int kS = 16;       // search window for the tile-start sync point
constexpr int kH = 64;       // halo words generated past the tile end
constexpr unsigned long long kSpinMax = 1ull << 24;  // bounded waits (x ~200 ns)

// ------------------------------------------------------------------ samplers
// Every sampler reads words through W(p) (padded shared-memory layout).
template <int C>
struct Buf {
  const u64* w;
  int lim;  // number of valid positions
  __device__ __forceinline__ u64 operator()(int p) const { return w[p + (p / C)]; }
};

struct SampU64 {
  static constexpr bool kTrivial = true;
  static constexpr bool kLen1 = true;
  typedef u64 out_t;
  __device__ static __forceinline__ u64 value1(u64 u, const SampArgs&) { return u; }
};

struct SampUniform {
  static constexpr bool kTrivial = true;
  static constexpr bool kLen1 = true;
  typedef double out_t;
  __device__ static __forceinline__ double value1(u64 u, const SampArgs&) { return u53_bits(u); }
};

// Lemire (Sec. 3.2): one word per attempt, accept when low64(u m) >= 2^64 mod m.
struct SampBounded {
  static constexpr bool kTrivial = false;
  static constexpr bool kLen1 = true;
  typedef u64 out_t;
  template <class B>
  __device__ static __forceinline__ int len(const B&, int, const ZigDev&) { return 1; }
  template <class B>
  __device__ static __forceinline__ bool acc(const B& w, int p, const ZigDev&, const SampArgs& a) {
    return w(p) * a.m >= a.thresh;
  }
  template <class B>
  __device__ static __forceinline__ u64 value(const B& w, int p, const ZigDev&, const SampArgs& a) {
    return __umul64hi(w(p), a.m);
  }
};

// Normal ziggurat (Sec. 3.1): bits 0-7 strip, bit 8 sign, bits 9-60 r.
struct SampNormal {
  static constexpr bool kTrivial = false;
  static constexpr bool kLen1 = false;
  typedef double out_t;
  template <class B>
  __device__ static int len(const B& w, int p, const ZigDev& z) {
    u64 u = w(p);
    int i = (int)(u & 0xff);
    u64 r = (u >> 9) & M52;
    if (r < z.k[i]) return 1;
    if (i != 0) return (p + 1 < w.lim) ? 2 : 0;
    int q = p + 1;
    for (;;) {  // tail pairs until 2b > a^2
      if (q + 1 >= w.lim) return 0;
      double a, b;
      tail_pair(w(q), w(q + 1), z.R, a, b);
      q += 2;
      if (__dadd_rn(b, b) > __dmul_rn(a, a)) return q - p;
    }
  }
  __device__ static __forceinline__ void tail_pair(u64 w1, u64 w2, double R, double& a, double& b) {
    double U1 = u53_bits(w1), U2 = u53_bits(w2);
    a = __ddiv_rn(-cr_log_dev(__dsub_rn(1.0, U1)), R);
    b = -cr_log_dev(__dsub_rn(1.0, U2));
  }
  __device__ static __forceinline__ double xval(u64 u, const ZigDev& z) {
    int i = (int)(u & 0xff);
    u64 r = (u >> 9) & M52;
    double x = mul_rn_int(r, z.msh[i], z.wtz[i], z.we[i]);
    return ((u >> 8) & 1) ? -x : x;
  }
  template <class B>
  __device__ static bool acc(const B& w, int p, const ZigDev& z, const SampArgs&) {
    u64 u = w(p);
    int i = (int)(u & 0xff);
    u64 r = (u >> 9) & M52;
    if (r < z.k[i] || i == 0) return true;
    double x = xval(u, z);
    double U = u53_bits(w(p + 1));
    double y = __dadd_rn(__dmul_rn(__dsub_rn(z.f[i - 1], z.f[i]), U), z.f[i]);
    double t = __dmul_rn(-0.5, __dmul_rn(x, x));
    return lt_cr_exp(y, t);
  }
  template <class B>
  __device__ static double value(const B& w, int p, const ZigDev& z, const SampArgs&) {
    u64 u = w(p);
    int i = (int)(u & 0xff);
    u64 r = (u >> 9) & M52;
    if (r < z.k[i] || i != 0) return xval(u, z);
    int q = p + 1;
    for (;;) {
      double a, b;
      tail_pair(w(q), w(q + 1), z.R, a, b);
      q += 2;
      if (__dadd_rn(b, b) > __dmul_rn(a, a)) {
        double v = __dadd_rn(z.R, a);
        return ((u >> 8) & 1) ? -v : v;
      }
    }
  }
};

// Exponential ziggurat (Sec. 3.1): bits 0-7 strip, bits 8-60 r; memoryless tail.
struct SampExp {
  static constexpr bool kTrivial = false;
  static constexpr bool kLen1 = false;
  typedef double out_t;
  template <class B>
  __device__ static __forceinline__ int len(const B& w, int p, const ZigDev& z) {
    u64 u = w(p);
    int i = (int)(u & 0xff);
    u64 r = (u >> 8) & M53;
    if (r < z.k[i]) return 1;
    return (p + 1 < w.lim) ? 2 : 0;
  }
  __device__ static __forceinline__ double xval(u64 u, const ZigDev& z) {
    int i = (int)(u & 0xff);
    return mul_rn_int((u >> 8) & M53, z.msh[i], z.wtz[i], z.we[i]);
  }
  template <class B>
  __device__ static bool acc(const B& w, int p, const ZigDev& z, const SampArgs&) {
    u64 u = w(p);
    int i = (int)(u & 0xff);
    u64 r = (u >> 8) & M53;
    if (r < z.k[i] || i == 0) return true;
    double x = xval(u, z);
    double U = u53_bits(w(p + 1));
    double y = __dadd_rn(__dmul_rn(__dsub_rn(z.f[i - 1], z.f[i]), U), z.f[i]);
    return lt_cr_exp(y, -x);
  }
  template <class B>
  __device__ static double value(const B& w, int p, const ZigDev& z, const SampArgs&) {
    u64 u = w(p);
    int i = (int)(u & 0xff);
    u64 r = (u >> 8) & M53;
    if (r < z.k[i] || i != 0) return xval(u, z);
    double U = u53_bits(w(p + 1));
    return __dsub_rn(z.R, cr_log_dev(__dsub_rn(1.0, U)));
  }
};

// ------------------------------------------------------------------ helpers
template <class S, class B>
__device__ int sync_point(const B& w, int q0, int s0, int s1, const ZigDev& z, int* ovf) {
  // first s in [s0, s1) with q + len(q) <= s for every q in [q0, s); -1 if none
  int reach = 0;
  for (int q = q0; q < s0; ++q) {
    int L = S::len(w, q, z);
    if (L == 0) { *ovf = 1; return -1; }
    reach = max(reach, q + L);
  }
  for (int s = s0; s < s1; ++s) {
    if (reach <= s) return s;
    int L = S::len(w, s, z);
    if (L == 0) { *ovf = 1; return -1; }
    reach = max(reach, s + L);
  }
  return -1;
}

__device__ __forceinline__ void set_err(Ctrl* c, unsigned e, unsigned long long info) {
  atomicOr(&c->err, e);
  atomicExch(&c->err_info, info);
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *(volatile const unsigned long long*)p;
}

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

// Decoupled look-back over tile counts.  Status word: bit 63 aggregate,
// bit 62 inclusive, low 62 bits value.  Returns the tile's exclusive prefix or
// ~0 if the wait timed out or the tile became unnecessary.
__device__ unsigned long long lookback(unsigned long long* st, unsigned long long k, unsigned long long cnt,
                                       Ctrl* ctrl) {
  const unsigned long long AGG = 1ull << 63, INC = 1ull << 62, VAL = INC - 1;
  if (k == 0) {
    *(volatile unsigned long long*)(st) = INC | cnt;
    return 0;
  }
  *(volatile unsigned long long*)(st + k) = AGG | cnt;
  unsigned long long excl = 0;
  long long j = (long long)k - 1;
  unsigned long long spins = 0;
  while (j >= 0) {
    unsigned long long v = ld_volatile(st + j);
    if (v & INC) { excl += v & VAL; break; }
    if (v & AGG) { excl += v & VAL; --j; continue; }
    if (ld_volatile(&ctrl->done_tile) < k) return ~0ull;
    if (++spins > kSpinMax) { set_err(ctrl, E_TIMEOUT, k); return ~0ull; }
    __nanosleep(128);
  }
  *(volatile unsigned long long*)(st + k) = INC | (excl + cnt);
  return excl;
}

// ------------------------------------------------------------------ the kernel
template <int NT, int C, class E, class S>
__global__ void __launch_bounds__(NT) k_fill(FillArgs a) {
  constexpr int T = NT * C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  u64* words = (u64*)smem_raw;                                   // (T + kH) padded
  constexpr int WPAD = T + kH + (T + kH) / C + 2;
  unsigned short* tmp = (unsigned short*)(words + WPAD);         // T + kH
  unsigned short* opos = tmp + (T + kH);                         // T + kH
  int* sig = (int*)(opos + (T + kH));                            // NT
  int* wsum = sig + NT;                                          // 32
  int* misc = wsum + 32;                                         // 8
  ZigDev* zs = (ZigDev*)(misc + 8);                              // shared copy (normal/exp)

  const int t = threadIdx.x;
  const ZigDev* zp = &g_zig[0];
  if (!S::kTrivial && !S::kLen1) {
    const int which = (a.dist == D_EXP) ? 1 : 0;
    const u64* src = (const u64*)&g_zig[which];
    u64* dst = (u64*)zs;
    for (int i = t; i < (int)(sizeof(ZigDev) / 8); i += NT) dst[i] = src[i];
    zp = zs;
    __syncthreads();
  }
  const ZigDev& z = *zp;

  // engine state at the start of this thread's chunk in the CTA's first tile
  E e;
  e.init(a.eng, (u64)blockIdx.x * T + (u64)t * C);

  for (u64 k = blockIdx.x; k < a.n_tiles; k += gridDim.x) {
    if (!S::kTrivial && ld_volatile(&a.ctrl->done_tile) < k) break;
    // ---- generate the tile (and the halo past its end) into shared memory
    {
      E g = e;
      u64* dst = words + t * (C + 1);
#pragma unroll 8
      for (int i = 0; i < C; ++i) dst[i] = g.next();
      if (!S::kTrivial && !S::kLen1 && t == NT - 1) {
        for (int i = 0; i < kH; ++i) {
          int p = T + i;
          words[p + p / C] = g.next();
        }
      }
      e.advance(a.eng);
    }
    __syncthreads();

    if constexpr (S::kTrivial) {
      typedef typename S::out_t OT;
      OT* out = (OT*)a.out;
      u64 base = k * (u64)T;
      u64 lim = a.n - base < (u64)T ? a.n - base : (u64)T;
      for (int j = t; j < (int)lim; j += NT) out[base + j] = S::value1(words[j + j / C], a.sp);
      __syncthreads();
      continue;
    } else {
      typedef typename S::out_t OT;
      Buf<C> w{words, T + (S::kLen1 ? 0 : kH)};
      int ovf = 0;
      const int b = t * C;
      // ---- sync points
      int s_t;
      if (S::kLen1) {
        s_t = b;
      } else if (t == 0) {
        s_t = (k == 0) ? 0 : sync_point<S>(w, 0, kG, kG + kS, z, &ovf);
        if (s_t < 0 && !ovf) set_err(a.ctrl, E_NOSYNC, k);
      } else {
        s_t = sync_point<S>(w, b - kG, b, b + C, z, &ovf);
      }
      if (ovf) set_err(a.ctrl, E_OVERFLOW, k);
      sig[t] = s_t;
      __syncthreads();
      // ---- walk own segment, record accepted positions at tmp[s_t ...]
      int cnt = 0;
      int end = -1;
      if (s_t >= 0) {
        for (int u = t + 1; u < NT; ++u)
          if (sig[u] >= 0) { end = sig[u]; break; }
        if (end < 0) {
          if (S::kLen1) end = T;
          else {
            int o2 = 0;
            end = sync_point<S>(w, T, T + kG, T + kG + kS, z, &o2);
            if (end < 0) { set_err(a.ctrl, o2 ? E_OVERFLOW : E_NOSYNC, k); end = T; }
            misc[0] = end;
          }
        }
        int p = s_t;
        while (p < end) {
          int L = S::len(w, p, z);
          if (L == 0) { set_err(a.ctrl, E_OVERFLOW, k); break; }
          if (S::acc(w, p, z, a.sp)) tmp[s_t + cnt++] = (unsigned short)p;
          p += L;
        }
        if (p != end) set_err(a.ctrl, E_LANDING, k);
      }
      // ---- in-tile offsets
      int off = block_exclusive_scan<NT>(cnt, wsum, &misc[1]);
      for (int j = 0; j < cnt; ++j) opos[off + j] = tmp[s_t + j];
      if (t == 0) {
        unsigned long long ex = lookback(a.tile_status, k, (unsigned long long)misc[1], a.ctrl);
        misc[2] = (int)(ex & 0x7fffffff);
        misc[3] = (int)(ex >> 31);
        misc[4] = (ex == ~0ull);
      }
      __syncthreads();
      if (misc[4]) break;
      const int tc = misc[1];
      const u64 base = (u64)(unsigned)misc[2] | ((u64)(unsigned)misc[3] << 31);
      OT* out = (OT*)a.out;
      if (base < a.n) {
        for (int j = t; j < tc; j += NT) {
          u64 g = base + j;
          if (g < a.n) {
            int p = opos[j];
            out[g] = S::value(w, p, z, a.sp);
            if (g == a.n - 1) {
              a.ctrl->next_pos = k * (u64)T + p + S::len(w, p, z);
              atomicMin(&a.ctrl->done_tile, k);
            }
          }
        }
      }
      if (t == 0 && k + 1 == a.n_tiles && base + tc < a.n) {
        // ran out of tiles: report where the chain continues
        a.ctrl->total = base + tc;
        a.ctrl->next_pos = k * (u64)T + (S::kLen1 ? T : misc[0]);
        a.ctrl->last_tile = k;
      }
      __syncthreads();
    }
  }
}

template <int NT, int C, class E, class S>
int smem_bytes_for() {
  constexpr int T = NT * C;
  if (S::kTrivial) return (T + T / C + 2) * 8;
  constexpr int WPAD = T + kH + (T + kH) / C + 2;
  int b = WPAD * 8 + 2 * (T + kH) * 2 + (NT + 40) * 4;
  b = (b + 15) & ~15;
  return b + (int)sizeof(ZigDev);
}

template <int NT, int C, class E, class S>
int launch_t(const FillArgs& a, int grid, cudaStream_t s) {
  int smem = smem_bytes_for<NT, C, E, S>();
  static bool attr = false;
  if (!attr) {
    cudaError_t r = cudaFuncSetAttribute(k_fill<NT, C, E, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (r != cudaSuccess) return (int)r;
    attr = true;
  }
  k_fill<NT, C, E, S><<<grid, NT, smem, s>>>(a);
  return (int)cudaGetLastError();
}

template <int NT, int C, class E, class S>
int occ_t() {
  int smem = smem_bytes_for<NT, C, E, S>();
  cudaFuncSetAttribute(k_fill<NT, C, E, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fill<NT, C, E, S>, NT, smem);
  return nb;
}

constexpr int NT_ = 128;
constexpr int C_ = 64;

template <class E>
int dispatch_dist(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  switch (a.dist) {
    case D_U64: return occ ? (*occ = occ_t<NT_, C_, E, SampU64>(), 0) : launch_t<NT_, C_, E, SampU64>(a, grid, s);
    case D_UNIFORM: return occ ? (*occ = occ_t<NT_, C_, E, SampUniform>(), 0) : launch_t<NT_, C_, E, SampUniform>(a, grid, s);
    case D_BOUNDED: return occ ? (*occ = occ_t<NT_, C_, E, SampBounded>(), 0) : launch_t<NT_, C_, E, SampBounded>(a, grid, s);
    case D_NORMAL: return occ ? (*occ = occ_t<NT_, C_, E, SampNormal>(), 0) : launch_t<NT_, C_, E, SampNormal>(a, grid, s);
    case D_EXP: return occ ? (*occ = occ_t<NT_, C_, E, SampExp>(), 0) : launch_t<NT_, C_, E, SampExp>(a, grid, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

int dispatch(const FillArgs& a, int grid, cudaStream_t s, int* occ) {
  switch (a.eng.engine) {
    case 1: return dispatch_dist<XoshiroDev>(a, grid, s, occ);
    case 2: return dispatch_dist<PcgDev>(a, grid, s, occ);
    case 3: return dispatch_dist<PhiloxDev>(a, grid, s, occ);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace

int launch_fill(const FillArgs& a, int grid, void* stream) { return dispatch(a, grid, (cudaStream_t)stream, nullptr); }

int occupancy_blocks(int engine, int dist) {
  FillArgs a{};
  a.eng.engine = engine;
  a.dist = dist;
  int occ = 0;
  dispatch(a, 0, 0, &occ);
  return occ;
}

TileGeom tile_geom(int engine, int dist) {
  (void)engine;
  (void)dist;
  return TileGeom{NT_, C_, NT_ * C_, 0};
}

int upload_zig(const void* host2) {
  return (int)cudaMemcpyToSymbol(g_zig, host2, 2 * sizeof(ZigDev));
}

}  // namespace rp
