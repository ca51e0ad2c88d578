// Multivariate normal samples x = mu + L z (Sec. 3.1, multivariate normal)
// and their gradients, on the FP64 tensor cores (mma.sync m8n8k4 f64).
//
// Layout: Z and X are n x d row-major (sample-major: sample j's d components
// are consecutive), L is d x d row-major lower triangular (entries above the
// diagonal are never read), mu has d entries.
//
//   forward:  X = Z L^T + mu                 (M = n samples, N = d, K = d)
//   backward: dL/dmu = sum_j G_j             (column sums of G)
//             dL/dL  = tril(G^T Z)           (M = d, N = d, K = n, split over
//                                             sample slices, partial tiles
//                                             summed in a fixed order)
//
// Tiles: 64 x 64 outputs per CTA, K in chunks of 16 staged in shared memory,
// four warps of 32 x 32 (4 x 4 m8n8 accumulators each).  Triangular L lets
// the forward stop its K loop at the tile's last row, and the backward skip
// tiles above the diagonal.
#include <cuda_runtime.h>

#include <algorithm>

#include "rp_internal.h"

namespace rp {
namespace {

typedef unsigned long long u64;
constexpr int BM = 64, BN = 64, BK = 16, LDW = BK + 4;   // padded rows: conflict-free fragment loads

// D += A B for one m8n8k4 tile: a = A[lane/4][lane%4], b = B[lane%4][lane/4],
// d = D[lane/4][2 (lane%4) + {0, 1}].
__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d[0]), "+d"(d[1])
               : "d"(a), "d"(b));
}

// Warp tile update from the staged chunk: As[m][k] (rows of A), Bs[n][k]
// (columns of B), both BK wide.
__device__ __forceinline__ void warp_mma(double (&acc)[4][4][2], const double (*As)[LDW], const double (*Bs)[LDW],
                                         int wm, int wn, int lane) {
#pragma unroll
  for (int kk = 0; kk < BK; kk += 4) {
    double a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = As[wm + i * 8 + (lane >> 2)][kk + (lane & 3)];
      b[i] = Bs[wn + i * 8 + (lane >> 2)][kk + (lane & 3)];
    }
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) dmma(acc[mi][ni], a[mi], b[ni]);
  }
}

__global__ void __launch_bounds__(128) k_mvn_apply(int d, u64 n, const double* __restrict__ mu,
                                                   const double* __restrict__ L, const double* __restrict__ Z,
                                                   double* __restrict__ X) {
  __shared__ double As[BM][LDW], Bs[BN][LDW];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const u64 m0 = (u64)blockIdx.x * BM;   // samples
  const int n0 = blockIdx.y * BN;        // output components
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
  const int kend = min(d, n0 + BN);      // L[i][k] = 0 for k > i
  for (int k0 = 0; k0 < kend; k0 += BK) {
    for (int e = t; e < BM * BK; e += 128) {
      const int r = e / BK, c = e % BK, k = k0 + c;
      const u64 j = m0 + r;
      As[r][c] = (j < n && k < d) ? Z[j * (u64)d + k] : 0.0;
      const int i = n0 + r;
      Bs[r][c] = (i < d && k <= i) ? L[(u64)i * d + k] : 0.0;
    }
    __syncthreads();
    warp_mma(acc, As, Bs, wm, wn, lane);
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 4; ++mi) {
    const u64 row = m0 + wm + mi * 8 + (lane >> 2);
    if (row >= n) continue;
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int col = n0 + wn + ni * 8 + (lane & 3) * 2 + h;
        if (col < d) X[row * (u64)d + col] = __dadd_rn(acc[mi][ni][h], mu[col]);
      }
  }
}

// Partial tiles of G^T Z over one slice of samples: part[s][i][k] for the
// tile (blockIdx.x, blockIdx.y) = (i tile, k tile) with i tile >= k tile.
__global__ void __launch_bounds__(128) k_mvn_gl_part(int d, u64 n, u64 slice, const double* __restrict__ G,
                                                     const double* __restrict__ Z, double* __restrict__ part) {
  const int ti = blockIdx.x, tk = blockIdx.y;
  if (tk > ti) return;
  __shared__ double As[BM][LDW], Bs[BN][LDW];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int i0 = ti * BM, k0t = tk * BN;
  const u64 s = blockIdx.z, j0 = s * slice, j1 = min(n, j0 + slice);
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;
  for (u64 jb = j0; jb < j1; jb += BK) {
    // A = G^T (rows i, columns j), B = Z (rows j, columns k): stage As[i][j], Bs[k][j]
    for (int e = t; e < BK * BM; e += 128) {
      const int r = e / BM, c = e % BM;   // r: sample within the chunk, c: component (coalesced)
      const u64 j = jb + r;
      const int i = i0 + c, k = k0t + c;
      As[c][r] = (j < j1 && i < d) ? G[j * (u64)d + i] : 0.0;
      Bs[c][r] = (j < j1 && k < d) ? Z[j * (u64)d + k] : 0.0;
    }
    __syncthreads();
    warp_mma(acc, As, Bs, wm, wn, lane);
    __syncthreads();
  }
  double* P = part + s * (u64)d * d;
#pragma unroll
  for (int mi = 0; mi < 4; ++mi) {
    const int row = i0 + wm + mi * 8 + (lane >> 2);
    if (row >= d) continue;
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int col = k0t + wn + ni * 8 + (lane & 3) * 2 + h;
        if (col < d) P[(u64)row * d + col] = acc[mi][ni][h];
      }
  }
}

// gL[i][k] = sum over slices in order (k <= i), 0 above the diagonal.
__global__ void k_mvn_gl_sum(int d, int slices, const double* __restrict__ part, double* __restrict__ gL) {
  const u64 dd = (u64)d * d;
  for (u64 e = blockIdx.x * (u64)blockDim.x + threadIdx.x; e < dd; e += (u64)gridDim.x * blockDim.x) {
    const int i = (int)(e / d), k = (int)(e % d);
    double v = 0.0;
    if (k <= i)
      for (int s = 0; s < slices; ++s) v = __dadd_rn(v, part[(u64)s * dd + e]);
    gL[e] = v;
  }
}

// Column sums of G over sample slices: part[s][i], then a fixed-order sum.
__global__ void k_mvn_gmu_part(int d, u64 n, u64 slice, const double* __restrict__ G, double* __restrict__ part) {
  const u64 s = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  const u64 j0 = s * slice, j1 = min(n, j0 + slice);
  double v = 0.0;
  for (u64 j = j0; j < j1; ++j) v = __dadd_rn(v, G[j * (u64)d + i]);
  part[s * (u64)d + i] = v;
}

__global__ void k_mvn_gmu_sum(int d, int slices, const double* __restrict__ part, double* __restrict__ gmu) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d) return;
  double v = 0.0;
  for (int s = 0; s < slices; ++s) v = __dadd_rn(v, part[(u64)s * d + i]);
  gmu[i] = v;
}

}  // namespace

int launch_mvn_apply(int d, unsigned long long n, const double* mu, const double* L, const double* Z, double* X,
                     void* stream) {
  dim3 grid((unsigned)((n + BM - 1) / BM), (unsigned)((d + BN - 1) / BN));
  k_mvn_apply<<<grid, 128, 0, (cudaStream_t)stream>>>(d, n, mu, L, Z, X);
  return (int)cudaGetLastError();
}

// Sample slices of the backward GEMM: enough CTAs for about four per SM
// over the lower-triangular tile pairs, each slice a whole number of K chunks.
int mvn_grad_slices(int d, unsigned long long n, unsigned long long* slice) {
  const unsigned long long tiles = (unsigned long long)((d + BM - 1) / BM);
  const unsigned long long lower = tiles * (tiles + 1) / 2;
  unsigned long long want = (4ull * 152 + lower - 1) / lower;
  if (want < 1) want = 1;
  unsigned long long s = (n + want - 1) / want;
  s = (s + BK - 1) / BK * BK;
  if (s < BK) s = BK;
  *slice = s;
  return (int)((n + s - 1) / s);
}

int launch_mvn_grads(int d, unsigned long long n, const double* G, const double* Z, double* gmu, double* gL,
                     double* part, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long slice = 0;
  const int slices = mvn_grad_slices(d, n, &slice);
  const int tiles = (d + BM - 1) / BM;
  k_mvn_gl_part<<<dim3(tiles, tiles, slices), 128, 0, st>>>(d, n, slice, G, Z, part);
  k_mvn_gl_sum<<<(int)std::min<unsigned long long>(((unsigned long long)d * d + 255) / 256, 4096), 256, 0, st>>>(
      d, slices, part, gL);
  k_mvn_gmu_part<<<dim3((d + 127) / 128, slices), 128, 0, st>>>(d, n, slice, G, part);
  k_mvn_gmu_sum<<<(d + 127) / 128, 128, 0, st>>>(d, slices, part, gmu);
  return (int)cudaGetLastError();
}

}  // namespace rp
