// Test helper: raw Philox4x32-10 blocks from cuRAND's device API, used as a
// black-box reference for the Philox bijection.  For each i < nblocks the
// block at counter (0, 0, subseq lo, subseq hi) + i with key = seed is
// written to out[4 i .. 4 i + 3].
#include <curand_kernel.h>

__global__ void k_blocks(unsigned long long seed, unsigned long long subseq, int nblocks, unsigned* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed, subseq, 0, &st);
  for (int i = 0; i < nblocks; ++i) {
    uint4 v = curand4(&st);
    out[4 * i] = v.x; out[4 * i + 1] = v.y; out[4 * i + 2] = v.z; out[4 * i + 3] = v.w;
  }
}

extern "C" int curand_philox_blocks(unsigned long long seed, unsigned long long subseq, int nblocks, unsigned* h_out) {
  unsigned* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned) * 4 * (size_t)nblocks) != cudaSuccess) return 1;
  k_blocks<<<1, 1>>>(seed, subseq, nblocks, d);
  cudaError_t e = cudaMemcpy(h_out, d, sizeof(unsigned) * 4 * (size_t)nblocks, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? 0 : 2;
}
