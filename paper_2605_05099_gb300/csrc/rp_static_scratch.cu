// Fixed device scratch of the normal fill that allocates nothing
// (rp_fill_normal_philox_static).  The block lives in this module's global
// memory, so it exists from the moment the module is loaded on a device and
// no allocation routine is ever called for it.  Layout (64-bit words):
//   [0, kStaticCtrlWords)            control block (Ctrl, padded to 256 bytes)
//   [kStaticCtrlWords, + kStaticTiles)  tile status words of the look-back
//   then kStaticTailCap tail-queue entries (TailEntry)
// One block per device and process: every call on a device uses the same
// words, so two calls in flight at once would race on them.
#include <cuda_runtime.h>

#include "rp_internal.h"

namespace rp {
namespace {
static __device__ __align__(256) unsigned long long g_static_scratch[kStaticWords];
}  // namespace

// Address of the block on the current device; returns a cudaError_t value.
int static_scratch_address(void** p) { return (int)cudaGetSymbolAddress(p, g_static_scratch); }

}  // namespace rp
