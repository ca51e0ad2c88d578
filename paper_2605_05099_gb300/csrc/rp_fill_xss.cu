// XoshiroSSDev (xoshiro256**) instantiations of the fill kernels (one
// translation unit per engine keeps the build parallel).
#include "rp_fill_impl.cuh"

RP_ENGINE_TU(xss, XoshiroSSDev)
