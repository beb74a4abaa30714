// static_scratch.cu -- the device scratch of dt_aggregate_noalloc: a file-scope array that is
// part of the library's device code, so that the call itself never allocates. The CUDA
// driver reserves it on a device when this module's code is loaded into the device's
// context: under lazy module loading (the default) at the first cudaGetSymbolAddress of it;
// under eager loading (CUDA_MODULE_LOADING=EAGER) when the context is created, whether the
// entry point is ever called or not. It has its own translation unit so that, under lazy
// loading, the other calls never load it.
#include "kernels.h"

namespace zncc {

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

cudaError_t noalloc_scratch_address(void** p) { return cudaGetSymbolAddress(p, g_noalloc_scratch); }

}  // namespace zncc
