// FP32 instantiation of the lattice kernels (links, updates and per-sample products in FP32;
// accumulators in FP64).  Compiled with -fmad=false like the FP64 unit: every fused
// multiply-add is written out, so each kernel evaluates a link update the same way.
#include "ul_kernels.cuh"

namespace ul {
UL_INSTANTIATE_KERNELS(float)

int class_block_threads(long work, bool fp32) { return fp32 ? wide_block_threads(work) : update_block_threads(work); }
} // namespace ul
