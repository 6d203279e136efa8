// FP64 instantiation of the lattice kernels.  Compiled with -fmad=false: the only fused
// multiply-adds are the explicit fma() calls of the elementary functions, so the link
// updates follow a fixed IEEE operation sequence.
#include "ul_kernels.cuh"

namespace ul {
UL_INSTANTIATE_KERNELS(double)
} // namespace ul
