// FP32 instantiation of the lattice kernels (links and updates in FP32; measurement
// products and accumulators in FP64).
#include "ul_kernels.cuh"

namespace ul {
UL_INSTANTIATE_KERNELS(float)
} // namespace ul
