// FP64 factorisation instantiation of the block-team kernel (sizes read at run time).
#include "kernels.cuh"

namespace bipm {
void* block_kernel_f64() { return (void*)ipm_block_kernel<double, double, 0>; }
}  // namespace bipm
