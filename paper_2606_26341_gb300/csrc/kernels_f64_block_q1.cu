// FP64 factorisation instantiation of the block-team kernel for one quadrotor per
// problem (sizes fixed at compile time).
#include "kernels.cuh"

namespace bipm {
void* block_kernel_f64_q1() { return (void*)ipm_block_kernel<double, double, 1>; }
}  // namespace bipm
