// FP32 factorisation (FP64 refinement) instantiation of the block-team kernel for one quadrotor per
// problem (sizes fixed at compile time).
#include "kernels.cuh"

namespace bipm {
void* block_kernel_f32_q1() { return (void*)ipm_block_kernel<float, float, 1>; }
}  // namespace bipm
