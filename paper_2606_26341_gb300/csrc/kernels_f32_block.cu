// FP32 factorisation (FP64 refinement) instantiation of the block-team kernel.
#include "kernels.cuh"

namespace bipm {
void* block_kernel_f32() { return (void*)ipm_block_kernel<float, float>; }
}  // namespace bipm
