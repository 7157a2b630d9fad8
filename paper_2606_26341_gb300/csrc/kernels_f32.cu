// FP32 factorisation (FP64 refinement) instantiation of the solver kernels for any number of
// quadrotors per problem (sizes read at run time).
#include "kernels.cuh"

namespace bipm {
void* iter_kernel_f32() { return (void*)ipm_kernel<float, float, 0>; }
void* init_kernel_f32() { return (void*)init_kernel<float, float, 0>; }
void* queue_kernel_f32() { return (void*)queue_kernel<float, float, 0>; }
void* queue_mixed_f32() { return (void*)queue_mixed_kernel<float, float, 0>; }
void* block_mixed_f32() { return (void*)block_mixed_kernel<float, float, 0>; }
}  // namespace bipm
