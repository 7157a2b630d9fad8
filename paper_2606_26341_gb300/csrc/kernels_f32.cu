// FP32 factorisation (FP64 refinement) instantiation of the solver kernels.
#include "kernels.cuh"

namespace bipm {
void* iter_kernel_f32() { return (void*)ipm_kernel<float, float>; }
void* init_kernel_f32() { return (void*)init_kernel<float, float>; }
void* queue_kernel_f32() { return (void*)queue_kernel<float, float>; }
void* queue_mixed_f32() { return (void*)queue_mixed_kernel<float, float>; }
void* block_mixed_f32() { return (void*)block_mixed_kernel<float, float>; }
}  // namespace bipm
