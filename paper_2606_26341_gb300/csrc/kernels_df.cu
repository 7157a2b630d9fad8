// Double-float factorisation instantiation of the solver kernels (FP32
// derivative blocks, double-float factorisation and solves, FP64 elsewhere).
#include "kernels.cuh"

namespace bipm {
void* iter_kernel_df() { return (void*)ipm_kernel<float, df>; }
void* init_kernel_df() { return (void*)init_kernel<float, df>; }
void* queue_kernel_df() { return (void*)queue_kernel<float, df>; }
}  // namespace bipm
