// FP64 factorisation instantiation of the solver kernels for any number of
// quadrotors per problem (sizes read at run time).
#include "kernels.cuh"

namespace bipm {
void* iter_kernel_f64() { return (void*)ipm_kernel<double, double, 0>; }
void* init_kernel_f64() { return (void*)init_kernel<double, double, 0>; }
void* queue_kernel_f64() { return (void*)queue_kernel<double, double, 0>; }
void* queue_mixed_f64() { return (void*)queue_mixed_kernel<double, double, 0>; }
void* block_mixed_f64() { return (void*)block_mixed_kernel<double, double, 0>; }
}  // namespace bipm
