// FP64 factorisation instantiation of the solver kernels.
#include "kernels.cuh"

namespace bipm {
void* iter_kernel_f64() { return (void*)ipm_kernel<double, double>; }
void* init_kernel_f64() { return (void*)init_kernel<double, double>; }
void* queue_kernel_f64() { return (void*)queue_kernel<double, double>; }
void* queue_mixed_f64() { return (void*)queue_mixed_kernel<double, double>; }
void* block_mixed_f64() { return (void*)block_mixed_kernel<double, double>; }
}  // namespace bipm
