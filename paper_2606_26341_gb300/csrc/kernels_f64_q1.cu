// FP64 factorisation instantiation of the solver kernels specialised for one
// quadrotor per problem (12 states, 4 inputs fixed at compile time).
#include "kernels.cuh"

namespace bipm {
void* iter_kernel_f64_q1() { return (void*)ipm_kernel<double, double, 1>; }
void* queue_kernel_f64_q1() { return (void*)queue_kernel<double, double, 1>; }
}  // namespace bipm
