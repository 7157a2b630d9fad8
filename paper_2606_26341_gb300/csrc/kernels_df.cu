// Double-float factorisation instantiation of the solver kernels for any number of
// quadrotors per problem (sizes read at run time).
#include "kernels.cuh"

namespace bipm {
void* iter_kernel_df() { return (void*)ipm_kernel<float, df, 0>; }
void* init_kernel_df() { return (void*)init_kernel<float, df, 0>; }
void* queue_kernel_df() { return (void*)queue_kernel<float, df, 0>; }
}  // namespace bipm
