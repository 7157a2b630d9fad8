// Double-float factorisation instantiation of the block-team kernel for one quadrotor per
// problem (sizes fixed at compile time).
#include "kernels.cuh"

namespace bipm {
void* block_kernel_df_q1() { return (void*)ipm_block_kernel<float, df, 1>; }
}  // namespace bipm
