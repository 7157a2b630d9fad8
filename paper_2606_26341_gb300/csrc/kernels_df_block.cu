// Double-float factorisation instantiation of the block-team kernel (sizes read at run time).
#include "kernels.cuh"

namespace bipm {
void* block_kernel_df() { return (void*)ipm_block_kernel<float, df, 0>; }
}  // namespace bipm
