// Double-float factorisation instantiation of the block-team kernel.
#include "kernels.cuh"

namespace bipm {
void* block_kernel_df() { return (void*)ipm_block_kernel<float, df>; }
}  // namespace bipm
