// Strided-axis kernels with the fused filter, Parseval sum and field bins:
// separable norm (no rotation).
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_filter(int log2l, bool big, int mode, int dir) {
    if (mode != kModeFilter || dir != -1) return {};
    return cols_table<kModeFilter, -1, 0>(log2l, big);
}

}  // namespace hf
