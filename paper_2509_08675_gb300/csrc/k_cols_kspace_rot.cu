// Strided-axis kernels that draw k-space noise and apply the fused filter,
// Parseval sum and field bins: rotated norm.
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_kspace_rot(int log2l, bool big, int mode, int dir) {
    if (mode != kModeKspace || dir != -1) return {};
    return cols_table<kModeKspace, -1, 1>(log2l, big);
}

}  // namespace hf
