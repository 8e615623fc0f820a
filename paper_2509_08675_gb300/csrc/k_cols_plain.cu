// Strided-axis FFT kernels (forward and inverse).
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_plain(int log2l, bool big, int mode, int dir) {
    if (mode != kModePlain) return {};
    if (dir == -1) return cols_table<kModePlain, -1>(log2l, big);
    if (dir == 1) return cols_table<kModePlain, 1>(log2l, big);
    return {};
}

}  // namespace hf
