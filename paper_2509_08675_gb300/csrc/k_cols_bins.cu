// Strided-axis kernels with the spectrum binning.
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_bins(int log2l, bool big, int mode, int dir) {
    if (mode != kModeBins || dir != -1) return {};
    return cols_table<kModeBins, -1>(log2l, big);
}

}  // namespace hf
