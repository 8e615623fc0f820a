// Strided-axis kernels with the fused filter, Parseval sum and field bins, for
// batches of fields that each carry their own filter (kModeFilterBatch).
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_filter_batch(int log2l, bool big, int mode, int dir) {
    if (mode != kModeFilterBatch || dir != -1) return {};
    return cols_table<kModeFilterBatch, -1>(log2l, big);
}

}  // namespace hf
