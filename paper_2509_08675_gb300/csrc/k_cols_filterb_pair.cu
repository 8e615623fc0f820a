// Strided-axis kernels with per-field filters of a batch, Parseval sums and
// field bins, staged in the paired order of radial bins (n0 and -n0 in one
// thread).
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_filter_batch_pair(int log2l, bool big) { return cols_pair_table<kModeFilterBatch>(log2l, big); }

}  // namespace hf
