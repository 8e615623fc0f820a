// Strided-axis kernels with the fused filter, Parseval sum and field bins,
// staged in the paired order of radial bins (n0 and -n0 in one thread):
// separable norm (no rotation).
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_filter_pair(int log2l, bool big) { return cols_pair_table<kModeFilter, 0>(log2l, big); }

}  // namespace hf
