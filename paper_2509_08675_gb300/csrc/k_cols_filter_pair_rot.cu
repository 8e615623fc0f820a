// Strided-axis kernels with the fused filter, Parseval sum and field bins,
// staged in the paired order of radial bins (n0 and -n0 in one thread):
// rotated norm.
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_filter_pair_rot(int log2l, bool big) { return cols_pair_table<kModeFilter, 1>(log2l, big); }

}  // namespace hf
