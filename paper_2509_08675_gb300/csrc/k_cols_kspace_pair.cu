// Strided-axis kernels with k-space noise, the fused filter, Parseval sum and
// field bins, staged in the paired order of radial bins (n0 and -n0 in one
// thread): separable norm (no rotation).
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_kspace_pair(int log2l, bool big) { return cols_pair_table<kModeKspace, 0>(log2l, big); }

}  // namespace hf
