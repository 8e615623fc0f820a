// Strided-axis kernels with the spectrum binning, staged in the
// paired order of radial bins (n0 and -n0 in one thread).
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_bins_pair(int log2l, bool big) { return cols_pair_table<kModeBins>(log2l, big); }

}  // namespace hf
