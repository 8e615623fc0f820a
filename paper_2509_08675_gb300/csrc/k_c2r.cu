// Row c2r kernels (normalise, sign maps, map r2c): FP32 or BF16 field, or
// the FP32 fields of a batch of fields (out_dtype 2, kOutBatch, one level per
// field).  variant = out_dtype, plus 4 for a single sign-map level (the
// kernels of k_c2r_one.cu).
#include "instantiate.cuh"

namespace hf {

KernelInfo c2r_kernel_one(int log2m, bool big, int out_dtype);

KernelInfo c2r_kernel(int log2m, bool big, int variant) {
    const int out_dtype = variant & 3;
    if (variant & 4) return c2r_kernel_one(log2m, big, out_dtype);
    switch (out_dtype) {
        case kOutF32: return c2r_table<kOutF32, false>(log2m, big);
        case kOutBF16: return c2r_table<kOutBF16, false>(log2m, big);
        case kOutBatch: return c2r_table<kOutBatch, true>(log2m, big);
        default: return {};
    }
}

}  // namespace hf
