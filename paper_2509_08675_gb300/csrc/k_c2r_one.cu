// Row c2r kernels of a single field with a single sign-map level (FP32 or
// BF16 field).
#include "instantiate.cuh"

namespace hf {

KernelInfo c2r_kernel_one(int log2m, bool big, int out_dtype) {
    switch (out_dtype) {
        case kOutF32: return c2r_table<kOutF32, true>(log2m, big);
        case kOutBF16: return c2r_table<kOutBF16, true>(log2m, big);
        default: return {};
    }
}

}  // namespace hf
