// Instantiations of the row r2c kernel for every row length and input source.
#include "kernels.cuh"
#include "launch.h"

namespace hf {

template <int LOG2M>
static const void* r2c_for_src(int src) {
    switch (src) {
        case kSrcNoise: return reinterpret_cast<const void*>(&k_r2c<LOG2M, kSrcNoise>);
        case kSrcF32: return reinterpret_cast<const void*>(&k_r2c<LOG2M, kSrcF32>);
        case kSrcBF16: return reinterpret_cast<const void*>(&k_r2c<LOG2M, kSrcBF16>);
        case kSrcI8: return reinterpret_cast<const void*>(&k_r2c<LOG2M, kSrcI8>);
        default: return nullptr;
    }
}

const void* r2c_kernel(int log2m, int src) {
    switch (log2m) {
        case 2: return r2c_for_src<2>(src);
        case 3: return r2c_for_src<3>(src);
        case 4: return r2c_for_src<4>(src);
        case 5: return r2c_for_src<5>(src);
        case 6: return r2c_for_src<6>(src);
        case 7: return r2c_for_src<7>(src);
        case 8: return r2c_for_src<8>(src);
        case 9: return r2c_for_src<9>(src);
        case 10: return r2c_for_src<10>(src);
        case 11: return r2c_for_src<11>(src);
        default: return nullptr;
    }
}

int row_elems(int log2m) { return log2m >= 4 ? 16 : (1 << log2m); }

}  // namespace hf
