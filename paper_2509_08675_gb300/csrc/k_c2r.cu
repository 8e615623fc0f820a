// Instantiations of the row c2r (normalise, threshold, map r2c) kernel.
#include "kernels.cuh"
#include "launch.h"

namespace hf {

template <int LOG2M>
static const void* c2r_for(int out_dtype) {
    return out_dtype == 0 ? reinterpret_cast<const void*>(&k_c2r<LOG2M, 0>)
                          : reinterpret_cast<const void*>(&k_c2r<LOG2M, 1>);
}

const void* c2r_kernel(int log2m, int out_dtype) {
    if (out_dtype != 0 && out_dtype != 1) return nullptr;
    switch (log2m) {
        case 2: return c2r_for<2>(out_dtype);
        case 3: return c2r_for<3>(out_dtype);
        case 4: return c2r_for<4>(out_dtype);
        case 5: return c2r_for<5>(out_dtype);
        case 6: return c2r_for<6>(out_dtype);
        case 7: return c2r_for<7>(out_dtype);
        case 8: return c2r_for<8>(out_dtype);
        case 9: return c2r_for<9>(out_dtype);
        case 10: return c2r_for<10>(out_dtype);
        case 11: return c2r_for<11>(out_dtype);
        default: return nullptr;
    }
}

}  // namespace hf
