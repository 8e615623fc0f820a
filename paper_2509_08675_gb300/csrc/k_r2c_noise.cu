// Row r2c kernels with the noise source (fused Philox + Box-Muller).
#include "instantiate.cuh"

namespace hf {

KernelInfo r2c_kernel_noise(int log2m, bool big, int src) {
    switch (log2m) {
        case 2:
            if (src == 0) return big ? r2c_info<2, 8, 0>() : r2c_info<2, 0, 0>();
            return {};
        case 3:
            if (src == 0) return big ? r2c_info<3, 8, 0>() : r2c_info<3, 0, 0>();
            return {};
        case 4:
            if (src == 0) return big ? r2c_info<4, 8, 0>() : r2c_info<4, 0, 0>();
            return {};
        case 5:
            if (src == 0) return big ? r2c_info<5, 7, 0>() : r2c_info<5, 0, 0>();
            return {};
        case 6:
            if (src == 0) return big ? r2c_info<6, 6, 0>() : r2c_info<6, 0, 0>();
            return {};
        case 7:
            if (src == 0) return big ? r2c_info<7, 5, 0>() : r2c_info<7, 0, 0>();
            return {};
        case 8:
            if (src == 0) return big ? r2c_info<8, 4, 0>() : r2c_info<8, 0, 0>();
            return {};
        case 9:
            if (src == 0) return big ? r2c_info<9, 3, 0>() : r2c_info<9, 0, 0>();
            return {};
        case 10:
            if (src == 0) return big ? r2c_info<10, 2, 0>() : r2c_info<10, 0, 0>();
            return {};
        case 11:
            if (src == 0) return big ? r2c_info<11, 1, 0>() : r2c_info<11, 0, 0>();
            return {};
        default: return {};
    }
}

}  // namespace hf
