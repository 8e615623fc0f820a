// Row r2c kernels with the noise source (fused Philox + Box-Muller), for one
// field (src 0) or for the fields of a batch (src 4, kSrcNoiseBatch).
#include "instantiate.cuh"

namespace hf {

KernelInfo r2c_kernel_noise(int log2m, bool big, int src) {
    switch (log2m) {
        case 2:
            if (src == 0) return big ? r2c_info<2, 8, 0>() : r2c_info<2, 0, 0>();
            if (src == 4) return big ? r2c_info<2, 8, 4>() : r2c_info<2, 0, 4>();
            return {};
        case 3:
            if (src == 0) return big ? r2c_info<3, 8, 0>() : r2c_info<3, 0, 0>();
            if (src == 4) return big ? r2c_info<3, 8, 4>() : r2c_info<3, 0, 4>();
            return {};
        case 4:
            if (src == 0) return big ? r2c_info<4, 8, 0>() : r2c_info<4, 0, 0>();
            if (src == 4) return big ? r2c_info<4, 8, 4>() : r2c_info<4, 0, 4>();
            return {};
        case 5:
            if (src == 0) return big ? r2c_info<5, 7, 0>() : r2c_info<5, 0, 0>();
            if (src == 4) return big ? r2c_info<5, 7, 4>() : r2c_info<5, 0, 4>();
            return {};
        case 6:
            if (src == 0) return big ? r2c_info<6, 6, 0>() : r2c_info<6, 0, 0>();
            if (src == 4) return big ? r2c_info<6, 6, 4>() : r2c_info<6, 0, 4>();
            return {};
        case 7:
            if (src == 0) return big ? r2c_info<7, 5, 0>() : r2c_info<7, 0, 0>();
            if (src == 4) return big ? r2c_info<7, 5, 4>() : r2c_info<7, 0, 4>();
            return {};
        case 8:
            if (src == 0) return big ? r2c_info<8, 4, 0>() : r2c_info<8, 0, 0>();
            if (src == 4) return big ? r2c_info<8, 4, 4>() : r2c_info<8, 0, 4>();
            return {};
        case 9:
            if (src == 0) return big ? r2c_info<9, 3, 0>() : r2c_info<9, 0, 0>();
            if (src == 4) return big ? r2c_info<9, 3, 4>() : r2c_info<9, 0, 4>();
            return {};
        case 10:
            if (src == 0) return big ? r2c_info<10, 2, 0>() : r2c_info<10, 0, 0>();
            if (src == 4) return big ? r2c_info<10, 2, 4>() : r2c_info<10, 0, 4>();
            return {};
        case 11:
            if (src == 0) return big ? r2c_info<11, 1, 0>() : r2c_info<11, 0, 0>();
            if (src == 4) return big ? r2c_info<11, 1, 4>() : r2c_info<11, 0, 4>();
            return {};
        default: return {};
    }
}

}  // namespace hf
