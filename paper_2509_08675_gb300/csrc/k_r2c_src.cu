// Row r2c kernels reading a stored field (F32, BF16, I8).
#include "instantiate.cuh"

namespace hf {

KernelInfo r2c_kernel_src(int log2m, bool big, int src) {
    switch (log2m) {
        case 2:
            if (src == 1) return big ? r2c_info<2, 8, 1>() : r2c_info<2, 0, 1>();
            if (src == 2) return big ? r2c_info<2, 8, 2>() : r2c_info<2, 0, 2>();
            if (src == 3) return big ? r2c_info<2, 8, 3>() : r2c_info<2, 0, 3>();
            return {};
        case 3:
            if (src == 1) return big ? r2c_info<3, 8, 1>() : r2c_info<3, 0, 1>();
            if (src == 2) return big ? r2c_info<3, 8, 2>() : r2c_info<3, 0, 2>();
            if (src == 3) return big ? r2c_info<3, 8, 3>() : r2c_info<3, 0, 3>();
            return {};
        case 4:
            if (src == 1) return big ? r2c_info<4, 8, 1>() : r2c_info<4, 0, 1>();
            if (src == 2) return big ? r2c_info<4, 8, 2>() : r2c_info<4, 0, 2>();
            if (src == 3) return big ? r2c_info<4, 8, 3>() : r2c_info<4, 0, 3>();
            return {};
        case 5:
            if (src == 1) return big ? r2c_info<5, 7, 1>() : r2c_info<5, 0, 1>();
            if (src == 2) return big ? r2c_info<5, 7, 2>() : r2c_info<5, 0, 2>();
            if (src == 3) return big ? r2c_info<5, 7, 3>() : r2c_info<5, 0, 3>();
            return {};
        case 6:
            if (src == 1) return big ? r2c_info<6, 6, 1>() : r2c_info<6, 0, 1>();
            if (src == 2) return big ? r2c_info<6, 6, 2>() : r2c_info<6, 0, 2>();
            if (src == 3) return big ? r2c_info<6, 6, 3>() : r2c_info<6, 0, 3>();
            return {};
        case 7:
            if (src == 1) return big ? r2c_info<7, 5, 1>() : r2c_info<7, 0, 1>();
            if (src == 2) return big ? r2c_info<7, 5, 2>() : r2c_info<7, 0, 2>();
            if (src == 3) return big ? r2c_info<7, 5, 3>() : r2c_info<7, 0, 3>();
            return {};
        case 8:
            if (src == 1) return big ? r2c_info<8, 4, 1>() : r2c_info<8, 0, 1>();
            if (src == 2) return big ? r2c_info<8, 4, 2>() : r2c_info<8, 0, 2>();
            if (src == 3) return big ? r2c_info<8, 4, 3>() : r2c_info<8, 0, 3>();
            return {};
        case 9:
            if (src == 1) return big ? r2c_info<9, 3, 1>() : r2c_info<9, 0, 1>();
            if (src == 2) return big ? r2c_info<9, 3, 2>() : r2c_info<9, 0, 2>();
            if (src == 3) return big ? r2c_info<9, 3, 3>() : r2c_info<9, 0, 3>();
            return {};
        case 10:
            if (src == 1) return big ? r2c_info<10, 2, 1>() : r2c_info<10, 0, 1>();
            if (src == 2) return big ? r2c_info<10, 2, 2>() : r2c_info<10, 0, 2>();
            if (src == 3) return big ? r2c_info<10, 2, 3>() : r2c_info<10, 0, 3>();
            return {};
        case 11:
            if (src == 1) return big ? r2c_info<11, 1, 1>() : r2c_info<11, 0, 1>();
            if (src == 2) return big ? r2c_info<11, 1, 2>() : r2c_info<11, 0, 2>();
            if (src == 3) return big ? r2c_info<11, 1, 3>() : r2c_info<11, 0, 3>();
            return {};
        default: return {};
    }
}

}  // namespace hf
