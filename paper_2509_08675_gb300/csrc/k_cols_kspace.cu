// Strided-axis kernels that draw k-space noise and apply the fused filter,
// Parseval sum and field bins.
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_kspace(int log2l, bool big, int mode, int dir) {
    switch (log2l) {
        case 3:
            if (mode == 3 && dir == -1) return big ? cols_info<3, 8, 3, -1>() : cols_info<3, 1, 3, -1>();
            return {};
        case 4:
            if (mode == 3 && dir == -1) return big ? cols_info<4, 8, 3, -1>() : cols_info<4, 1, 3, -1>();
            return {};
        case 5:
            if (mode == 3 && dir == -1) return big ? cols_info<5, 7, 3, -1>() : cols_info<5, 1, 3, -1>();
            return {};
        case 6:
            if (mode == 3 && dir == -1) return big ? cols_info<6, 6, 3, -1>() : cols_info<6, 1, 3, -1>();
            return {};
        case 7:
            if (mode == 3 && dir == -1) return big ? cols_info<7, 5, 3, -1>() : cols_info<7, 1, 3, -1>();
            return {};
        case 8:
            if (mode == 3 && dir == -1) return big ? cols_info<8, 4, 3, -1>() : cols_info<8, 1, 3, -1>();
            return {};
        case 9:
            if (mode == 3 && dir == -1) return big ? cols_info<9, 3, 3, -1>() : cols_info<9, 1, 3, -1>();
            return {};
        case 10:
            if (mode == 3 && dir == -1) return big ? cols_info<10, 3, 3, -1>() : cols_info<10, 1, 3, -1>();
            return {};
        case 11:
            if (mode == 3 && dir == -1) return big ? cols_info<11, 2, 3, -1>() : cols_info<11, 1, 3, -1>();
            return {};
        case 12:
            if (mode == 3 && dir == -1) return big ? cols_info<12, 1, 3, -1>() : cols_info<12, 1, 3, -1>();
            return {};
        default: return {};
    }
}

}  // namespace hf
