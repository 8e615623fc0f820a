// Strided-axis kernels with the fused filter, Parseval sum and field bins.
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_filter(int log2l, bool big, int mode, int dir) {
    switch (log2l) {
        case 3:
            if (mode == 1 && dir == -1) return big ? cols_info<3, 8, 1, -1>() : cols_info<3, 1, 1, -1>();
            return {};
        case 4:
            if (mode == 1 && dir == -1) return big ? cols_info<4, 8, 1, -1>() : cols_info<4, 1, 1, -1>();
            return {};
        case 5:
            if (mode == 1 && dir == -1) return big ? cols_info<5, 7, 1, -1>() : cols_info<5, 1, 1, -1>();
            return {};
        case 6:
            if (mode == 1 && dir == -1) return big ? cols_info<6, 6, 1, -1>() : cols_info<6, 1, 1, -1>();
            return {};
        case 7:
            if (mode == 1 && dir == -1) return big ? cols_info<7, 5, 1, -1>() : cols_info<7, 1, 1, -1>();
            return {};
        case 8:
            if (mode == 1 && dir == -1) return big ? cols_info<8, 4, 1, -1>() : cols_info<8, 1, 1, -1>();
            return {};
        case 9:
            if (mode == 1 && dir == -1) return big ? cols_info<9, 3, 1, -1>() : cols_info<9, 1, 1, -1>();
            return {};
        case 10:
            if (mode == 1 && dir == -1) return big ? cols_info<10, 3, 1, -1>() : cols_info<10, 1, 1, -1>();
            return {};
        case 11:
            if (mode == 1 && dir == -1) return big ? cols_info<11, 2, 1, -1>() : cols_info<11, 1, 1, -1>();
            return {};
        case 12:
            if (mode == 1 && dir == -1) return big ? cols_info<12, 1, 1, -1>() : cols_info<12, 1, 1, -1>();
            return {};
        default: return {};
    }
}

}  // namespace hf
