// Strided-axis FFT kernels (forward and inverse).
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_plain(int log2l, bool big, int mode, int dir) {
    switch (log2l) {
        case 3:
            if (mode == 0 && dir == -1) return big ? cols_info<3, 8, 0, -1>() : cols_info<3, 1, 0, -1>();
            if (mode == 0 && dir == 1) return big ? cols_info<3, 8, 0, 1>() : cols_info<3, 1, 0, 1>();
            return {};
        case 4:
            if (mode == 0 && dir == -1) return big ? cols_info<4, 8, 0, -1>() : cols_info<4, 1, 0, -1>();
            if (mode == 0 && dir == 1) return big ? cols_info<4, 8, 0, 1>() : cols_info<4, 1, 0, 1>();
            return {};
        case 5:
            if (mode == 0 && dir == -1) return big ? cols_info<5, 7, 0, -1>() : cols_info<5, 1, 0, -1>();
            if (mode == 0 && dir == 1) return big ? cols_info<5, 7, 0, 1>() : cols_info<5, 1, 0, 1>();
            return {};
        case 6:
            if (mode == 0 && dir == -1) return big ? cols_info<6, 6, 0, -1>() : cols_info<6, 1, 0, -1>();
            if (mode == 0 && dir == 1) return big ? cols_info<6, 6, 0, 1>() : cols_info<6, 1, 0, 1>();
            return {};
        case 7:
            if (mode == 0 && dir == -1) return big ? cols_info<7, 5, 0, -1>() : cols_info<7, 1, 0, -1>();
            if (mode == 0 && dir == 1) return big ? cols_info<7, 5, 0, 1>() : cols_info<7, 1, 0, 1>();
            return {};
        case 8:
            if (mode == 0 && dir == -1) return big ? cols_info<8, 4, 0, -1>() : cols_info<8, 1, 0, -1>();
            if (mode == 0 && dir == 1) return big ? cols_info<8, 4, 0, 1>() : cols_info<8, 1, 0, 1>();
            return {};
        case 9:
            if (mode == 0 && dir == -1) return big ? cols_info<9, 3, 0, -1>() : cols_info<9, 1, 0, -1>();
            if (mode == 0 && dir == 1) return big ? cols_info<9, 3, 0, 1>() : cols_info<9, 1, 0, 1>();
            return {};
        case 10:
            if (mode == 0 && dir == -1) return big ? cols_info<10, 3, 0, -1>() : cols_info<10, 1, 0, -1>();
            if (mode == 0 && dir == 1) return big ? cols_info<10, 3, 0, 1>() : cols_info<10, 1, 0, 1>();
            return {};
        case 11:
            if (mode == 0 && dir == -1) return big ? cols_info<11, 2, 0, -1>() : cols_info<11, 1, 0, -1>();
            if (mode == 0 && dir == 1) return big ? cols_info<11, 2, 0, 1>() : cols_info<11, 1, 0, 1>();
            return {};
        case 12:
            if (mode == 0 && dir == -1) return big ? cols_info<12, 1, 0, -1>() : cols_info<12, 1, 0, -1>();
            if (mode == 0 && dir == 1) return big ? cols_info<12, 1, 0, 1>() : cols_info<12, 1, 0, 1>();
            return {};
        default: return {};
    }
}

}  // namespace hf
