// Strided-axis kernels with the fused filter, Parseval sum and field bins, for
// batches of fields that each carry their own filter (kModeFilterBatch).
#include "instantiate.cuh"

namespace hf {

KernelInfo cols_kernel_filter_batch(int log2l, bool big, int mode, int dir) {
    switch (log2l) {
        case 3:
            if (mode == 4 && dir == -1) return big ? cols_info<3, 8, 4, -1>() : cols_info<3, 1, 4, -1>();
            return {};
        case 4:
            if (mode == 4 && dir == -1) return big ? cols_info<4, 8, 4, -1>() : cols_info<4, 1, 4, -1>();
            return {};
        case 5:
            if (mode == 4 && dir == -1) return big ? cols_info<5, 7, 4, -1>() : cols_info<5, 1, 4, -1>();
            return {};
        case 6:
            if (mode == 4 && dir == -1) return big ? cols_info<6, 6, 4, -1>() : cols_info<6, 1, 4, -1>();
            return {};
        case 7:
            if (mode == 4 && dir == -1) return big ? cols_info<7, 5, 4, -1>() : cols_info<7, 1, 4, -1>();
            return {};
        case 8:
            if (mode == 4 && dir == -1) return big ? cols_info<8, 4, 4, -1>() : cols_info<8, 1, 4, -1>();
            return {};
        case 9:
            if (mode == 4 && dir == -1) return big ? cols_info<9, 3, 4, -1>() : cols_info<9, 1, 4, -1>();
            return {};
        case 10:
            if (mode == 4 && dir == -1) return big ? cols_info<10, 3, 4, -1>() : cols_info<10, 1, 4, -1>();
            return {};
        case 11:
            if (mode == 4 && dir == -1) return big ? cols_info<11, 2, 4, -1>() : cols_info<11, 1, 4, -1>();
            return {};
        case 12:
            if (mode == 4 && dir == -1) return big ? cols_info<12, 1, 4, -1>() : cols_info<12, 1, 4, -1>();
            return {};
        default: return {};
    }
}

}  // namespace hf
