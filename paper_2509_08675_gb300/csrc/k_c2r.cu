// Row c2r kernels (normalise, sign maps, map r2c): FP32 or BF16 field, or
// the FP32 fields of a batch of fields (out_dtype 2, kOutBatch).
#include "instantiate.cuh"

namespace hf {

KernelInfo c2r_kernel(int log2m, bool big, int out_dtype) {
    switch (log2m) {
        case 2:
            if (out_dtype == 0) return big ? c2r_info<2, 8, 0>() : c2r_info<2, 0, 0>();
            if (out_dtype == 1) return big ? c2r_info<2, 8, 1>() : c2r_info<2, 0, 1>();
            if (out_dtype == 2) return big ? c2r_info<2, 8, 2>() : c2r_info<2, 0, 2>();
            return {};
        case 3:
            if (out_dtype == 0) return big ? c2r_info<3, 8, 0>() : c2r_info<3, 0, 0>();
            if (out_dtype == 1) return big ? c2r_info<3, 8, 1>() : c2r_info<3, 0, 1>();
            if (out_dtype == 2) return big ? c2r_info<3, 8, 2>() : c2r_info<3, 0, 2>();
            return {};
        case 4:
            if (out_dtype == 0) return big ? c2r_info<4, 8, 0>() : c2r_info<4, 0, 0>();
            if (out_dtype == 1) return big ? c2r_info<4, 8, 1>() : c2r_info<4, 0, 1>();
            if (out_dtype == 2) return big ? c2r_info<4, 8, 2>() : c2r_info<4, 0, 2>();
            return {};
        case 5:
            if (out_dtype == 0) return big ? c2r_info<5, 7, 0>() : c2r_info<5, 0, 0>();
            if (out_dtype == 1) return big ? c2r_info<5, 7, 1>() : c2r_info<5, 0, 1>();
            if (out_dtype == 2) return big ? c2r_info<5, 7, 2>() : c2r_info<5, 0, 2>();
            return {};
        case 6:
            if (out_dtype == 0) return big ? c2r_info<6, 6, 0>() : c2r_info<6, 0, 0>();
            if (out_dtype == 1) return big ? c2r_info<6, 6, 1>() : c2r_info<6, 0, 1>();
            if (out_dtype == 2) return big ? c2r_info<6, 6, 2>() : c2r_info<6, 0, 2>();
            return {};
        case 7:
            if (out_dtype == 0) return big ? c2r_info<7, 5, 0>() : c2r_info<7, 0, 0>();
            if (out_dtype == 1) return big ? c2r_info<7, 5, 1>() : c2r_info<7, 0, 1>();
            if (out_dtype == 2) return big ? c2r_info<7, 5, 2>() : c2r_info<7, 0, 2>();
            return {};
        case 8:
            if (out_dtype == 0) return big ? c2r_info<8, 4, 0>() : c2r_info<8, 0, 0>();
            if (out_dtype == 1) return big ? c2r_info<8, 4, 1>() : c2r_info<8, 0, 1>();
            if (out_dtype == 2) return big ? c2r_info<8, 4, 2>() : c2r_info<8, 0, 2>();
            return {};
        case 9:
            if (out_dtype == 0) return big ? c2r_info<9, 3, 0>() : c2r_info<9, 0, 0>();
            if (out_dtype == 1) return big ? c2r_info<9, 3, 1>() : c2r_info<9, 0, 1>();
            if (out_dtype == 2) return big ? c2r_info<9, 3, 2>() : c2r_info<9, 0, 2>();
            return {};
        case 10:
            if (out_dtype == 0) return big ? c2r_info<10, 2, 0>() : c2r_info<10, 0, 0>();
            if (out_dtype == 1) return big ? c2r_info<10, 2, 1>() : c2r_info<10, 0, 1>();
            if (out_dtype == 2) return big ? c2r_info<10, 2, 2>() : c2r_info<10, 0, 2>();
            return {};
        case 11:
            if (out_dtype == 0) return big ? c2r_info<11, 1, 0>() : c2r_info<11, 0, 0>();
            if (out_dtype == 1) return big ? c2r_info<11, 1, 1>() : c2r_info<11, 0, 1>();
            if (out_dtype == 2) return big ? c2r_info<11, 1, 2>() : c2r_info<11, 0, 2>();
            return {};
        default: return {};
    }
}

}  // namespace hf
