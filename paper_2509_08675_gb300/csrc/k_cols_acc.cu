// Instantiations of the strided-axis kernel (acc modes).
#include "kernels.cuh"
#include "launch.h"

namespace hf {

template <int LOG2L>
static const void* pick(int mode, int dir) {
    (void)dir;
    if (mode == kModeFilter) return reinterpret_cast<const void*>(&k_cols<LOG2L, kModeFilter, -1>);
    if (mode == kModeBins) return reinterpret_cast<const void*>(&k_cols<LOG2L, kModeBins, -1>);
    return nullptr;
}

const void* cols_acc_kernel(int log2l, int mode, int dir) {
    switch (log2l) {
        case 3: return pick<3>(mode, dir);
        case 4: return pick<4>(mode, dir);
        case 5: return pick<5>(mode, dir);
        case 6: return pick<6>(mode, dir);
        case 7: return pick<7>(mode, dir);
        case 8: return pick<8>(mode, dir);
        case 9: return pick<9>(mode, dir);
        case 10: return pick<10>(mode, dir);
        case 11: return pick<11>(mode, dir);
        case 12: return pick<12>(mode, dir);
        default: return nullptr;
    }
}

}  // namespace hf
