// launch.h -- kernel tables of the pass kernels.  Each length has two tile
// widths compiled in: the "big" tile (256 or 512 threads) and a 2-line tile
// for lattices whose other extents are too small for the big one.
#pragma once

#include <stddef.h>

namespace hf {

constexpr int kRowLog2Min = 2, kRowLog2Max = 11;  // row FFT length M = n_last / 2
constexpr int kColLog2Min = 3, kColLog2Max = 12;  // strided-axis length

struct KernelInfo {
    const void* fn = nullptr;  // kernel entry point (nullptr: length outside the table)
    int threads = 0;           // threads per CTA
    int log2_lines = 0;        // log2 of rows (row kernels) or columns (column kernels) per tile
    size_t fixed_smem = 0;     // dynamic shared memory before any per-call tables
    bool map_bits_packed = false;  // c2r: packs one-bit map words itself (else ORs into cleared words)
};

// log2 lines per tile of each variant
constexpr int row_logtr(int log2m, bool big) { return big ? (log2m <= 4 ? 8 : 12 - log2m) : 0; }
constexpr int col_logtb(int log2l, bool big) {
    return big ? (log2l <= 4 ? 8 : (log2l >= 10 ? 13 - log2l : 12 - log2l)) : 1;
}

KernelInfo r2c_kernel(int log2m, bool big, int src);
// variant: the output type (C2ROut), plus 4 for a single sign-map level
KernelInfo c2r_kernel(int log2m, bool big, int variant);
// pair: the variant staged in the paired order of radial bins (binning modes
// on pairable tiles); rot: the filter and k-space modes' variant for a rotated
// norm (see k_cols)
KernelInfo cols_kernel(int log2l, bool big, int mode, int dir, bool pair = false, bool rot = false);

}  // namespace hf
