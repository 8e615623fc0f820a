// launch.h -- kernel tables of the pass kernels (one entry per length).
#pragma once

namespace hf {

constexpr int kRowLog2Min = 2, kRowLog2Max = 11;  // row FFT length M = n_last / 2
constexpr int kColLog2Min = 3, kColLog2Max = 12;  // strided-axis length

// Kernel entry points; nullptr when the length is outside the table.
const void* r2c_kernel(int log2m, int src);
const void* c2r_kernel(int log2m, int out_dtype);
const void* cols_kernel(int log2l, int mode, int dir);

// Elements per thread of each kernel family (threads = lines * length / E).
int row_elems(int log2m);
int col_elems(int log2l);

}  // namespace hf
