// instantiate.cuh -- helpers that turn a compile-time kernel choice into a
// KernelInfo (entry point, threads, tile width, fixed shared memory).
#pragma once

#include "kernels.cuh"
#include "launch.h"

namespace hf {

template <int LOG2M, int LOGTR, int SRC>
KernelInfo r2c_info() {
    using G = Geo<LOG2M, LOGTR, true>;
    return {reinterpret_cast<const void*>(&k_r2c<LOG2M, LOGTR, SRC>), G::T, LOGTR,
            (size_t)G::TB * G::L * 8 + (size_t)G::L * 8 + (size_t)TwTables<LOG2M, false>::size() * 8};
}

template <int LOG2M, int LOGTR, int OUTDT, bool ONE>
KernelInfo c2r_info() {
    using G = Geo<LOG2M, LOGTR, true>;
    return {reinterpret_cast<const void*>(&k_c2r<LOG2M, LOGTR, OUTDT, ONE>), G::T, LOGTR,
            (size_t)2 * G::TB * G::L * 8 + (size_t)G::L * 8 + (size_t)plan_twiddle_slots<LOG2M>() * 8 + 16,
            map_bits_packed(LOG2M, LOGTR, OUTDT == kOutBatch)};
}

template <int LOG2L, int LOGTB, int MODE, int DIR, bool PAIR = false, int ROT = 2>
KernelInfo cols_info() {
    using CG = ColGeo<LOG2L, LOGTB, MODE>;
    return {reinterpret_cast<const void*>(&k_cols<LOG2L, LOGTB, MODE, DIR, PAIR, ROT>), CG::G::T, LOGTB,
            CG::fixed_bytes};
}

// Every row length's wide and one-row tiles of the c2r kernel for one output
// type and level count (ONE: a single sign-map level).
template <int OUTDT, bool ONE>
KernelInfo c2r_table(int log2m, bool big) {
    switch (log2m) {
        case 2: return big ? c2r_info<2, 8, OUTDT, ONE>() : c2r_info<2, 0, OUTDT, ONE>();
        case 3: return big ? c2r_info<3, 8, OUTDT, ONE>() : c2r_info<3, 0, OUTDT, ONE>();
        case 4: return big ? c2r_info<4, 8, OUTDT, ONE>() : c2r_info<4, 0, OUTDT, ONE>();
        case 5: return big ? c2r_info<5, 7, OUTDT, ONE>() : c2r_info<5, 0, OUTDT, ONE>();
        case 6: return big ? c2r_info<6, 6, OUTDT, ONE>() : c2r_info<6, 0, OUTDT, ONE>();
        case 7: return big ? c2r_info<7, 5, OUTDT, ONE>() : c2r_info<7, 0, OUTDT, ONE>();
        case 8: return big ? c2r_info<8, 4, OUTDT, ONE>() : c2r_info<8, 0, OUTDT, ONE>();
        case 9: return big ? c2r_info<9, 3, OUTDT, ONE>() : c2r_info<9, 0, OUTDT, ONE>();
        case 10: return big ? c2r_info<10, 2, OUTDT, ONE>() : c2r_info<10, 0, OUTDT, ONE>();
        case 11: return big ? c2r_info<11, 1, OUTDT, ONE>() : c2r_info<11, 0, OUTDT, ONE>();
        default: return {};
    }
}

// Every length's wide and two-column tiles of one mode, direction and norm
// (the plain staging order).  The wide tile's columns: 256 up to L = 16,
// 4096 / L from 32 to 512, 8192 / L from 1024 (col_logtb).
template <int MODE, int DIR, int ROT = 2>
KernelInfo cols_table(int log2l, bool big) {
    switch (log2l) {
        case 3: return big ? cols_info<3, 8, MODE, DIR, false, ROT>() : cols_info<3, 1, MODE, DIR, false, ROT>();
        case 4: return big ? cols_info<4, 8, MODE, DIR, false, ROT>() : cols_info<4, 1, MODE, DIR, false, ROT>();
        case 5: return big ? cols_info<5, 7, MODE, DIR, false, ROT>() : cols_info<5, 1, MODE, DIR, false, ROT>();
        case 6: return big ? cols_info<6, 6, MODE, DIR, false, ROT>() : cols_info<6, 1, MODE, DIR, false, ROT>();
        case 7: return big ? cols_info<7, 5, MODE, DIR, false, ROT>() : cols_info<7, 1, MODE, DIR, false, ROT>();
        case 8: return big ? cols_info<8, 4, MODE, DIR, false, ROT>() : cols_info<8, 1, MODE, DIR, false, ROT>();
        case 9: return big ? cols_info<9, 3, MODE, DIR, false, ROT>() : cols_info<9, 1, MODE, DIR, false, ROT>();
        case 10: return big ? cols_info<10, 3, MODE, DIR, false, ROT>() : cols_info<10, 1, MODE, DIR, false, ROT>();
        case 11: return big ? cols_info<11, 2, MODE, DIR, false, ROT>() : cols_info<11, 1, MODE, DIR, false, ROT>();
        case 12: return cols_info<12, 1, MODE, DIR, false, ROT>();
        default: return {};
    }
}

// The paired-staging variants (PAIR = true) of a binning mode on every
// pairable tile: 16 values per thread and at most 256 threads, i.e. lengths
// 16 to 512 in the wide tile and 16 to 2048 in the two-column one.
template <int MODE, int ROT = 2>
KernelInfo cols_pair_table(int log2l, bool big) {
    switch (log2l) {
        case 4: return big ? cols_info<4, 8, MODE, -1, true, ROT>() : cols_info<4, 1, MODE, -1, true, ROT>();
        case 5: return big ? cols_info<5, 7, MODE, -1, true, ROT>() : cols_info<5, 1, MODE, -1, true, ROT>();
        case 6: return big ? cols_info<6, 6, MODE, -1, true, ROT>() : cols_info<6, 1, MODE, -1, true, ROT>();
        case 7: return big ? cols_info<7, 5, MODE, -1, true, ROT>() : cols_info<7, 1, MODE, -1, true, ROT>();
        case 8: return big ? cols_info<8, 4, MODE, -1, true, ROT>() : cols_info<8, 1, MODE, -1, true, ROT>();
        case 9: return big ? cols_info<9, 3, MODE, -1, true, ROT>() : cols_info<9, 1, MODE, -1, true, ROT>();
        case 10: return big ? KernelInfo{} : cols_info<10, 1, MODE, -1, true, ROT>();
        case 11: return big ? KernelInfo{} : cols_info<11, 1, MODE, -1, true, ROT>();
        default: return {};
    }
}

}  // namespace hf

// Switch over a log2 length from LO to HI calling F<n>(args...).
#define HF_CASE(F, n, ...) \
    case n: return F<n>(__VA_ARGS__);
