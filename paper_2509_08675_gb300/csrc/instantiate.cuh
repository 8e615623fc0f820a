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

template <int LOG2M, int LOGTR, int OUTDT>
KernelInfo c2r_info() {
    using G = Geo<LOG2M, LOGTR, true>;
    return {reinterpret_cast<const void*>(&k_c2r<LOG2M, LOGTR, OUTDT>), G::T, LOGTR,
            (size_t)2 * G::TB * G::L * 8 + (size_t)G::L * 8 + (size_t)plan_twiddle_slots<LOG2M>() * 8 + 16,
            map_bits_packed(LOG2M, LOGTR, OUTDT == kOutBatch)};
}

template <int LOG2L, int LOGTB, int MODE, int DIR>
KernelInfo cols_info() {
    using CG = ColGeo<LOG2L, LOGTB, MODE>;
    return {reinterpret_cast<const void*>(&k_cols<LOG2L, LOGTB, MODE, DIR>), CG::G::T, LOGTB, CG::fixed_bytes};
}

}  // namespace hf

// Switch over a log2 length from LO to HI calling F<n>(args...).
#define HF_CASE(F, n, ...) \
    case n: return F<n>(__VA_ARGS__);
