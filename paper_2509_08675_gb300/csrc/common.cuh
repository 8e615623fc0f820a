// common.cuh -- complex arithmetic, counter-based noise (Philox4x32-10 +
// Box-Muller) and launch-argument structs shared by the sm_103a kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hf {

// Twiddle table: tw[q] = exp(-2 pi i q / 4096), q in [0, 4096), computed in
// FP64 once per plan and rounded to FP32.  Every power-of-two length L <= 4096
// reads W_L^m = tw[m * 4096 / L].
constexpr int kTwLog2 = 12;
constexpr int kTwN = 1 << kTwLog2;

constexpr int kMaxLevels = 8;
constexpr int kMaxTheta = 64;
constexpr int kMaxBins = 4096;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// a * w
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// a * conj(w)
__device__ __forceinline__ float2 cmulc(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}
// a * (DIR * i): DIR = -1 multiplies by -i (forward), +1 by +i (inverse)
template <int DIR>
__device__ __forceinline__ float2 cmul_i(float2 a) {
    return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies by the round multipliers; the high halves are mixed
// with words 1 and 3 and with the key, which is bumped by the Weyl constants
// between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Words of the noise block j of field (seed, field_idx).
__device__ __forceinline__ uint4 noise_block(uint64_t seed, uint32_t field_idx, uint64_t j) {
    return philox4x32_10(make_uint4((uint32_t)j, (uint32_t)(j >> 32), field_idx, 0u), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

// ln u for u = (x + 1/2) 2^-32.  Below 1/2 the FP32 value of u carries the
// full relative precision; above it the complement 1 - u = (~x + 1/2) 2^-32
// is exact in integers and log1pf keeps the small logarithm accurate.
__device__ __forceinline__ float log_uniform(uint32_t x) {
    if (x < 0x80000000u) {
        return logf(fmaf(__uint2float_rn(x), 0x1p-32f, 0x1p-33f));
    }
    const float d = fmaf(__uint2float_rn(~x), 0x1p-32f, 0x1p-33f);
    return log1pf(-d);
}

// (cos, sin)(2 pi u) for u = (x + 1/2) 2^-32: the quadrant comes from the top
// two bits (after centring), the remainder |y| <= 1/4 (units of pi) is
// formed exactly in integers before one rounding to FP32.
__device__ __forceinline__ float2 cis_uniform(uint32_t x) {
    const uint32_t xs = x + 0x20000000u;  // centre the quadrants
    const uint32_t q = xs >> 30;
    const int32_t rem = (int32_t)(xs & 0x3FFFFFFFu) - 0x20000000;  // [-2^29, 2^29)
    // angle = q pi/2 + 2 pi (rem + 1/2) / 2^32  ->  sincospi argument (2 rem + 1) 2^-32
    const float y = __int2float_rn(2 * rem + 1) * 0x1p-32f;
    float s, c;
    sincospif(y, &s, &c);
    switch (q) {
        case 0: return make_float2(c, s);
        case 1: return make_float2(-s, c);
        case 2: return make_float2(-c, -s);
        default: return make_float2(s, -c);
    }
}

// Box-Muller on one block: z0,z1 from (x0,x1), z2,z3 from (x2,x3).
__device__ __forceinline__ float4 box_muller(uint4 x) {
    const float r0 = sqrtf(-2.0f * log_uniform(x.x));
    const float2 a = cis_uniform(x.y);
    const float r1 = sqrtf(-2.0f * log_uniform(x.z));
    const float2 b = cis_uniform(x.w);
    return make_float4(r0 * a.x, r0 * a.y, r1 * b.x, r1 * b.y);
}

// ---------------------------------------------------------------------------
// Filter parameters (FP32, derived on the host from hufield_filter).
// ---------------------------------------------------------------------------
struct FilterParams {
    float inv_a[3];     // 1 / semi-axis
    float p, inv_p;     // superellipse exponent
    float cr, sr;       // cos, sin of the rotation
    int rotated;        // 0: no rotation, the norm is separable per axis
    float k0;           // band centre
    float kstar;        // analytic maximiser of K^s exp(-(K-k0)^2/(2w^2))
    float log2_kstar;
    float two_k0;
    float inv_2w2;      // 1 / (2 w^2)
    float half_s_ln2;   // s ln2 / 2   (H = exp(0.5 ln chi))
    float half;         // 0.5 (kept in the struct to keep FMAs uniform)
};

// Binning parameters; the angle table lives in shared memory at run time.
struct BinParams {
    int nr, ntheta, nbins;
    int shift[3];        // nmax / n[i] = 1 << shift[i]
    int log2nmax;
    long long ang_c[kMaxTheta];
    long long ang_s[kMaxTheta];
};

}  // namespace hf
