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

// The same ten rounds with the round keys given: keys[2r], keys[2r + 1] =
// (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85).  A launch whose threads share one
// key passes them as kernel parameters, read as operands of the XORs, instead
// of bumping the key in every thread.
__device__ __forceinline__ uint4 philox4x32_10_keyed(uint4 c, const uint32_t (&keys)[20]) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ keys[2 * round], lo1, hi0 ^ c.w ^ keys[2 * round + 1], lo0);
    }
    return c;
}

// Words of the noise block j of field (seed, field_idx).
__device__ __forceinline__ uint4 noise_block(uint64_t seed, uint32_t field_idx, uint64_t j) {
    return philox4x32_10(make_uint4((uint32_t)j, (uint32_t)(j >> 32), field_idx, 0u), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

// Hardware approximations (PTX): base-2 logarithm (absolute error about
// 2^-22 for arguments in [1/2, 2)) and square root (relative error about
// 2^-23).
__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Box-Muller radius sqrt(-2 ln u) for u = (x + 1/2) 2^-32.  Near u = 1 the
// complement d = 1 - u = (~x + 1/2) 2^-32 is exact, and for d < 1/16
// -ln u = -ln(1 - d) = d + d^2/2 + ... + d^7/7 (Taylor series; the rest is
// below 5e-10 of the sum), so the radius keeps full relative precision where
// it is small.  Elsewhere |log2 u| >= 0.093 and -ln u = -ln2 log2 u with the
// hardware log2: its absolute error of ~2^-22 is at most 2.6e-6 of -ln u,
// 1.3e-6 of the radius (~5e-7 absolute at d = 1/16, less beyond).  Both
// branches are evaluated and one is selected (no divergence).
__device__ __forceinline__ float bm_radius(uint32_t x) {
    const float u = fmaf(__uint2float_rn(x), 0x1p-32f, 0x1p-33f);
    const float d = fmaf(__uint2float_rn(~x), 0x1p-32f, 0x1p-33f);
    const float far = -0.693147180559945309f * lg2_approx(u);
    const float near = fmaf(d * d,
                            fmaf(d, fmaf(d, fmaf(d, fmaf(d, fmaf(d, 1.0f / 7.0f, 1.0f / 6.0f), 0.2f), 0.25f),
                                         1.0f / 3.0f),
                                 0.5f),
                            d);
    return sqrt_approx(2.0f * (d < 0.0625f ? near : far));
}

// (cos, sin)(2 pi u) for u = (x + 1/2) 2^-32: the quadrant comes from the top
// two bits (after centring) and the remainder y = (2 rem + 1) 2^-32, |y| <= 1/4
// (angle pi y), is formed exactly in integers before one rounding to FP32.
// sin(pi y) and cos(pi y) are their Taylor series in pi y up to the y^9 and
// y^10 terms (truncation below 2e-9 on |y| <= 1/4), evaluated by Horner.  The
// quadrant swaps the pair (odd quadrants) and flips signs (cos negative in
// quadrants 1 and 2, sin in 2 and 3) without branches.
__device__ __forceinline__ float2 cis_uniform(uint32_t x) {
    const uint32_t xs = x + 0x20000000u;  // centre the quadrants
    const uint32_t q = xs >> 30;
    const int32_t rem = (int32_t)(xs & 0x3FFFFFFFu) - 0x20000000;  // [-2^29, 2^29)
    const float y = __int2float_rn(2 * rem + 1) * 0x1p-32f;
    const float y2 = y * y;
    // pi, -pi^3/3!, pi^5/5!, -pi^7/7!, pi^9/9!
    const float sp = y * fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, 0.0821458866111282287f, -0.599264529320792077f),
                                                 2.55016403987734544f),
                                      -5.16771278004997003f),
                              3.14159265358979324f);
    // 1, -pi^2/2!, pi^4/4!, -pi^6/6!, pi^8/8!, -pi^10/10!
    const float cp = fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, fmaf(y2, -0.0258068913900140600f, 0.235330630358893204f),
                                                     -1.33526276885458949f),
                                          4.05871212641676822f),
                               -4.93480220054467931f),
                          1.0f);
    const bool odd = (q & 1u) != 0u;
    const float c = odd ? sp : cp, s = odd ? cp : sp;
    const uint32_t cneg = ((q + 1u) >> 1) & 1u, sneg = q >> 1;
    return make_float2(__uint_as_float(__float_as_uint(c) ^ (cneg << 31)),
                       __uint_as_float(__float_as_uint(s) ^ (sneg << 31)));
}

// Box-Muller on one block: z0,z1 from (x0,x1), z2,z3 from (x2,x3).
__device__ __forceinline__ float4 box_muller(uint4 x) {
    const float r0 = bm_radius(x.x);
    const float2 a = cis_uniform(x.y);
    const float r1 = bm_radius(x.z);
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
    float half_s;       // s / 2                 H = 2^(s/2 (log2 K - log2 K*) - c d),
    float c_d;          // log2(e) / (4 w^2)     d = (K - k0)^2 - (K* - k0)^2
    float u_zero;       // p log2 K from which the exponent is below -140: H flushes to 0 exactly
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
