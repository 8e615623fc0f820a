// window.cuh -- window variance sigma_F^2(R), Eq. (1) of Sec. II.A, from the
// spectrum: the variance of the field averaged over a ball of radius R is
//   sigma_F^2(R) = (1/N^2) sum_{n != 0} |Y(n)|^2 m(|k_n| R)^2,
// m the transform of the ball's indicator over its volume (2 J1(x)/x in 2D,
// 3 (sin x - x cos x)/x^3 in 3D), k_n with components 2 pi n_d / N_d, n_d
// signed, lengths in lattice spacings.  A diagnostic off the generator's path:
// FP64 throughout the window terms.
#pragma once

#include <cuda_bf16.h>

#include "kernels.cuh"

namespace hf {

constexpr int kMaxRadii = 64;

struct WindowArgs {
    int ndim;
    int log2n[3];
    int logM;                 // log2 (n_last / 2)
    long long half;           // N / 2 stored half-spectrum modes (k_last < n_last / 2)
    int nradii;
    float radii[kMaxRadii];
    const float2* spec;       // field variant: half spectrum [n0][n1][k_last]
    const double2* plane;     // field variant: Nyquist plane k_last = n_last / 2, [n0][n1] (3D) or [n0] (2D)
    FilterParams fp;          // filter variant
    double* acc;              // nradii sums, then (filter variant) the sum of A^2
};

__device__ __forceinline__ double ball_transform(int ndim, double x) {
    if (x == 0.0) return 1.0;
    if (ndim == 2) return 2.0 * j1(x) / x;
    if (x < 1e-2) return 1.0 - x * x / 10.0 + x * x * x * x / 280.0;
    double s, c;
    sincos(x, &s, &c);
    return 3.0 * (s - x * c) / (x * x * x);
}

// |k| of the mode with signed indices (i0, i1, i2) (unused axes 0)
__device__ __forceinline__ double mode_k(const WindowArgs& a, int i0, int i1, int i2) {
    const double k0 = 6.283185307179586 * (double)i0 / (double)(1 << a.log2n[0]);
    double k2 = k0 * k0;
    const double k1 = 6.283185307179586 * (double)i1 / (double)(1 << a.log2n[1]);
    k2 += k1 * k1;
    if (a.ndim == 3) {
        const double kk = 6.283185307179586 * (double)i2 / (double)(1 << a.log2n[2]);
        k2 += kk * kk;
    }
    return sqrt(k2);
}

// Signed indices of stored half-spectrum mode m (natural layout) and its weight
// in the full-lattice sum (1 at k_last = 0, 2 elsewhere: k and -k).
__device__ __forceinline__ void half_mode(const WindowArgs& a, long long m, int& i0, int& i1, int& i2, double& w) {
    const int M = 1 << a.logM;
    const int kl = (int)(m & (M - 1));
    const long long row = m >> a.logM;
    if (a.ndim == 3) {
        i1 = signed_index((int)(row & ((1 << a.log2n[1]) - 1)), a.log2n[1]);
        i0 = signed_index((int)(row >> a.log2n[1]), a.log2n[0]);
        i2 = kl;
    } else {
        i0 = signed_index((int)row, a.log2n[0]);
        i1 = kl;
        i2 = 0;
    }
    w = kl == 0 ? 1.0 : 2.0;
}

__device__ __forceinline__ void block_add(double v, double* dst) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double part[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0) atomicAdd(dst, v);
    }
}

// Field variant, stored modes: blockIdx.y = radius, grid-stride over modes.
__global__ void k_window_field(const __grid_constant__ WindowArgs a) {
    const int r = blockIdx.y;
    const double R = (double)a.radii[r];
    double sum = 0.0;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < a.half;
         m += (long long)gridDim.x * blockDim.x) {
        if (m == 0) continue;  // n = 0
        int i0, i1, i2;
        double w;
        half_mode(a, m, i0, i1, i2, w);
        const float2 y = a.spec[m];
        const double p2 = (double)y.x * y.x + (double)y.y * y.y;
        const double mt = ball_transform(a.ndim, mode_k(a, i0, i1, i2) * R);
        sum += w * p2 * mt * mt;
    }
    block_add(sum, a.acc + r);
}

// Field variant, the Nyquist plane k_last = -n_last / 2 (each mode once).
__global__ void k_window_plane(const __grid_constant__ WindowArgs a) {
    const int r = blockIdx.y;
    const double R = (double)a.radii[r];
    const long long nplane = a.ndim == 3 ? (1ll << (a.log2n[0] + a.log2n[1])) : (1ll << a.log2n[0]);
    double sum = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nplane;
         q += (long long)gridDim.x * blockDim.x) {
        int i0, i1, i2;
        if (a.ndim == 3) {
            i0 = signed_index((int)(q >> a.log2n[1]), a.log2n[0]);
            i1 = signed_index((int)(q & ((1 << a.log2n[1]) - 1)), a.log2n[1]);
            i2 = -(1 << a.logM);
        } else {
            i0 = signed_index((int)q, a.log2n[0]);
            i1 = -(1 << a.logM);
            i2 = 0;
        }
        const double2 v = a.plane[q];
        const double mt = ball_transform(a.ndim, mode_k(a, i0, i1, i2) * R);
        sum += (v.x * v.x + v.y * v.y) * mt * mt;
    }
    block_add(sum, a.acc + r);
}

// Filter variant: E sigma_F^2(R) = sigma_f^2 sum A^2 m^2 / sum A^2; blockIdx.y
// = radius, and the blocks of radius 0 also sum A^2 into acc[nradii].
__global__ void k_window_filter(const __grid_constant__ WindowArgs a) {
    const int r = blockIdx.y;
    const double R = (double)a.radii[r];
    double sum = 0.0, norm = 0.0;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < a.half;
         m += (long long)gridDim.x * blockDim.x) {
        int i0, i1, i2;
        double w;
        half_mode(a, m, i0, i1, i2, w);
        // zero on the Nyquist planes (the stored half has none along the last axis)
        if (i0 == -(1 << (a.log2n[0] - 1)) || (a.ndim == 3 && i1 == -(1 << (a.log2n[1] - 1)))) continue;
        const float x = (float)i0 * __int_as_float((127 + 1 - a.log2n[0]) << 23);
        const float y = (float)i1 * __int_as_float((127 + 1 - a.log2n[1]) << 23);
        const float z = a.ndim == 3 ? (float)i2 * __int_as_float((127 + 1 - a.log2n[2]) << 23) : 0.0f;
        const float A = filter_amplitude(a.fp, x, y, z, a.ndim);
        const double a2 = w * (double)A * (double)A;
        if (a2 == 0.0) continue;
        const double mt = ball_transform(a.ndim, mode_k(a, i0, i1, i2) * R);
        sum += a2 * mt * mt;
        norm += a2;
    }
    block_add(sum, a.acc + r);
    if (r == 0) {
        __syncthreads();
        block_add(norm, a.acc + a.nradii);
    }
}

// Nyquist plane, step 1: v[row] = sum_j y[row][j] (-1)^j, the row's DFT at
// k_last = n_last / 2 (real for a real row); one warp per row.
template <int SRC>
__global__ void k_nyquist_rows(const void* y, long long nrows, int log2nl, double2* v) {
    const int lane = threadIdx.x & 31;
    const long long nl = 1ll << log2nl;
    for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < nrows;
         row += ((long long)gridDim.x * blockDim.x) >> 5) {
        double s = 0.0;
        for (long long j = lane; j < nl; j += 32) {
            double x;
            if constexpr (SRC == kSrcF32) {
                x = (double)static_cast<const float*>(y)[row * nl + j];
            } else if constexpr (SRC == kSrcBF16) {
                x = (double)__bfloat162float(static_cast<const __nv_bfloat16*>(y)[row * nl + j]);
            } else {
                x = (double)static_cast<const signed char*>(y)[row * nl + j];
            }
            s += (j & 1) ? -x : x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) v[row] = make_double2(s, 0.0);
    }
}

// Nyquist plane, step 2: a plain DFT along the middle axis of [A][L][B]
// complex doubles (out[a][k][b] = sum_n in[a][n][b] e^{-2 pi i k n / L}); the
// plane is at most 4096 x 4096 / 4096 long per axis, so O(L^2) per line.
__global__ void k_dft_axis(const double2* in, double2* out, long long A, int log2L, long long B) {
    const long long L = 1ll << log2L;
    const long long total = A * L * B;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long b = q % B, k = (q / B) & (L - 1), aa = q / (B * L);
        double re = 0.0, im = 0.0;
        for (long long n = 0; n < L; ++n) {
            const double2 x = in[(aa * L + n) * B + b];
            double s, c;
            sincospi(-2.0 * (double)((k * n) & (L - 1)) / (double)L, &s, &c);
            re += x.x * c - x.y * s;
            im += x.x * s + x.y * c;
        }
        out[q] = make_double2(re, im);
    }
}

// Per-mode outputs over the stored half spectrum (k_last < n_last / 2),
// natural layout [n0][n1][k_last]: the spectral density of a field,
// S(n) = |Y(n)|^2 / N, or the filter's A(n)^2 (Eq. 8: the target spectrum up
// to its normalisation; zero at n = 0 and on Nyquist planes).
__global__ void k_spectrum_modes(const float2* spec, long long half, float inv_n, float* out) {
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < half;
         m += (long long)gridDim.x * blockDim.x) {
        const float2 y = spec[m];
        out[m] = (y.x * y.x + y.y * y.y) * inv_n;
    }
}

__global__ void k_filter_modes(const __grid_constant__ WindowArgs a, float* out) {
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < a.half;
         m += (long long)gridDim.x * blockDim.x) {
        int i0, i1, i2;
        double w;
        half_mode(a, m, i0, i1, i2, w);
        float A = 0.0f;
        if (i0 != -(1 << (a.log2n[0] - 1)) && !(a.ndim == 3 && i1 == -(1 << (a.log2n[1] - 1)))) {
            const float x = (float)i0 * __int_as_float((127 + 1 - a.log2n[0]) << 23);
            const float y = (float)i1 * __int_as_float((127 + 1 - a.log2n[1]) << 23);
            const float z = a.ndim == 3 ? (float)i2 * __int_as_float((127 + 1 - a.log2n[2]) << 23) : 0.0f;
            A = filter_amplitude(a.fp, x, y, z, a.ndim);
        }
        out[m] = A * A;
    }
}

__global__ void k_window_finalize(const double* acc, int nradii, double scale, int by_norm, double* out) {
    const int r = threadIdx.x;
    if (r < nradii) out[r] = by_norm ? (acc[nradii] > 0.0 ? scale * acc[r] / acc[nradii] : 0.0) : scale * acc[r];
}

}  // namespace hf
