// kernels.cuh -- the pass kernels of the generator (arXiv 2509.08675, Sec. II.B).
//
// Data layout: the spectrum of a real lattice n0 x ... x n_{d-1} is kept as
// its r2c half along the contiguous axis WITHOUT the Nyquist plane:
// complex64 [n0][...][M], M = n_{d-1}/2, k_last = 0..M-1.  The filter is zero
// on every Nyquist plane and the spectrum bins drop |kappa| >= 1, so that
// plane never carries information; dropping it keeps every row a power of two.
//
// Passes (all persistent: a grid of resident CTAs walks contiguous chunks of
// tiles):
//   k_r2c   rows    noise (Philox + Box-Muller) or a stored field -> real FFT
//                   of every row -> half spectrum
//   k_cols  columns FFT along a strided axis; MODE_FILTER additionally does,
//                   per mode, G = A X (Eqs. 8, 12, 13), the Parseval sum and
//                   the field's spectrum bins, then the inverse along the same
//                   axis; MODE_BINS forms |X|^2/N and bins it
//   k_c2r   rows    inverse real FFT of every row -> scale to sigma_f (Eq. 15)
//                   -> store the field -> sign maps -> real FFT of each map row
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace hf {

enum NoiseSource { kSrcNoise = 0, kSrcF32 = 1, kSrcBF16 = 2, kSrcI8 = 3 };
enum ColMode { kModePlain = 0, kModeFilter = 1, kModeBins = 2 };

struct RowArgs {
    const void* src;        // real input rows (kSrcF32/BF16/I8)
    float2* out;            // [nrows][M] half spectrum
    long long nrows;
    int logTR;              // rows per CTA
    unsigned long long seed;
    unsigned int field_idx;
    const float2* tw;
};

struct C2RArgs {
    float2* spec;           // [nrows][M] filtered spectrum in; map spectra out (level t at spec + t * half)
    long long nrows;
    int logTR;
    long long half;         // N / 2
    long long N;
    void* out_f;            // field (F32 or BF16), may be null
    signed char* out_maps;  // nlev * N sign maps, may be null
    int nlev;
    float levels[kMaxLevels];
    const double* P;        // sum over the full lattice of |G|^2
    float sigma_f;
    const float2* tw;
};

struct ColArgs {
    float2* data;           // element (a, l, c) at data[a * bstride + l * B + c]
    long long B;            // contiguous columns
    long long A;            // batches
    long long bstride;
    int logTB;              // columns per CTA
    long long ntiles;       // A * B / TB
    const float2* tw;
    // mode decoding for the pass along axis 0 (FILTER, BINS)
    int ndim;
    int logM;               // 3D: column c -> n1 = c >> logM, k2 = c & (M - 1); 2D: k1 = c
    int log2n[3];
    FilterParams fp;
    BinParams bp;
    double* gbins;          // FILTER: raw field bins [nbins]; BINS: [A][nbins]
    double* gP;             // FILTER: Parseval sum
    float scale;            // BINS: 1 / N
};

__device__ __forceinline__ int signed_index(int i, int log2n) {
    return i < (1 << (log2n - 1)) ? i : i - (1 << log2n);
}

// |t|^p for t >= 0 (one term of the superellipse sum, Eq. 12).
__device__ __forceinline__ float pow_term(float t, float p) { return t > 0.0f ? exp2f(p * log2f(t)) : 0.0f; }

// A = sqrt(chi) from S = K^p (Eqs. 8, 12, 13): zero at K = 0.
__device__ __forceinline__ float amplitude_from_sum(const FilterParams& fp, float S) {
    if (!(S > 0.0f)) return 0.0f;
    const float log2K = log2f(S) * fp.inv_p;
    const float K = exp2f(log2K);
    // (K - k0)^2 - (K* - k0)^2 = (K - K*)(K + K* - 2 k0)
    const float d = (K - fp.kstar) * (K + fp.kstar - fp.two_k0);
    const float half_lnchi = fp.half_s_ln2 * (log2K - fp.log2_kstar) - d * fp.inv_2w2 * 0.5f;
    return expf(half_lnchi);
}

// A(kappa) for a rotated filter (the norm is not separable).
__device__ __forceinline__ float filter_amplitude(const FilterParams& fp, float x, float y, float z, int ndim) {
    const float xr = fmaf(fp.cr, x, fp.sr * y);
    const float yr = fmaf(fp.cr, y, -fp.sr * x);
    float S = pow_term(fabsf(xr) * fp.inv_a[0], fp.p) + pow_term(fabsf(yr) * fp.inv_a[1], fp.p);
    if (ndim == 3) S += pow_term(fabsf(z) * fp.inv_a[2], fp.p);
    return amplitude_from_sum(fp, S);
}

// Exact angular sector of a folded, nonzero vector (a1 > 0, or a1 = 0 < a0):
// the largest j with cross(d_j, a) >= 0, d_j the rounded edge directions.
__device__ __forceinline__ int sector_exact(const long long* ang, int ntheta, long long a0, long long a1) {
    int lo = 0, hi = ntheta - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ang[mid] * a1 - ang[ntheta + mid] * a0 >= 0)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Bin of a mode (signed indices), -1 when |kappa| >= 1.
// Radial: Q = |kappa|^2 nmax^2 = 4 sum (n_i nmax / n_i)^2 is an integer below
// 2^26, and bin b holds b^2 nmax^2 <= nr^2 Q < (b+1)^2 nmax^2, i.e.
// thr[b] <= Q < thr[b+1] with the integer thresholds thr[b] =
// ceil(b^2 nmax^2 / nr^2) (thr[nr] = nmax^2); a float square root gives the
// first guess and integer compares settle it.  Angular (2D): the folded angle
// from atan2f gives the sector unless it lies within 1e-4 of a sector edge,
// where the exact 64-bit cross products against the rounded edge directions
// decide.
__device__ __forceinline__ int bin_index(const BinParams& bp, const int* thr, const long long* ang, int n0, int n1,
                                         int n2, int ndim) {
    const int v0 = n0 << bp.shift[0];
    const int v1 = n1 << bp.shift[1];
    const int v2 = ndim == 3 ? (n2 << bp.shift[2]) : 0;
    const int Q = 4 * (v0 * v0 + v1 * v1 + v2 * v2);
    if (Q >= thr[bp.nr]) return -1;
    int b = (int)(sqrtf((float)Q) * __int_as_float((127 - bp.log2nmax) << 23) * (float)bp.nr);
    b = b < bp.nr - 1 ? b : bp.nr - 1;
    while (b > 0 && Q < thr[b]) --b;
    while (Q >= thr[b + 1]) ++b;
    int sector = 0;
    if (bp.ntheta > 1) {
        int a0 = v0, a1 = v1;
        if (a1 < 0 || (a1 == 0 && a0 < 0)) {
            a0 = -a0;
            a1 = -a1;
        }
        if (a0 != 0 || a1 != 0) {
            const float t = atan2f((float)a1, (float)a0) * ((float)bp.ntheta * 0.318309886183790672f);
            int s = (int)t;
            const float frac = t - (float)s;
            if (frac < 1e-4f || frac > 1.0f - 1e-4f || s >= bp.ntheta) {
                s = sector_exact(ang, bp.ntheta, a0, a1);
            }
            sector = s;
        }
    }
    return b * bp.ntheta + sector;
}

// Integer radial thresholds thr[b] = ceil(b^2 nmax^2 / nr^2), b = 0..nr.
__device__ __forceinline__ void fill_thresholds(const BinParams& bp, int* thr, int t, int T) {
    const unsigned long long nm2 = 1ull << (2 * bp.log2nmax);
    const unsigned long long nr2 = (unsigned long long)bp.nr * (unsigned long long)bp.nr;
    for (int b = t; b <= bp.nr; b += T) {
        const unsigned long long num = (unsigned long long)b * (unsigned long long)b * nm2;
        thr[b] = (int)((num + nr2 - 1) / nr2);
    }
}

__device__ __forceinline__ void chunk_of(long long ntiles, long long& t0, long long& t1) {
    const long long G = gridDim.x;
    t0 = ntiles * (long long)blockIdx.x / G;
    t1 = ntiles * ((long long)blockIdx.x + 1) / G;
}

// r2c post-processing of one row held in shared memory: from Z = DFT_M of
// z[j] = x[2j] + i x[2j+1], X[k] = (Z[k] + Z*[M-k])/2 - i W_N^k (Z[k] - Z*[M-k])/2.
template <int LOG2M>
__device__ __forceinline__ float2 r2c_post(float2 Z, float2 Zm_conj, const float2* __restrict__ tw, int k) {
    const float2 ev = cscale(cadd(Z, Zm_conj), 0.5f);
    const float2 od = cscale(cmul_i<-1>(csub(Z, Zm_conj)), 0.5f);
    const float2 w = __ldg(tw + (k << (kTwLog2 - LOG2M - 1)));
    return cadd(ev, cmul(od, w));
}

// ---------------------------------------------------------------------------
// Rows: real input -> half spectrum.
// ---------------------------------------------------------------------------
template <int LOG2M, int SRC>
__global__ void __launch_bounds__(256) k_r2c(const __grid_constant__ RowArgs a) {
    constexpr int M = 1 << LOG2M;
    constexpr int E = RowShape<LOG2M>::E;
    using PF = Plan<LOG2M, false>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    const Ctx c{(int)threadIdx.x, (int)blockDim.x, a.logTR};
    long long t0, t1;
    chunk_of(a.nrows >> a.logTR, t0, t1);
    const int nq = (1 << (a.logTR + LOG2M)) >> 1;  // blocks of four reals per tile
    for (long long tile = t0; tile < t1; ++tile) {
        const long long row0 = tile << a.logTR;
        __syncthreads();  // previous tile is done with shared memory
        for (int q = c.t; q < nq; q += c.T) {
            const long long gq = row0 * (M / 2) + q;  // global block index
            float4 x;
            if constexpr (SRC == kSrcNoise) {
                x = box_muller(noise_block(a.seed, a.field_idx, (unsigned long long)gq));
            } else if constexpr (SRC == kSrcF32) {
                x = __ldg(reinterpret_cast<const float4*>(a.src) + gq);
            } else if constexpr (SRC == kSrcBF16) {
                const uint2 raw = __ldg(reinterpret_cast<const uint2*>(a.src) + gq);
                const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
                const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
                x = make_float4(lo.x, lo.y, hi.x, hi.y);
            } else {
                const char4 raw = __ldg(reinterpret_cast<const char4*>(a.src) + gq);
                x = make_float4((float)raw.x, (float)raw.y, (float)raw.z, (float)raw.w);
            }
            const int e2 = 2 * q;
            const int b = e2 >> LOG2M, j = e2 & (M - 1);
            sm[smem_slot<LOG2M, true>(c, j, b)] = make_float2(x.x, x.y);
            sm[smem_slot<LOG2M, true>(c, j + 1, b)] = make_float2(x.z, x.w);
        }
        __syncthreads();
        float2 v[E];
        for_each_element<LOG2M, true, PF::first_radix(), E>(
            c, [&](int e, int b, int l) { v[e] = sm[smem_slot<LOG2M, true>(c, l, b)]; });
        fft<LOG2M, E, -1, false, true>(v, sm, a.tw, c);
        __syncthreads();
        for_each_element<LOG2M, true, PF::last_radix(), E>(
            c, [&](int e, int b, int l) { sm[smem_slot<LOG2M, true>(c, l, b)] = v[e]; });
        __syncthreads();
        for_each_element<LOG2M, true, PF::last_radix(), E>(c, [&](int e, int b, int k) {
            const float2 zc = cconj(sm[smem_slot<LOG2M, true>(c, (M - k) & (M - 1), b)]);
            a.out[(row0 + b) * M + k] = r2c_post<LOG2M>(v[e], zc, a.tw, k);
        });
    }
}

// ---------------------------------------------------------------------------
// Rows: filtered half spectrum -> field (Eq. 15) -> sign maps -> map spectra.
// ---------------------------------------------------------------------------
template <int LOG2M, int OUTDT>
__global__ void __launch_bounds__(256) k_c2r(const __grid_constant__ C2RArgs a) {
    constexpr int M = 1 << LOG2M;
    constexpr int E = RowShape<LOG2M>::E;
    using PF = Plan<LOG2M, false>;
    using PI = Plan<LOG2M, true>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    const Ctx c{(int)threadIdx.x, (int)blockDim.x, a.logTR};
    // f = sigma_f * u / sqrt(sum |G|^2), u the unnormalised inverse (the mean
    // is zero because A(0) = 0): Var = sum|G|^2 / N^2 by Parseval.
    const float scale = (float)((double)a.sigma_f / sqrt(*a.P));
    long long t0, t1;
    chunk_of(a.nrows >> a.logTR, t0, t1);
    for (long long tile = t0; tile < t1; ++tile) {
        const long long row0 = tile << a.logTR;
        float2 v[E];
        // c2r pre-processing: Z[k] = (X[k] + X*[M-k]) + i (X[k] - X*[M-k]) W_N^{-k}
        for_each_element<LOG2M, true, PI::first_radix(), E>(c, [&](int e, int b, int k) {
            const float2* rowp = a.spec + (row0 + b) * M;
            float2 X = rowp[k];
            float2 Xmc = make_float2(0.0f, 0.0f);
            if (k == 0) {
                X.y = 0.0f;  // the DC of a real row is real; the Nyquist term is zero
            } else {
                Xmc = cconj(rowp[M - k]);
            }
            const float2 ep = cadd(X, Xmc);
            const float2 w = __ldg(a.tw + (k << (kTwLog2 - LOG2M - 1)));
            const float2 op = cmulc(csub(X, Xmc), w);
            v[e] = cadd(ep, cmul_i<+1>(op));
        });
        fft<LOG2M, E, +1, true, true>(v, sm, a.tw, c);
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cscale(v[e], scale);
        // v[e] now holds f[2j], f[2j+1] of row b at the forward plan's input positions
        if (a.out_f != nullptr) {
            for_each_element<LOG2M, true, PF::first_radix(), E>(c, [&](int e, int b, int j) {
                const long long off = (row0 + b) * M + j;  // in pairs of reals
                if constexpr (OUTDT == 0) {
                    reinterpret_cast<float2*>(a.out_f)[off] = v[e];
                } else {
                    reinterpret_cast<__nv_bfloat162*>(a.out_f)[off] = __floats2bfloat162_rn(v[e].x, v[e].y);
                }
            });
        }
        for (int lev = 0; lev < a.nlev; ++lev) {
            const float t = a.levels[lev];
            float2 u[E];
#pragma unroll
            for (int e = 0; e < E; ++e)
                u[e] = make_float2(v[e].x >= t ? 1.0f : -1.0f, v[e].y >= t ? 1.0f : -1.0f);
            if (a.out_maps != nullptr) {
                for_each_element<LOG2M, true, PF::first_radix(), E>(c, [&](int e, int b, int j) {
                    char2 m;
                    m.x = u[e].x > 0.0f ? (signed char)1 : (signed char)-1;
                    m.y = u[e].y > 0.0f ? (signed char)1 : (signed char)-1;
                    reinterpret_cast<char2*>(a.out_maps + (long long)lev * a.N)[(row0 + b) * M + j] = m;
                });
            }
            fft<LOG2M, E, -1, false, true>(u, sm, a.tw, c);
            __syncthreads();
            for_each_element<LOG2M, true, PF::last_radix(), E>(
                c, [&](int e, int b, int l) { sm[smem_slot<LOG2M, true>(c, l, b)] = u[e]; });
            __syncthreads();
            float2* dst = a.spec + (long long)lev * a.half;
            for_each_element<LOG2M, true, PF::last_radix(), E>(c, [&](int e, int b, int k) {
                const float2 zc = cconj(sm[smem_slot<LOG2M, true>(c, (M - k) & (M - 1), b)]);
                dst[(row0 + b) * M + k] = r2c_post<LOG2M>(u[e], zc, a.tw, k);
            });
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Columns: FFT along a strided axis (+ filter / bins on the last axis pass).
// ---------------------------------------------------------------------------
template <int LOG2L, int MODE, int DIR>
__global__ void __launch_bounds__(512) k_cols(const __grid_constant__ ColArgs a) {
    constexpr int E = ColShape<LOG2L>::E;
    using PF = Plan<LOG2L, false>;
    using PI = Plan<LOG2L, true>;
    constexpr bool kAcc = MODE != kModePlain;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Ctx c{(int)threadIdx.x, (int)blockDim.x, a.logTB};
    float2* sm = reinterpret_cast<float2*>(smem_raw);
    const int nb = a.bp.nbins;
    double* dbin = reinterpret_cast<double*>(sm + (1 << (a.logTB + LOG2L)));  // nb + 1 (last: Parseval)
    long long* ang = reinterpret_cast<long long*>(dbin + nb + 1);              // 2 * ntheta
    float* fbin = reinterpret_cast<float*>(ang + 2 * a.bp.ntheta);             // nb + 1
    int* thr = reinterpret_cast<int*>(fbin + nb + 1);                          // nr + 1
    float* tab0 = reinterpret_cast<float*>(thr + a.bp.nr + 1);                 // FILTER: |kappa_0 / a|^p, L
    if constexpr (MODE == kModeFilter) {
        if (!a.fp.rotated) {
            for (int l = c.t; l < (1 << LOG2L); l += c.T) {
                const float x = (float)signed_index(l, LOG2L) * __int_as_float((127 + 1 - LOG2L) << 23);
                tab0[l] = l == (1 << (LOG2L - 1)) ? 0.0f : powf(fabsf(x) * a.fp.inv_a[0], a.fp.p);
            }
        }
    }
    if constexpr (kAcc) {
        for (int i = c.t; i <= nb; i += c.T) {
            dbin[i] = 0.0;
            fbin[i] = 0.0f;
        }
        for (int i = c.t; i < a.bp.ntheta; i += c.T) {
            ang[i] = a.bp.ang_c[i];
            ang[a.bp.ntheta + i] = a.bp.ang_s[i];
        }
        if (nb > 0) fill_thresholds(a.bp, thr, c.t, c.T);
        __syncthreads();
    }
    const long long tpb = a.B >> a.logTB;
    long long t0, t1;
    chunk_of(a.ntiles, t0, t1);
    long long cur = -1;
    auto flush = [&](long long batch) {
        __syncthreads();
        double* g = MODE == kModeBins ? a.gbins + batch * nb : a.gbins;
        for (int i = c.t; i < nb; i += c.T) {
            if (dbin[i] != 0.0) atomicAdd(g + i, dbin[i]);
            dbin[i] = 0.0;
        }
        if (MODE == kModeFilter && c.t == 0) {
            atomicAdd(a.gP, dbin[nb]);
            dbin[nb] = 0.0;
        }
        __syncthreads();
    };
    for (long long ti = t0; ti < t1; ++ti) {
        const long long ab = ti / tpb;
        const long long c0 = (ti - ab * tpb) << a.logTB;
        if constexpr (MODE == kModeBins) {
            if (ab != cur) {
                if (cur >= 0) flush(cur);
                cur = ab;
            }
        }
        float2* base = a.data + ab * a.bstride + c0;
        float2 v[E];
        if constexpr (MODE == kModePlain && DIR > 0) {
            for_each_element<LOG2L, false, PI::first_radix(), E>(
                c, [&](int e, int b, int l) { v[e] = base[(long long)l * a.B + b]; });
            fft<LOG2L, E, +1, true, false>(v, sm, a.tw, c);
            for_each_element<LOG2L, false, PI::last_radix(), E>(
                c, [&](int e, int b, int l) { base[(long long)l * a.B + b] = v[e]; });
        } else {
            for_each_element<LOG2L, false, PF::first_radix(), E>(
                c, [&](int e, int b, int l) { v[e] = base[(long long)l * a.B + b]; });
            fft<LOG2L, E, -1, false, false>(v, sm, a.tw, c);
            if constexpr (MODE == kModePlain) {
                for_each_element<LOG2L, false, PF::last_radix(), E>(
                    c, [&](int e, int b, int l) { base[(long long)l * a.B + b] = v[e]; });
            } else {
                // Per-mode power (weight 2 for the k_last > 0 half) goes through
                // shared memory so that each thread then owns E consecutive n0 of
                // one column: consecutive modes share a bin, so one atomic per
                // run of equal bins replaces one per mode.
                constexpr int L = 1 << LOG2L;
                float pacc = 0.0f;
                if constexpr (MODE == kModeFilter) {
                    // a thread's column is fixed: T is a multiple of TB
                    const int col = (int)(c0 + (c.t & ((1 << c.logTB) - 1)));
                    int n1, n2;
                    if (a.ndim == 3) {
                        n1 = signed_index(col >> a.logM, a.log2n[1]);
                        n2 = col & ((1 << a.logM) - 1);
                    } else {
                        n1 = col;
                        n2 = 0;
                    }
                    const bool nyq_col = a.ndim == 3 && n1 == -(1 << (a.log2n[1] - 1));
                    const float y = (float)n1 * __int_as_float((127 + 1 - a.log2n[1]) << 23);
                    const float z = a.ndim == 3 ? (float)n2 * __int_as_float((127 + 1 - a.log2n[2]) << 23) : 0.0f;
                    float s_col = 0.0f;  // separable case: the column's terms of the sum
                    if (!a.fp.rotated) {
                        s_col = powf(fabsf(y) * a.fp.inv_a[1], a.fp.p);
                        if (a.ndim == 3) s_col += powf(fabsf(z) * a.fp.inv_a[2], a.fp.p);
                    }
                    for_each_element<LOG2L, false, PF::last_radix(), E>(c, [&](int e, int b, int l) {
                        const bool nyq = nyq_col || l == (1 << (LOG2L - 1));
                        float h = 0.0f;
                        if (!nyq) {
                            if (!a.fp.rotated) {
                                h = amplitude_from_sum(a.fp, tab0[l] + s_col);
                            } else {
                                const float x = (float)signed_index(l, LOG2L) * __int_as_float((127 + 1 - LOG2L) << 23);
                                h = filter_amplitude(a.fp, x, y, z, a.ndim);
                            }
                        }
                        v[e] = cscale(v[e], h);
                    });
                }
                if (nb > 0 || MODE == kModeFilter) {
                    float* ps = reinterpret_cast<float*>(sm);  // [b][L + 1] powers
                    __syncthreads();                           // the FFT's last exchange is read
                    for_each_element<LOG2L, false, PF::last_radix(), E>(c, [&](int e, int b, int l) {
                        const int col = (int)(c0 + b);
                        const int klast = a.ndim == 3 ? (col & ((1 << a.logM) - 1)) : col;
                        const float w = klast == 0 ? 1.0f : 2.0f;  // k and -k share a half-spectrum slot
                        const float pw = (MODE == kModeBins ? w * a.scale : w) * cabs2(v[e]);
                        pacc += pw;
                        ps[b * (L + 1) + l] = pw;
                    });
                    __syncthreads();
                    if (nb > 0) {
                        const int g0 = c.t * E;
                        const int b = g0 >> LOG2L;
                        const int l0 = g0 & (L - 1);
                        const int col = (int)(c0 + b);
                        int n1, n2;
                        if (a.ndim == 3) {
                            n1 = signed_index(col >> a.logM, a.log2n[1]);
                            n2 = col & ((1 << a.logM) - 1);
                        } else {
                            n1 = col;
                            n2 = 0;
                        }
                        int cur_bin = -1;
                        float acc = 0.0f;
                        const int rot = c.t & (E - 1);  // staggered start: spreads the banks
#pragma unroll 4
                        for (int i = 0; i < E; ++i) {
                            const int l = l0 + ((i + rot) & (E - 1));
                            const float pw = ps[b * (L + 1) + l];
                            const int bin = bin_index(a.bp, thr, ang, signed_index(l, LOG2L), n1, n2, a.ndim);
                            if (bin != cur_bin) {
                                if (cur_bin >= 0 && acc != 0.0f) atomicAdd(fbin + cur_bin, acc);
                                cur_bin = bin;
                                acc = 0.0f;
                            }
                            acc += pw;
                        }
                        if (cur_bin >= 0 && acc != 0.0f) atomicAdd(fbin + cur_bin, acc);
                    }
                }
                if constexpr (MODE == kModeFilter) {
                    if (c.T >= 32) {  // T is a power of two: whole warps
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) pacc += __shfl_xor_sync(0xffffffffu, pacc, o);
                        if ((c.t & 31) == 0) atomicAdd(fbin + nb, pacc);
                    } else {
                        atomicAdd(fbin + nb, pacc);
                    }
                    fft<LOG2L, E, +1, true, false>(v, sm, a.tw, c);
                    for_each_element<LOG2L, false, PI::last_radix(), E>(
                        c, [&](int e, int b, int l) { base[(long long)l * a.B + b] = v[e]; });
                }
            }
        }
        if constexpr (kAcc) {
            __syncthreads();
            for (int i = c.t; i <= nb; i += c.T) {
                dbin[i] += (double)fbin[i];
                fbin[i] = 0.0f;
            }
            __syncthreads();
        }
    }
    if constexpr (MODE == kModeBins) {
        if (cur >= 0) flush(cur);
    } else if constexpr (MODE == kModeFilter) {
        flush(0);
    }
}

}  // namespace hf
