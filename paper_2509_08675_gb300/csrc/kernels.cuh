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
#include <type_traits>

#include "fft.cuh"
#include "tma.cuh"

namespace hf {

// kSrcNoiseBatch: noise of many fields of one lattice in one launch (a field's
// rows are consecutive; see RowArgs).  kModeFilterBatch: the filter pass over
// many fields, each batch with its own filter (see ColArgs).
enum NoiseSource { kSrcNoise = 0, kSrcF32 = 1, kSrcBF16 = 2, kSrcI8 = 3, kSrcNoiseBatch = 4 };
enum ColMode { kModePlain = 0, kModeFilter = 1, kModeBins = 2, kModeKspace = 3, kModeFilterBatch = 4 };
// c2r output: FP32 or BF16 field; kOutBatch: FP32 fields of many fields of one lattice
enum C2ROut { kOutF32 = 0, kOutBF16 = 1, kOutBatch = 2 };

struct RowArgs {
    const void* src;        // real input rows (kSrcF32/BF16/I8)
    float2* out;            // [nrows][M] half spectrum
    long long nrows;
    unsigned long long seed;
    unsigned int field_idx;
    const float2* tw;       // plan twiddles (4096)
    // kSrcNoiseBatch: row r belongs to field f = r >> log2_rows_field, whose noise
    // is that of (fseed[f], fidx[f]) with blocks counted from the field's first row
    const unsigned long long* fseed;
    const unsigned* fidx;
    int log2_rows_field;
    long long nrows_valid;  // kSrcNoiseBatch: rows at or past this (the last tile's tail) are not written
    unsigned int keys[20];  // kSrcNoise: the Philox round keys of seed (philox4x32_10_keyed)
};

struct C2RArgs {
    float2* spec;           // [nrows][M] filtered spectrum in; map spectra out (level t at spec + t * half)
    long long nrows;
    long long half;         // N / 2
    long long N;
    void* out_f;            // field (F32 or BF16), may be null
    signed char* out_maps;  // nlev * N sign maps, may be null
    int nlev;
    float levels[kMaxLevels];
    const double* P;        // sum over the full lattice of |G|^2, followed by the field's raw bins
    float sigma_f;
    // CTA 0 also finishes the field's bins, sums_f[b] += raw[b] N / P (S_f = N |G|^2 / P),
    // and clears the other accumulator set (the next field's P and raw bins)
    double* sums_f;         // may be null (no field bins)
    int nbins;
    double* next_acc;       // 1 + nbins doubles to clear
    int next_len;
    const float2* tw;
    unsigned* status;       // workspace status word (kStatusTimeout)
    long long wait_budget;  // clock cycles allowed per mbarrier wait
    int inject_skip;        // test hook: 1 = the first tile's load is never issued
    int kz;                 // entries k_last >= kz of each row are zero (<= M)
    // kOutBatch (one level per field): row r belongs to field f = r >> log2_rows_field,
    // scaled by fscale[f] (sigma_f / sqrt(P_f), set by k_fields_scale), thresholded at
    // flevel[f]; its field and map start fout[f] reals into out_f / out_maps.  P,
    // sums_f and next_acc are not used.
    int log2_rows_field;
    const float* fscale;
    const float* flevel;
    const long long* fout;
    long long nrows_valid;  // kOutBatch: rows at or past this are neither loaded nor written
    // 1: out_maps holds one bit per site (32-bit words, site i at bit i mod 32 of word
    // i / 32 of its map, 1 for +1; a batched field's map from site fout[f] on)
    int map_bits;
};

struct ColArgs {
    CUtensorMap map;        // (B, L, A) of 8-byte elements, box (TB, min(L, 256), 1); loads and stores
    float2* data;           // element (a, l, c) at data[a * bstride + l * B + c]
    long long B;            // contiguous columns
    long long A;            // batches
    long long bstride;
    long long ntiles;       // A * tpb
    // Tiles that are run: the columns form rows of row_tiles tiles, of which
    // the first live_tiles of each row are run (all with row_tiles =
    // live_tiles = 1); tpb of them per batch.
    long long tpb;
    int row_tiles, live_tiles;
    const float2* tw;
    // mode decoding for the pass along axis 0 (FILTER, BINS)
    int ndim;
    int logM;               // 3D: column c -> n1 = c >> logM, k2 = c & (M - 1); 2D: k1 = c
    int log2n[3];
    FilterParams fp;
    BinParams bp;
    const unsigned short* bintab;  // FILTER/BINS: bin of every mode in tile order (tile, b, l); 0xFFFF = dropped
    double* gbins;          // FILTER: raw field bins [nbins]; BINS: [A][nbins]
    double* gP;             // FILTER: Parseval sum
    float scale;            // BINS: 1 / N
    unsigned* status;       // workspace status word (kStatusTimeout)
    long long wait_budget;  // clock cycles allowed per mbarrier wait
    int inject_skip;        // test hook: 1 = the first tile's load is never issued (its wait must time out)
    // KSPACE: the noise coefficients are drawn in the pass instead of loaded
    unsigned long long seed;
    unsigned int field_idx;
    float kscale;           // sqrt(N / 2)
    // FILTER_BATCH: batch ab (a field) is filtered with fparr[ab] and gathers its
    // Parseval sum at gP + ab acc_stride and its raw field bins at gbins + ab acc_stride
    const FilterParams* fparr;
    long long acc_stride;
    // BINS: batch ab's bins at gbins + boff[ab] when boff is set (else + ab nbins)
    const long long* boff;
    int interleave;         // 1: CTA c runs tiles c, c + grid, ...; 0: a contiguous chunk (see tiles_of)
};

// Minimum resident CTAs per SM asked of the compiler: keeps the kernels of
// 128 threads or more at 128 registers per thread or fewer (65536 / (128 T)
// CTAs of T threads); the small tiles of tiny lattices are left unbounded.
// Sign maps stored one bit per site (site i at bit i mod 32 of word i / 32).
// The c2r kernel packs whole 16-pair words itself when each row holds whole
// words (M >= 16), or, for a single field (rows contiguous), when its tile of
// TR rows does (TR M >= 16); otherwise it ORs bits into words cleared
// beforehand.
__host__ __device__ constexpr bool map_bits_packed(int log2m, int logtr, bool batch) {
    return log2m >= 4 || (!batch && log2m + logtr >= 4);
}

// Four bytes holding 2-bit values b0..b3 -> b0 | b1 << 2 | b2 << 4 | b3 << 6.
__device__ __forceinline__ uint32_t pack_two_bit_bytes(uint32_t x) {
    const uint32_t r = x | (x >> 6);  // b1 to bits 2-3, b2 to 10-11, b3 to 18-19
    return (r | (r >> 12)) & 0xffu;    // b2 to 4-5, b3 to 6-7
}

constexpr int min_blocks(int T) { return T >= 512 ? 1 : (T >= 128 ? 512 / T : 1); }
// Three CTAs of 256 threads (80 registers) for the passes that gain more from
// occupancy than they lose to register pressure (measured: the 256-point
// noise rows of 512^3 0.428 -> 0.408 ms, the 512-point ones of 1024^3 3.53 ->
// 3.44 ms despite a few spills, the 512^3 maps' bins 0.308 -> 0.270 ms; the
// 2048-point noise rows, the 256-point c2r rows and the filter pass lose).
constexpr int min_blocks_r2c(int log2m, int T) { return (log2m <= 9 && T == 256) ? 3 : min_blocks(T); }
constexpr int min_blocks_cols(int mode, int T) { return (mode == 2 && T == 256) ? 3 : min_blocks(T); }

__device__ __forceinline__ int signed_index(int i, int log2n) {
    return i < (1 << (log2n - 1)) ? i : i - (1 << log2n);
}

// Filter amplitude, Eqs. (8), (12), (13), evaluated in the log domain so that
// S = sum |kappa'_i / a_i|^p neither underflows nor overflows for any p: each
// term enters as u_i = p log2 |kappa'_i / a_i| and log2 S = m + log2 sum
// 2^(u_i - m), m = max u_i.  fast_lg2/fast_ex2 are the hardware
// approximations (absolute error ~2^-22 in a log2, relative ~2^-22 in a power
// of two).  A narrow band (small w) multiplies the relative error of K by
// about 2 |K - k0| K / (w^2 ln 4) in log2 A, so K itself comes from the
// library exp2f, and the per-axis terms that are tabulated (once per CTA or
// tile) from log2f; an error in log2 S is divided by p in log2 K.
constexpr float kLog2Zero = -1e30f;  // u of a zero term (kappa'_i = 0)

__device__ __forceinline__ float fast_lg2(float x) { return lg2_approx(x); }
__device__ __forceinline__ float fast_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// u = p log2 t for t > 0; kLog2Zero for t = 0 (hardware log2; plog2_exact: library log2f).
__device__ __forceinline__ float plog2(float t, float p) { return t > 0.0f ? p * fast_lg2(t) : kLog2Zero; }
__device__ __forceinline__ float plog2_exact(float t, float p) { return t > 0.0f ? p * log2f(t) : kLog2Zero; }

// log2(2^a + 2^b) without forming either power.
__device__ __forceinline__ float log2_sum2(float a, float b) {
    const float m = fmaxf(a, b);
    return m + fast_lg2(1.0f + fast_ex2(fminf(a, b) - m));
}

// A = sqrt(chi) from log2 S, S = K^p: zero at K = 0.  With
// (K - k0)^2 - (K* - k0)^2 = (K - K*)(K + K* - 2 k0), A = exp(ln(chi) / 2) is
// one power of two.
__device__ __forceinline__ float amplitude_from_log2s(const FilterParams& fp, float l2s) {
    if (l2s < 0.5f * kLog2Zero) return 0.0f;
    const float log2K = l2s * fp.inv_p;
    const float K = exp2f(log2K);
    const float d = (K - fp.kstar) * (K + fp.kstar - fp.two_k0);
    return fast_ex2(fmaf(fp.half_s, log2K - fp.log2_kstar, -fp.c_d * d));
}

// A(kappa) for a rotated filter (the norm is not separable).
__device__ __forceinline__ float filter_amplitude(const FilterParams& fp, float x, float y, float z, int ndim) {
    const float xr = fmaf(fp.cr, x, fp.sr * y);
    const float yr = fmaf(fp.cr, y, -fp.sr * x);
    const float u0 = plog2(fabsf(xr) * fp.inv_a[0], fp.p);
    const float u1 = plog2(fabsf(yr) * fp.inv_a[1], fp.p);
    const float u2 = ndim == 3 ? plog2(fabsf(z) * fp.inv_a[2], fp.p) : kLog2Zero;
    const float m = fmaxf(fmaxf(u0, u1), u2);
    // log2 S >= m: K is zero, or far enough out that the power of two flushes to 0
    if (m < 0.5f * kLog2Zero || m >= fp.u_zero) return 0.0f;
    return amplitude_from_log2s(fp, m + fast_lg2(fast_ex2(u0 - m) + fast_ex2(u1 - m) + fast_ex2(u2 - m)));
}

// ---------------------------------------------------------------------------
// Binning.  Radial: Q = |kappa|^2 nmax^2 = 4 sum (n_i nmax / n_i)^2 is an
// integer below 2^26 and bin b holds b^2 nmax^2 <= nr^2 Q < (b+1)^2 nmax^2,
// i.e. thr[b] <= Q < thr[b+1] with the integer thresholds thr[b] =
// ceil(b^2 nmax^2 / nr^2) (thr[nr] = nmax^2: beyond it |kappa| >= 1, dropped).
// Angular (2D): the folded vector's sector is the largest j with
// cross(d_j, a) >= 0 for the edge directions d_j = round(2^30 (cos, sin)
// (j pi / ntheta)), j = 0..ntheta, d_ntheta = (-2^30, 0).
// ---------------------------------------------------------------------------
// Angle table in shared memory: C_j at ang[j], S_j at ang[ntheta + 1 + j].
__device__ __forceinline__ long long ang_c(const long long* ang, int j) { return ang[j]; }
__device__ __forceinline__ long long ang_s(const long long* ang, int nt, int j) { return ang[nt + 1 + j]; }

__device__ __forceinline__ long long cross_edge(const long long* ang, int nt, int j, int a0, int a1) {
    return ang_c(ang, j) * (long long)a1 - ang_s(ang, nt, j) * (long long)a0;
}

// Exact sector of a folded, nonzero vector by bisection.
__device__ __forceinline__ int sector_exact(const long long* ang, int ntheta, int a0, int a1) {
    int lo = 0, hi = ntheta - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cross_edge(ang, ntheta, mid, a0, a1) >= 0)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void fold_vector(int& a0, int& a1) {
    if (a1 < 0 || (a1 == 0 && a0 < 0)) {
        a0 = -a0;
        a1 = -a1;
    }
}

// Radial bin (or nr when outside) from scratch: a float square root gives the
// first guess and integer compares settle it.
__device__ __forceinline__ int radial_from_scratch(const BinParams& bp, const int* thr, int Q) {
    if (Q >= thr[bp.nr]) return bp.nr;
    int b = (int)(sqrtf((float)Q) * __int_as_float((127 - bp.log2nmax) << 23) * (float)bp.nr);
    b = b < bp.nr - 1 ? b : bp.nr - 1;
    while (b > 0 && Q < thr[b]) --b;
    while (Q >= thr[b + 1]) ++b;
    return b;
}

// Sector from scratch: the folded angle from atan2f gives it unless it lies
// within 1e-4 of an edge, where the exact bisection decides.
__device__ __forceinline__ int sector_from_scratch(const BinParams& bp, const long long* ang, int a0, int a1) {
    if (a0 == 0 && a1 == 0) return 0;
    const float t = atan2f((float)a1, (float)a0) * ((float)bp.ntheta * 0.318309886183790672f);
    int s = (int)t;
    const float frac = t - (float)s;
    if (frac < 1e-4f || frac > 1.0f - 1e-4f || s >= bp.ntheta) s = sector_exact(ang, bp.ntheta, a0, a1);
    return s;
}

// Bin of one mode (signed indices), -1 when |kappa| >= 1.
__device__ __forceinline__ int bin_index(const BinParams& bp, const int* thr, const long long* ang, int n0, int n1,
                                         int n2, int ndim) {
    const int v0 = n0 << bp.shift[0];
    const int v1 = n1 << bp.shift[1];
    const int v2 = ndim == 3 ? (n2 << bp.shift[2]) : 0;
    const int Q = 4 * (v0 * v0 + v1 * v1 + v2 * v2);
    const int rb = radial_from_scratch(bp, thr, Q);
    if (rb >= bp.nr) return -1;
    if (bp.ntheta == 1) return rb;
    int a0 = v0, a1 = v1;
    fold_vector(a0, a1);
    return rb * bp.ntheta + sector_from_scratch(bp, ang, a0, a1);
}

// Angle table (ntheta + 1 edges) from the parameter block into shared memory.
__device__ __forceinline__ void fill_angles(const BinParams& bp, long long* ang, int t, int T) {
    for (int i = t; i <= bp.ntheta; i += T) {
        ang[i] = i < bp.ntheta ? bp.ang_c[i] : -(1ll << 30);
        ang[bp.ntheta + 1 + i] = i < bp.ntheta ? bp.ang_s[i] : 0ll;
    }
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

// The tiles a CTA of a strided pass runs: tile first + k step for k < cnt.
// Contiguous chunks (step 1), or every grid-th tile (interleaved): then
// neighbouring tiles run at about the same time on different CTAs, so the
// narrow tiles whose box rows share DRAM sectors meet in L2 instead of each
// fetching the sector again.
__device__ __forceinline__ void tiles_of(long long ntiles, int interleave, long long& first, long long& step,
                                         long long& cnt) {
    if (interleave) {
        first = blockIdx.x;
        step = gridDim.x;
        cnt = ntiles > first ? (ntiles - first + step - 1) / step : 0;
    } else {
        long long t0, t1;
        chunk_of(ntiles, t0, t1);
        first = t0;
        step = 1;
        cnt = t1 - t0;
    }
}

// k-space noise: Philox block J of counter word 3 = 1 gives the coefficients
// of the mode pair (k_last even, k_last + 1) of one row, each sqrt(N/2) Z
// with Z = sqrt(-2 ln u_a) exp(2 pi i u_b) from the pair's two words.
__device__ __forceinline__ void kspace_pair(unsigned long long seed, unsigned int field_idx, float kscale,
                                            unsigned long long J, float2& z0, float2& z1) {
    const uint4 x = philox4x32_10(make_uint4((uint32_t)J, (uint32_t)(J >> 32), field_idx, 1u), (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    const float4 z = box_muller(x);
    z0 = make_float2(z.x * kscale, z.y * kscale);
    z1 = make_float2(z.z * kscale, z.w * kscale);
}

// One elected thread polls the mbarrier (bounded); the CTA then agrees.
// Returns false (for every thread) when the wait ran out.
__device__ __forceinline__ bool cta_wait(uint64_t* bar, uint32_t parity, long long budget) {
    bool ok = true;
    if (threadIdx.x == 0) ok = mbar_wait_bounded(bar, parity, budget);
    return !__syncthreads_or(!ok);
}

// r2c post-processing: from Z = DFT_M of z[j] = x[2j] + i x[2j+1],
// X[k] = (Z[k] + Z*[M-k])/2 - i W_N^k (Z[k] - Z*[M-k])/2, with W_N^k = tw[k]
// in the CTA's table of length N = 2M.
__device__ __forceinline__ float2 r2c_post(float2 Z, float2 Zm_conj, float2 w) {
    const float2 ev = cscale(cadd(Z, Zm_conj), 0.5f);
    const float2 od = cscale(cmul_i<-1>(csub(Z, Zm_conj)), 0.5f);
    return cadd(ev, cmul(od, w));
}

// ---------------------------------------------------------------------------
// Rows: real input -> half spectrum.
// ---------------------------------------------------------------------------
template <int LOG2M, int LOGTR, int SRC>
__global__ void __launch_bounds__(Geo<LOG2M, LOGTR, true>::T, min_blocks_r2c(LOG2M, Geo<LOG2M, LOGTR, true>::T))
    k_r2c(const __grid_constant__ RowArgs a) {
    using G = Geo<LOG2M, LOGTR, true>;
    constexpr int M = G::L;
    constexpr int E = G::E;
    using PF = Plan<LOG2M, false>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);  // TR * M exchange
    float2* tw = sm + G::TB * M;                        // W_{2M}^k, k < M
    float2* twf = tw + M;                               // stage tables of the forward plan
    const int t = threadIdx.x;
    load_half_twiddles<LOG2M>(tw, a.tw, t, G::T);
    load_stage_twiddles<LOG2M, false>(twf, a.tw, t, G::T);
    long long t0, t1;
    chunk_of(a.nrows >> LOGTR, t0, t1);
    constexpr int nq = (G::TB * M) / 2;  // blocks of four reals per tile
    for (long long tile = t0; tile < t1; ++tile) {
        const long long row0 = tile << LOGTR;
        __syncthreads();  // previous tile is done with shared memory (and the twiddles are loaded)
#pragma unroll
        for (int q = t; q < nq; q += G::T) {
            const long long gq = row0 * (M / 2) + q;  // global block index
            float4 x;
            if constexpr (SRC == kSrcNoise) {
                x = box_muller(philox4x32_10_keyed(
                    make_uint4((uint32_t)gq, (uint32_t)((unsigned long long)gq >> 32), a.field_idx, 0u), a.keys));
            } else if constexpr (SRC == kSrcNoiseBatch) {
                // a row holds M / 2 blocks of four reals; the last tile may run past the fields
                if ((gq >> (LOG2M - 1)) < a.nrows_valid) {
                    const long long f = gq >> (LOG2M - 1 + a.log2_rows_field);
                    const long long jl = gq - (f << (LOG2M - 1 + a.log2_rows_field));
                    x = box_muller(noise_block(a.fseed[f], a.fidx[f], (unsigned long long)jl));
                } else {
                    x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
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
            sm[smem_slot<G>(j, b)] = make_float2(x.x, x.y);
            sm[smem_slot<G>(j + 1, b)] = make_float2(x.z, x.w);
        }
        __syncthreads();
        float2 v[E];
        for_each_element<G, PF::first_radix()>(t, [&](int e, int b, int l) { v[e] = sm[smem_slot<G>(l, b)]; });
        fft<G, -1, false>(v, sm, twf, t);
        __syncthreads();
        for_each_element<G, PF::last_radix()>(t, [&](int e, int b, int l) { sm[smem_slot<G>(l, b)] = v[e]; });
        __syncthreads();
        for_each_element<G, PF::last_radix()>(t, [&](int e, int b, int k) {
            const float2 zc = cconj(sm[smem_slot<G>((M - k) & (M - 1), b)]);
            if (SRC != kSrcNoiseBatch || row0 + b < a.nrows_valid)
                a.out[(row0 + b) * M + k] = r2c_post(v[e], zc, tw[k]);
        });
    }
}

// ---------------------------------------------------------------------------
// Rows: filtered half spectrum -> field (Eq. 15) -> sign maps -> map spectra.
// Row tiles (TR contiguous rows) arrive by 1D bulk copies into two
// shared-memory buffers, the next tile in flight while the current one is
// transformed; the current buffer then serves as the FFT exchange area.
// ---------------------------------------------------------------------------
// ONE: a single sign-map level, known at compile time (the host picks it for
// nlev = 1; batches always have one level per field): the field's registers
// are free once its map is formed, so single-field rows of up to 256 points
// fit three 256-thread CTAs per SM at 80 registers without spills (the
// 512-point rows would spill there and keep two).
constexpr int min_blocks_c2r(int log2m, int T, bool one, int outdt) {
    return (one && outdt != kOutBatch && log2m <= 8 && T == 256) ? 3 : min_blocks(T);
}

template <int LOG2M, int LOGTR, int OUTDT, bool ONE>
__global__ void __launch_bounds__(Geo<LOG2M, LOGTR, true>::T,
                                  min_blocks_c2r(LOG2M, Geo<LOG2M, LOGTR, true>::T, ONE, OUTDT))
    k_c2r(const __grid_constant__ C2RArgs a) {
    using G = Geo<LOG2M, LOGTR, true>;
    constexpr int M = G::L;
    constexpr int E = G::E;
    using PF = Plan<LOG2M, false>;
    using PI = Plan<LOG2M, true>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int tile_elems = G::TB * M;
    float2* const buf0 = reinterpret_cast<float2*>(smem_raw);  // two tile buffers: buf0 + s tile_elems
    float2* tw = buf0 + 2 * tile_elems;  // W_{2M}^k, k < M
    float2* twf = tw + M;               // stage tables: forward plan, then its reverse
    uint64_t* bar = reinterpret_cast<uint64_t*>(twf + plan_twiddle_slots<LOG2M>());
    constexpr uint32_t tile_bytes = (uint32_t)tile_elems * (uint32_t)sizeof(float2);
    const int t = threadIdx.x;
    // f = sigma_f * u / sqrt(sum |G|^2), u the unnormalised inverse (the mean
    // is zero because A(0) = 0): Var = sum|G|^2 / N^2 by Parseval.
    // (batched fields: each field's scale comes from fscale)
    float scale = 0.0f;
    if constexpr (OUTDT != kOutBatch) {
        const double Pv = *a.P;
        // no power at all (a band beyond the lattice): Eq. (15) is read as f = 0
        const bool empty = !(Pv > 0.0);
        scale = empty ? 0.0f : (float)((double)a.sigma_f / sqrt(Pv));
        if (blockIdx.x == 0) {
            if (empty && t == 0) atomicOr(a.status, kStatusNoPower);
            if (a.sums_f && !empty) {
                const double sN = (double)a.N / Pv;
                for (int b = t; b < a.nbins; b += G::T) a.sums_f[b] += a.P[1 + b] * sN;
            }
            for (int i = t; i < a.next_len; i += G::T) a.next_acc[i] = 0.0;
        }
    }
    // field of row r and its first row (batched fields)
    [[maybe_unused]] auto field_of = [&](long long r) { return r >> a.log2_rows_field; };
    long long t0, t1;
    chunk_of(a.nrows >> LOGTR, t0, t1);
    // Entries k_last >= kz are zero (the filter's band ends before them) and
    // were not written by the passes before: they are loaded with the rest of
    // the tile (one bulk copy measured faster than a copy per row of the
    // entries below kz) and read as zero.
    const int kz = a.kz;
    auto issue = [&](long long tile, float2* dst, uint64_t* b) {
        uint32_t bytes = tile_bytes;
        if constexpr (OUTDT == kOutBatch) {  // the last tile may hold fewer rows
            const long long rows = a.nrows_valid - (tile << LOGTR);
            if (rows < G::TB) bytes = (uint32_t)rows * (uint32_t)(M * sizeof(float2));
        }
        mbar_arrive_expect_tx(b, bytes);
        bulk_load(dst, a.spec + tile * tile_elems, bytes, b);
    };
    load_half_twiddles<LOG2M>(tw, a.tw, t, G::T);
    float2* twi = load_plan_twiddles<LOG2M>(twf, a.tw, t, G::T);
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (t == 0) {
        if (t0 < t1 && !a.inject_skip) issue(t0, buf0, &bar[0]);
        if (t0 + 1 < t1) issue(t0 + 1, buf0 + tile_elems, &bar[1]);
    }
    uint32_t phases = 0u;  // bit s: parity of the next completion of bar[s]
    long long failed_at = -1;
    for (long long tile = t0; tile < t1; ++tile) {
        const int s = (int)((tile - t0) & 1);
        float2* buf = buf0 + s * tile_elems;
        if (!cta_wait(&bar[s], (phases >> s) & 1u, a.wait_budget)) {
            failed_at = tile;
            break;
        }
        phases ^= 1u << s;
        const long long row0 = tile << LOGTR;
        float2 v[E];
        // c2r pre-processing: Z[k] = (X[k] + X*[M-k]) + i (X[k] - X*[M-k]) W_N^{-k}
        for_each_element<G, PI::first_radix()>(t, [&](int e, int b, int k) {
            const float2* rowp = buf + (b << LOG2M);
            float2 X = k < kz ? rowp[k] : make_float2(0.0f, 0.0f);
            float2 Xmc = make_float2(0.0f, 0.0f);
            if (k == 0) {
                X.y = 0.0f;  // the DC of a real row is real; the Nyquist term is zero
            } else if (M - k < kz) {
                Xmc = cconj(rowp[M - k]);
            }
            const float2 ep = cadd(X, Xmc);
            const float2 op = cmulc(csub(X, Xmc), tw[k]);
            v[e] = cadd(ep, cmul_i<+1>(op));
        });
        fft<G, +1, true>(v, buf, twi, t);
        if constexpr (OUTDT == kOutBatch) {
            for_each_element<G, PF::first_radix()>(t, [&](int e, int b, int j) {
                v[e] = cscale(v[e], row0 + b < a.nrows_valid ? __ldg(a.fscale + field_of(row0 + b)) : 0.0f);
            });
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = cscale(v[e], scale);
        }
        // v[e] now holds f[2j], f[2j+1] of row b at the forward plan's input positions;
        // out_pair: its index in pairs of reals in the field and map outputs
        auto out_pair = [&](int b, int j) -> long long {
            if constexpr (OUTDT == kOutBatch) {
                const long long r = row0 + b, f = field_of(r);
                return (__ldg(a.fout + f) >> 1) + ((r - (f << a.log2_rows_field)) << LOG2M) + j;
            } else {
                return (row0 + b) * M + j;
            }
        };
        // rows past the fields (the last tile of a batch) hold stale data: nothing of them is written
        auto valid = [&](int b) { return OUTDT != kOutBatch || row0 + b < a.nrows_valid; };
        if (a.out_f != nullptr) {
            for_each_element<G, PF::first_radix()>(t, [&](int e, int b, int j) {
                if (!valid(b)) return;
                const long long off = out_pair(b, j);
                if constexpr (OUTDT == kOutBF16) {
                    reinterpret_cast<__nv_bfloat162*>(a.out_f)[off] = __floats2bfloat162_rn(v[e].x, v[e].y);
                } else {
                    reinterpret_cast<float2*>(a.out_f)[off] = v[e];
                }
            });
        }
        const int nlev = ONE ? 1 : a.nlev;
        for (int lev = 0; lev < nlev; ++lev) {
            float2 u[E];
            if constexpr (OUTDT == kOutBatch) {  // one level per field
                for_each_element<G, PF::first_radix()>(t, [&](int e, int b, int j) {
                    const float th = valid(b) ? __ldg(a.flevel + field_of(row0 + b)) : 0.0f;
                    u[e] = make_float2(v[e].x >= th ? 1.0f : -1.0f, v[e].y >= th ? 1.0f : -1.0f);
                });
            } else {
                const float th = a.levels[lev];
#pragma unroll
                for (int e = 0; e < E; ++e)
                    u[e] = make_float2(v[e].x >= th ? 1.0f : -1.0f, v[e].y >= th ? 1.0f : -1.0f);
            }
            if (a.out_maps != nullptr && a.map_bits) {
                // one bit per site: sites 2 out_pair and 2 out_pair + 1 of each element
                // (one level per field in batches: lev = 0, each field's map at its fout)
                uint32_t* words = reinterpret_cast<uint32_t*>(a.out_maps) + (long long)lev * (a.N >> 5);
                if constexpr (map_bits_packed(LOG2M, LOGTR, OUTDT == kOutBatch)) {
                    // the tile's pairs stage as 2-bit bytes in buf, which the inverse FFT
                    // and the previous level's spectrum no longer read; a thread then
                    // packs 16 bytes into each word
                    unsigned char* sb = reinterpret_cast<unsigned char*>(buf);
                    __syncthreads();
                    for_each_element<G, PF::first_radix()>(t, [&](int e, int b, int j) {
                        sb[(b << LOG2M) + j] = (unsigned char)((u[e].x > 0.0f ? 1 : 0) | (u[e].y > 0.0f ? 2 : 0));
                    });
                    __syncthreads();
                    if constexpr (LOG2M >= 4) {
                        // rows of whole words: row b's M / 16 words from its first pair on
                        constexpr int kLogRowWords = LOG2M - 4;
#pragma unroll 1
                        for (int q = t; q < (G::TB << kLogRowWords); q += G::T) {
                            const int b = q >> kLogRowWords;
                            if (!valid(b)) continue;
                            const uint4 c = reinterpret_cast<const uint4*>(sb)[q];
                            words[(out_pair(b, 0) >> 4) + (q & ((1 << kLogRowWords) - 1))] =
                                pack_two_bit_bytes(c.x) | (pack_two_bit_bytes(c.y) << 8) |
                                (pack_two_bit_bytes(c.z) << 16) | (pack_two_bit_bytes(c.w) << 24);
                        }
                    } else {
                        // short rows, contiguous tile (single fields): the tile's whole words
                        uint32_t* tw_words = words + ((row0 << LOG2M) >> 4);
#pragma unroll 1
                        for (int q = t; q < tile_elems / 16; q += G::T) {
                            const uint4 c = reinterpret_cast<const uint4*>(sb)[q];
                            tw_words[q] = pack_two_bit_bytes(c.x) | (pack_two_bit_bytes(c.y) << 8) |
                                          (pack_two_bit_bytes(c.z) << 16) | (pack_two_bit_bytes(c.w) << 24);
                        }
                    }
                    // the FFT below reaches a barrier before its first write to buf
                } else {
                    // words span tiles: the caller cleared them
                    for_each_element<G, PF::first_radix()>(t, [&](int e, int b, int j) {
                        if (!valid(b)) return;
                        const long long site = 2 * out_pair(b, j);
                        const uint32_t two = (u[e].x > 0.0f ? 1u : 0u) | (u[e].y > 0.0f ? 2u : 0u);
                        if (two) atomicOr(words + (site >> 5), two << (site & 31));
                    });
                }
            } else if (a.out_maps != nullptr) {
                for_each_element<G, PF::first_radix()>(t, [&](int e, int b, int j) {
                    if (!valid(b)) return;
                    char2 m;
                    m.x = u[e].x > 0.0f ? (signed char)1 : (signed char)-1;
                    m.y = u[e].y > 0.0f ? (signed char)1 : (signed char)-1;
                    reinterpret_cast<char2*>(a.out_maps + (long long)lev * a.N)[out_pair(b, j)] = m;
                });
            }
            fft<G, -1, false>(u, buf, twf, t);
            __syncthreads();
            for_each_element<G, PF::last_radix()>(t, [&](int e, int b, int l) { buf[smem_slot<G>(l, b)] = u[e]; });
            __syncthreads();
            float2* dst = a.spec + (long long)lev * a.half;
            for_each_element<G, PF::last_radix()>(t, [&](int e, int b, int k) {
                const float2 zc = cconj(buf[smem_slot<G>((M - k) & (M - 1), b)]);
                if (valid(b)) dst[(row0 + b) * M + k] = r2c_post(u[e], zc, tw[k]);
            });
        }
        // buf is free once every thread is past its last read: refill it with tile + 2
        fence_proxy_async_smem();
        __syncthreads();
        if (t == 0 && tile + 2 < t1) issue(tile + 2, buf, &bar[s]);
    }
    if (failed_at >= 0 && t == 0) {
        atomicOr(a.status, kStatusTimeout);
        const int s = (int)((failed_at - t0) & 1);
        if (!(a.inject_skip && failed_at == t0)) mbar_wait_bounded(&bar[s], (phases >> s) & 1u, a.wait_budget);
        if (failed_at + 1 < t1) mbar_wait_bounded(&bar[s ^ 1], (phases >> (s ^ 1)) & 1u, a.wait_budget);
    }
}

// ---------------------------------------------------------------------------
// Columns: FFT along a strided axis (+ filter / bins on the last axis pass).
//
// Tiles of TB adjacent columns x L rows stream through two shared-memory
// buffers: one elected thread issues the bulk tensor loads (TMA) of tile i+2
// into the buffer tile i has just released, so the next tile is always in
// flight while the current one is transformed.  The FFT exchanges run inside
// the current tile's buffer, and the results leave by a TMA store from the
// same buffer.  Every mbarrier wait is bounded; when one runs out the CTA
// records kStatusTimeout in the workspace status word, drains its own copies
// and returns.
// ---------------------------------------------------------------------------
// The k-space noise coefficients of a tile's modes, in the layout the
// forward axis-0 FFT leaves (the inverse plan's input positions).  Mode
// (n0, col) lies in row n0 A1 + n1 (A1 = N1, n1 = col >> logM in 3D; A1 = 1,
// n1 = 0 in 2D) at k_last = col & (M - 1).  The columns 2c and 2c + 1 of a
// row share a Philox block, and they sit in lanes t and t ^ 1 with the same
// n0 in every slot: each lane draws the blocks of half of the slots and
// hands the other column's coefficient to its neighbour.  On k_last = 0 the
// mode whose mirror -n has the smaller row takes the conjugate of the
// mirror's draw, and a self-conjugate mode keeps sqrt(2) times its real part.
template <class G>
__device__ __forceinline__ void kspace_tile(float2 (&v)[G::E], const ColArgs& a, int c0, int t) {
    constexpr int E = G::E;
    constexpr int L = G::L;
    using PF = Plan<G::LOG2L, false>;
    const int col = c0 + (t & (G::TB - 1));
    const int h = col & 1;
    const int M = 1 << a.logM;
    const int n1 = col >> a.logM;
    const int klast = col & (M - 1);
    const int a1log = a.ndim == 3 ? a.log2n[1] : 0;
    const unsigned long long bpr = (unsigned long long)(M / 2 + 1);  // Philox blocks per row
    int ls[E];
    for_each_element<G, PF::last_radix()>(t, [&](int e, int b, int l) { ls[e] = l; });
    constexpr unsigned mask = G::T >= 32 ? 0xffffffffu : (1u << G::T) - 1u;
#pragma unroll
    for (int k = 0; k < E / 2; ++k) {
        const int l = h ? ls[k + E / 2] : ls[k];
        const unsigned long long row = ((unsigned long long)l << a1log) + (unsigned long long)n1;
        float2 z0, z1;
        kspace_pair(a.seed, a.field_idx, a.kscale, row * bpr + (unsigned long long)(klast >> 1), z0, z1);
        const float2 mine = h ? z1 : z0;
        const float2 other = h ? z0 : z1;
        float2 recv;
        recv.x = __shfl_xor_sync(mask, other.x, 1);
        recv.y = __shfl_xor_sync(mask, other.y, 1);
        v[k] = h ? recv : mine;
        v[k + E / 2] = h ? mine : recv;
    }
    if (klast == 0) {
        const int n1m = (-n1) & ((1 << a1log) - 1);
        unsigned need = 0;  // bit e: the mirror's row is the smaller, draw it
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int lm = (-ls[e]) & (L - 1);
            const unsigned long long row = ((unsigned long long)ls[e] << a1log) + (unsigned long long)n1;
            const unsigned long long rowm = ((unsigned long long)lm << a1log) + (unsigned long long)n1m;
            if (rowm < row) need |= 1u << e;
            if (rowm == row) v[e] = make_float2(v[e].x * 1.41421356237309505f, 0.0f);
        }
        // one copy of the draw in the code (this branch is rare): loop over the set bits
        while (need) {
            const int e = __ffs(need) - 1;
            need &= need - 1;
            const int lm = (-col_element_l<G, PF::last_radix()>(threadIdx.x, e)) & (L - 1);
            const unsigned long long rowm = ((unsigned long long)lm << a1log) + (unsigned long long)n1m;
            float2 z0, z1;
            kspace_pair(a.seed, a.field_idx, a.kscale, rowm * bpr, z0, z1);
            const float2 w = cconj(z0);
#pragma unroll
            for (int q = 0; q < E; ++q)
                if (q == e) v[q] = w;
        }
    }
}

// Layout of the power staging (see k_cols): value i of thread o at slot
// i TS + o + (o / 32) PAD.  TS = T + (T / 32) PAD + q exceeds the largest
// o-part, so the map is one-to-one, and q makes TS = 1 mod 32 (reads, i fixed
// and o running over a warp, are conflict-free for any PAD).  PAD in [0, 40)
// is the one whose write pattern has the fewest bank conflicts, simulated at
// compile time for the first warps of a tile, every element slot of the FFT's
// output layout (radix R last), 4-byte words, 32 banks.
// Where the power of tile element (b, l) is staged: thread o, value i.
// Plain order: o = (b L + l) / E, i = (b L + l) mod E (E consecutive n0 of one
// column).  Paired order (radial bins only, where n0 and -n0 share a bin): the
// column's n0 = +m and n0 = -m (m = 0 pairs with the dropped Nyquist n0 =
// -L/2) are values 2 (m mod 8) and 2 (m mod 8) + 1 of thread
// o = b L/16 + m/8, which then adds each pair before binning: half the bin
// lookups and about half the runs.
__host__ __device__ constexpr bool pairable_tile(int e, int t) { return e == 16 && t <= 256; }
__host__ __device__ constexpr int stage_o(int b, int l, int log2l, int e, bool paired) {
    if (!paired) return ((b << log2l) + l) / e;
    const int L = 1 << log2l;
    const int m = l < L / 2 ? l : (l == L / 2 ? 0 : L - l);
    return b * (L / 16) + m / 8;
}
__host__ __device__ constexpr int stage_i(int l, int log2l, int e, bool paired) {
    if (!paired) return l % e;
    const int L = 1 << log2l;
    const int m = l < L / 2 ? l : (l == L / 2 ? 0 : L - l);
    return 2 * (m % 8) + (l < L / 2 ? 0 : 1);
}

template <class G>
constexpr int staging_stride(int pad) {
    if (G::T < 32) return G::T + 1;
    const int base = G::T + (G::T / 32) * pad;
    return base + (((1 - base) % 32) + 32) % 32;
}
template <class G, int R, bool PAIRED>
constexpr int staging_cost(int pad) {
    constexpr int T = G::T, E = G::E, L = G::L;
    constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
    const int ts = staging_stride<G>(pad);
    int cost = 0;
    const int warps = T / 32 < 4 ? T / 32 : 4;
    for (int w = 0; w < warps; ++w) {
        for (int e = 0; e < E; ++e) {
            int count[32] = {};
            int worst = 0;
            for (int lane = 0; lane < 32; ++lane) {
                const int g = 32 * w + lane + T * (e >> LR);
                const int b = g & (G::TB - 1), j = g >> G::LOGTB;
                const int l = j + (e & (R - 1)) * (L / R);
                const int o = stage_o(b, l, G::LOG2L, E, PAIRED);
                const int bank = (stage_i(l, G::LOG2L, E, PAIRED) * ts + o + (o >> 5) * pad) & 31;
                worst = ++count[bank] > worst ? count[bank] : worst;
            }
            cost += worst;
        }
    }
    return cost;
}
template <class G, int R, bool PAIRED>
constexpr int staging_pad() {
    int best = 0, best_cost = staging_cost<G, R, PAIRED>(0);
    for (int pad = 1; pad < 40 && G::T >= 32; ++pad) {
        if (G::E * staging_stride<G>(pad) > 2 * G::TB * G::L) break;  // must fit the tile buffer (2 x float)
        const int c = staging_cost<G, R, PAIRED>(pad);
        if (c < best_cost) {
            best = pad;
            best_cost = c;
        }
    }
    return best;
}

// Tile buffers of a strided pass: three for the plain passes (pure
// streaming: a third tile in flight covers more of the HBM latency) where
// they fit in 220 KB with the stage tables, else two.
constexpr int col_buffers(int mode, size_t tile_bytes, size_t table_bytes) {
    return (mode == kModePlain && 3 * tile_bytes + table_bytes <= 220 * 1024) ? 3 : 2;
}

template <int LOG2L, int LOGTB, int MODE>
struct ColGeo {
    using G = Geo<LOG2L, LOGTB, false>;
    static constexpr int tile_elems = G::TB * G::L;
    static constexpr int nbuf = col_buffers(MODE, (size_t)tile_elems * 8, (size_t)plan_twiddle_slots<LOG2L>() * 8);
    // dynamic shared memory before the bins: the tile buffers, the stage twiddles, one mbarrier per buffer
    static constexpr size_t fixed_bytes =
        (size_t)nbuf * tile_elems * 8 + (size_t)plan_twiddle_slots<LOG2L>() * 8 + (size_t)nbuf * 8;
};

// PAIR: the staging of the filter and bins modes in the paired order (radial
// bins only, pairable tiles; see stage_o), chosen by the host with the bin
// table's layout.  Each layout is its own kernel: one that holds both staging
// loops needs more registers than either (the 512^3 filter pass spilled).
// ROT: the filter's norm, separable (0) or rotated (1), fixed at compile time
// for the filter and k-space modes (the host picks the kernel from the
// filter); 2 reads it from the filter at run time (batches of filters).
template <int LOG2L, int LOGTB, int MODE, int DIR, bool PAIR, int ROT>
__global__ void __launch_bounds__(Geo<LOG2L, LOGTB, false>::T, min_blocks_cols(MODE, Geo<LOG2L, LOGTB, false>::T))
    k_cols(const __grid_constant__ ColArgs a) {
    using CG = ColGeo<LOG2L, LOGTB, MODE>;
    using G = typename CG::G;
    constexpr int L = G::L;
    constexpr int E = G::E;
    constexpr int TB = G::TB;
    constexpr int T = G::T;
    constexpr int LB = L < 256 ? L : 256;  // rows per TMA box
    using PF = Plan<LOG2L, false>;
    using PI = Plan<LOG2L, true>;
    constexpr bool kAcc = MODE != kModePlain;
    constexpr bool kStore = MODE != kModeBins;
    constexpr bool kFilt = MODE == kModeFilter || MODE == kModeKspace || MODE == kModeFilterBatch;
    constexpr bool kFiltBatch = MODE == kModeFilterBatch;
    // paired staging needs 16 values per thread (L >= 16); left out of the
    // 512-thread tiles, where the second binning variant costs spills
    constexpr bool kPairable = kAcc && pairable_tile(E, T);
    static_assert(!PAIR || kPairable, "paired staging on a pairable tile of a binning mode only");
    static_assert(ROT == 2 || MODE == kModeFilter || MODE == kModeKspace, "a fixed norm for single filters only");
    constexpr bool kLoad = MODE != kModeKspace;
    static_assert(TB >= 2, "k-space mode pairs rely on two columns per tile");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int tile_elems = CG::tile_elems;
    constexpr int NBUF = CG::nbuf;
    static_assert(NBUF == 2 || kLoad, "the k-space mode's store ring assumes two buffers");
    float2* const buf0 = reinterpret_cast<float2*>(smem_raw);  // NBUF tile buffers: buf0 + s tile_elems
    float2* twf = buf0 + NBUF * tile_elems;  // stage tables: forward plan, then its reverse
    uint64_t* bar = reinterpret_cast<uint64_t*>(twf + plan_twiddle_slots<LOG2L>());
    const int nb = a.bp.nbins;
    double* dbin = reinterpret_cast<double*>(bar + NBUF);   // nb + 1 (last: Parseval)
    float* fbin = reinterpret_cast<float*>(dbin + nb + 1);  // nb + 1
    float* tab0 = fbin + nb + 1;                          // FILTER: p log2 |kappa_0 / a|, L
    const int t = threadIdx.x;
    // the filter: the call's, or (batched fields) the current batch's copy in shared memory
    __shared__ FilterParams sfp;
    const FilterParams* fpp;
    if constexpr (kFiltBatch) {
        fpp = &sfp;
    } else {
        fpp = &a.fp;
    }
    const FilterParams& fpr = *fpp;
    // the norm is rotated (not separable per axis)
    auto rotated = [&]() -> bool { return ROT == 2 ? fpr.rotated != 0 : ROT == 1; };
    // the filter's per-row terms p log2 |kappa_0 / a_0| (separable case)
    auto fill_tab0 = [&]() {
        if (!rotated()) {
            for (int l = t; l < L; l += T) {
                const float x = (float)signed_index(l, LOG2L) * __int_as_float((127 + 1 - LOG2L) << 23);
                tab0[l] = plog2_exact(fabsf(x) * fpr.inv_a[0], fpr.p);
            }
        }
    };

    long long tfirst, tstep, tcnt;
    tiles_of(a.ntiles, a.interleave, tfirst, tstep, tcnt);
    auto tile_at = [&](long long k) { return tfirst + k * tstep; };
    // run tile ti: batch ab, tile tcol of the batch in the full tile order
    // (tile counts stay below 2^31: 32-bit divisions, the second one only
    // when columns are skipped)
    auto tile_of = [&](long long ti, long long& ab, long long& tcol) {
        const unsigned q = (unsigned)ti / (unsigned)a.tpb;
        const unsigned r = (unsigned)ti - q * (unsigned)a.tpb;
        ab = q;
        if (a.live_tiles == a.row_tiles) {
            tcol = r;
        } else {
            const unsigned row = r / (unsigned)a.live_tiles;
            tcol = (long long)row * a.row_tiles + (r - row * (unsigned)a.live_tiles);
        }
    };
    constexpr uint32_t tile_bytes = (uint32_t)tile_elems * (uint32_t)sizeof(float2);
    auto issue = [&](long long ti, float2* dst, uint64_t* b) {
        long long ab, tcol;
        tile_of(ti, ab, tcol);
        const int c0 = (int)(tcol << LOGTB);
        mbar_arrive_expect_tx(b, tile_bytes);
#pragma unroll
        for (int y = 0; y < L; y += LB) tma_load_3d(dst + y * TB, &a.map, c0, y, (int)ab, b);
    };

    float2* twi = load_plan_twiddles<LOG2L>(twf, a.tw, t, T);
    if (t == 0) {
#pragma unroll
        for (int q = 0; q < NBUF; ++q) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    if constexpr (kFilt && !kFiltBatch) fill_tab0();
    if constexpr (kAcc) {
        for (int i = t; i <= nb; i += T) {
            dbin[i] = 0.0;
            fbin[i] = 0.0f;
        }
    }
    __syncthreads();
    if (kLoad && t == 0) {
        if (tcnt > 0 && !a.inject_skip) issue(tile_at(0), buf0, &bar[0]);
#pragma unroll
        for (int q = 1; q < NBUF; ++q)
            if (q < tcnt) issue(tile_at(q), buf0 + q * tile_elems, &bar[q]);
    }

    // The bins gather in FP32 (shared-memory atomics) over up to kMergeTiles
    // tiles, then in FP64: a bin takes a few dozen run sums in FP32 at most,
    // far inside the 1e-4 relative bound of the bins, and the FP64 adds (slow
    // on this part) run once per kMergeTiles tiles.  The Parseval sum goes to
    // FP64 every tile (it sets the field's normalisation).
    constexpr int kMergeTiles = 4;
    int since_merge = 0;
    auto flush = [&](long long batch) {
        __syncthreads();
        double* g = a.gbins;
        double* gp = a.gP;
        if constexpr (MODE == kModeBins) {
            g += a.boff ? a.boff[batch] : batch * nb;
        } else if constexpr (kFiltBatch) {
            g += batch * a.acc_stride;
            gp += batch * a.acc_stride;
        }
        for (int i = t; i < nb; i += T) {
            const double v = dbin[i] + (double)fbin[i];
            if (v != 0.0) atomicAdd(g + i, v);
            dbin[i] = 0.0;
            fbin[i] = 0.0f;
        }
        since_merge = 0;
        if (kFilt && t == 0) {
            atomicAdd(gp, dbin[nb]);
            dbin[nb] = 0.0;
        }
        __syncthreads();
    };

    uint32_t phases = 0u;  // bit s: parity of the next completion of bar[s]
    long long cur = -1;
    long long failed_at = -1;
    for (long long k = 0; k < tcnt; ++k) {
        const long long ti = tile_at(k);
        const int s = (int)(k % NBUF);
        float2* buf = buf0 + s * tile_elems;
        if constexpr (kLoad) {
            if (!cta_wait(&bar[s], (phases >> s) & 1u, a.wait_budget)) {
                failed_at = k;
                break;
            }
            phases ^= 1u << s;
        } else {
            // buf is free once the store of two tiles ago has read it; the
            // barrier before the first write of buf (power staging) makes
            // every thread wait for this
            if (t == 0) bulk_wait_read_1();
        }
        long long ab, tcol;
        tile_of(ti, ab, tcol);
        const long long c0 = tcol << LOGTB;
        if constexpr (MODE == kModeBins || kFiltBatch) {
            if (ab != cur) {
                if (cur >= 0) flush(cur);
                cur = ab;
                if constexpr (kFiltBatch) {
                    // the new batch's filter and its per-row terms (flush ended with a
                    // barrier, so no thread still reads the previous ones)
                    if (t == 0) sfp = a.fparr[ab];
                    __syncthreads();
                    fill_tab0();
                    __syncthreads();
                }
            }
        }
        // the bins of the E modes this thread will own after the staging
        // (tile order: element (b, l) at b L + l, thread t owns t E .. t E + E - 1),
        // loaded once the forward FFT is done so that they hold no registers through it
        uint32_t binw[E / 2 > 0 ? E / 2 : 1];
        auto load_binw = [&]() {
            if constexpr (kAcc) {
                if (nb > 0) {
                    // E entries per thread (E/2 pair bins when paired, see stage_o)
                    constexpr int per = PAIR ? E / 2 : E;
                    const unsigned short* src = a.bintab + tcol * (tile_elems / E * per) + t * per;
                    if constexpr (per == E / 2 && E >= 16) {
#pragma unroll
                        for (int q = 0; q < E / 16; ++q) {
                            const uint4 w4 = __ldg(reinterpret_cast<const uint4*>(src) + q);
                            binw[4 * q] = w4.x;
                            binw[4 * q + 1] = w4.y;
                            binw[4 * q + 2] = w4.z;
                            binw[4 * q + 3] = w4.w;
                        }
                    } else if constexpr (E >= 8) {
#pragma unroll
                        for (int q = 0; q < E / 8; ++q) {
                            const uint4 w4 = __ldg(reinterpret_cast<const uint4*>(src) + q);
                            binw[4 * q] = w4.x;
                            binw[4 * q + 1] = w4.y;
                            binw[4 * q + 2] = w4.z;
                            binw[4 * q + 3] = w4.w;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < E / 2; ++q) binw[q] = __ldg(reinterpret_cast<const uint32_t*>(src) + q);
                    }
                }
            }
        };
        float2 v[E];
        if constexpr (MODE == kModePlain && DIR > 0) {
            for_each_element<G, PI::first_radix()>(t, [&](int e, int b, int l) { v[e] = buf[(l << LOGTB) + b]; });
            fft<G, +1, true>(v, buf, twi, t);
            __syncthreads();
            for_each_element<G, PI::last_radix()>(t, [&](int e, int b, int l) { buf[(l << LOGTB) + b] = v[e]; });
        } else {
            if constexpr (MODE == kModeKspace) {
                kspace_tile<G>(v, a, (int)c0, t);
            } else {
                for_each_element<G, PF::first_radix()>(t, [&](int e, int b, int l) { v[e] = buf[(l << LOGTB) + b]; });
                fft<G, -1, false>(v, buf, twf, t);
            }
            load_binw();
            if constexpr (MODE == kModePlain) {
                __syncthreads();
                for_each_element<G, PF::last_radix()>(t, [&](int e, int b, int l) { buf[(l << LOGTB) + b] = v[e]; });
            } else {
                // A thread's column is fixed (T is a multiple of TB), and so is
                // the weight of its modes' power: 2 for the k_last > 0 half,
                // where k and -k share a half-spectrum slot.
                const int col = (int)(c0 + (t & (TB - 1)));
                const int klast = a.ndim == 3 ? (col & ((1 << a.logM) - 1)) : col;
                const float wcol = (klast == 0 ? 1.0f : 2.0f) * (MODE == kModeBins ? a.scale : 1.0f);
                [[maybe_unused]] bool nyq_col = false;
                [[maybe_unused]] float y = 0.0f, z = 0.0f, u_col = 0.0f;
                if constexpr (kFilt) {
                    int n1, n2;
                    if (a.ndim == 3) {
                        n1 = signed_index(col >> a.logM, a.log2n[1]);
                        n2 = klast;
                    } else {
                        n1 = col;
                        n2 = 0;
                    }
                    nyq_col = a.ndim == 3 && n1 == -(1 << (a.log2n[1] - 1));
                    y = (float)n1 * __int_as_float((127 + 1 - a.log2n[1]) << 23);
                    z = a.ndim == 3 ? (float)n2 * __int_as_float((127 + 1 - a.log2n[2]) << 23) : 0.0f;
                    if (!rotated()) {  // separable case: the column's terms of the sum
                        u_col = plog2_exact(fabsf(y) * fpr.inv_a[1], fpr.p);
                        if (a.ndim == 3) {
                            const float u2 = plog2_exact(fabsf(z) * fpr.inv_a[2], fpr.p);
                            const float m = fmaxf(u_col, u2);
                            u_col = m + log2f(1.0f + exp2f(fminf(u_col, u2) - m));
                        }
                    }
                }
                // The filter (Eqs. 12-13) scales each mode; its power then goes
                // through shared memory so that each thread owns E consecutive
                // n0 of one column (element (b, l) to thread o = (b L + l) / E,
                // value i = (b L + l) mod E, at slot i TS + o + (o / 32) PAD with
                // TS and PAD chosen at compile time so that the writes are
                // conflict-free; the reads, i fixed and o running over a warp,
                // always are); their bins come precomputed from the bin
                // table, and consecutive modes mostly share a bin, so one atomic
                // per run of equal bins replaces one per mode.
                constexpr int PAD0 = staging_pad<G, PF::last_radix(), false>();
                constexpr int TS0 = staging_stride<G>(PAD0);
                constexpr int PAD1 = staging_pad<G, PF::last_radix(), true>();
                constexpr int TS1 = staging_stride<G>(PAD1);
                static_assert(T - 1 + ((T - 1) >> 5) * PAD0 < TS0, "staging slots are one-to-one");
                static_assert(T - 1 + ((T - 1) >> 5) * PAD1 < TS1, "staging slots are one-to-one");
                static_assert(E * TS0 <= 2 * tile_elems && E * TS1 <= 2 * tile_elems, "staging fits the tile buffer");
                float pacc = 0.0f;
                if (nb > 0 || kFilt) {
                    float* ps = reinterpret_cast<float*>(buf);
                    __syncthreads();  // the FFT's last exchange is read
                    // Element e of the FFT's output layout sits at l = j + r L/R
                    // (r = e mod R, j < L/R), so l < L/2 exactly when r < R/2: the
                    // paired order's m and side follow from r without comparing l.
                    constexpr int R = PF::last_radix();
                    constexpr bool P = PAIR;  // radial bins only: n0 and -n0 share every bin
                    constexpr int TSP = P ? TS1 : TS0, PADP = P ? PAD1 : PAD0;
                    {
                        for_each_element<G, R>(t, [&](int e, int b, int l) {
                            const int r = e & (R - 1);    // compile-time digit
                            const int j = l - r * (L / R);  // per butterfly
                            if constexpr (kFilt) {
                                float h = 0.0f;
                                // the Nyquist row n0 = -L/2 (l = L/2: digit R/2, j = 0) has A = 0
                                const bool live = !nyq_col && !(r == R / 2 && j == 0);
                                if (!rotated()) {
                                    // log2 S >= the larger term: from u_zero on A is 0 exactly.
                                    // The warp skips the amplitude when none of its
                                    // lanes needs it (every thread of the CTA runs this loop).
                                    constexpr unsigned kWarp = T >= 32 ? 0xffffffffu : (1u << T) - 1u;
                                    const float t0 = tab0[l];
                                    const bool need = live && fmaxf(t0, u_col) < fpr.u_zero;
                                    if (__any_sync(kWarp, need)) {
                                        const float hv = amplitude_from_log2s(fpr, log2_sum2(t0, u_col));
                                        h = need ? hv : 0.0f;
                                    }
                                } else if (live) {
                                    const int n0 = r < R / 2 ? l : l - L;  // signed index of l
                                    const float x = (float)n0 * __int_as_float((127 + 1 - LOG2L) << 23);
                                    h = filter_amplitude(fpr, x, y, z, a.ndim);
                                }
                                v[e] = cscale(v[e], h);
                            }
                            const float pw = wcol * cabs2(v[e]);
                            pacc += pw;
                            int owner, slot_i;
                            float val = pw;
                            if constexpr (P) {
                                // stage_o / stage_i of the paired order
                                int m;
                                if (r < R / 2) {
                                    m = l;
                                } else if (r > R / 2) {
                                    m = (R - r) * (L / R) - j;
                                } else {
                                    // l = L/2 + j; the Nyquist n0 = -L/2 (j = 0) is dropped from
                                    // the bins: it stages as 0 next to n0 = 0
                                    m = j == 0 ? 0 : L / 2 - j;
                                    if (j == 0) val = 0.0f;
                                }
                                owner = b * (L / 16) + (m >> 3);
                                slot_i = 2 * (m & 7) + (r < R / 2 ? 0 : 1);
                            } else {
                                owner = ((b << LOG2L) + l) / E;
                                slot_i = l & (E - 1);
                            }
                            ps[slot_i * TSP + owner + (owner >> 5) * PADP] = val;
                        });
                    }
                    __syncthreads();
                    if (nb > 0) {
                        // runs of equal bins (E values, or E/2 pairs), one atomic per run
                        auto binning = [&](auto npos, auto pair) {
                            constexpr int K = decltype(npos)::value;
                            constexpr bool P = decltype(pair)::value;
                            int cur_bin = -1;
                            float acc = 0.0f;
                            constexpr int TSP = P ? TS1 : TS0, PADP = P ? PAD1 : PAD0;
#pragma unroll
                            for (int q = 0; q < K; ++q) {
                                float pw = ps[(P ? 2 * q : q) * TSP + t + (t >> 5) * PADP];
                                if constexpr (P) pw += ps[(2 * q + 1) * TSP + t + (t >> 5) * PADP];
                                const int raw = (int)((binw[q >> 1] >> (16 * (q & 1))) & 0xffffu);
                                const int bin = raw == 0xffff ? -1 : raw;
                                if (bin != cur_bin) {
                                    if (cur_bin >= 0 && acc != 0.0f) atomicAdd(fbin + cur_bin, acc);
                                    cur_bin = bin;
                                    acc = 0.0f;
                                }
                                acc += pw;
                            }
                            if (cur_bin >= 0 && acc != 0.0f) atomicAdd(fbin + cur_bin, acc);
                        };
                        binning(std::integral_constant<int, PAIR ? E / 2 : E>{}, std::bool_constant<PAIR>{});
                    }
                }
                if constexpr (kFilt) {
                    if constexpr (T >= 32) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) pacc += __shfl_xor_sync(0xffffffffu, pacc, o);
                        if ((t & 31) == 0) atomicAdd(fbin + nb, pacc);
                    } else {
                        atomicAdd(fbin + nb, pacc);
                    }
                    fft<G, +1, true>(v, buf, twi, t);
                    __syncthreads();
                    for_each_element<G, PI::last_radix()>(t, [&](int e, int b, int l) { buf[(l << LOGTB) + b] = v[e]; });
                }
            }
        }
        // the tile's results are in buf: store them, then refill buf with tile i+NBUF
        fence_proxy_async_smem();
        __syncthreads();
        if (t == 0) {
            if constexpr (kStore) {
#pragma unroll
                for (int y = 0; y < L; y += LB) tma_store_3d(&a.map, (int)c0, y, (int)ab, buf + y * TB);
                bulk_commit();
            }
            if (kLoad && k + NBUF < tcnt) {
                if constexpr (kStore) bulk_wait_read_all();
                issue(tile_at(k + NBUF), buf, &bar[s]);
            }
        }
        if constexpr (kAcc) {
            if (kFilt && t == 0) {
                dbin[nb] += (double)fbin[nb];
                fbin[nb] = 0.0f;
            }
            if (++since_merge == kMergeTiles) {
                for (int i = t; i < nb; i += T) {
                    dbin[i] += (double)fbin[i];
                    fbin[i] = 0.0f;
                }
                since_merge = 0;
            }
            // no barrier here: the next tile's first atomics on fbin come after
            // the barriers of its wait and FFT, and flush starts with one
        }
    }
    if (failed_at >= 0) {
        if (t == 0) {
            atomicOr(a.status, kStatusTimeout);
            // drain this CTA's own loads still in flight (bounded): tiles
            // failed_at .. failed_at + NBUF - 1 were issued (all but a skipped
            // first load), none of them waited for yet; then its stores
            for (int q = 0; q < NBUF && failed_at + q < tcnt; ++q) {
                if (q == 0 && a.inject_skip && failed_at == 0) continue;
                const int s = (int)((failed_at + q) % NBUF);
                mbar_wait_bounded(&bar[s], (phases >> s) & 1u, a.wait_budget);
            }
            if constexpr (kStore) bulk_wait_all();
        }
        __syncthreads();
        return;
    }
    if constexpr (kStore) {
        if (t == 0) bulk_wait_all();
    }
    if constexpr (MODE == kModeBins || kFiltBatch) {
        if (cur >= 0) flush(cur);
    } else if constexpr (kFilt) {
        flush(0);
    }
}

// ---------------------------------------------------------------------------
// Bin table: the bin of every half-spectrum mode, in the tile order of the
// axis-0 pass (tile of TB columns, element (b, l) at b L + l), 0xFFFF for
// modes with |kappa| >= 1; and the number of full-lattice modes per bin
// (weight 1 at k_last = 0, 2 elsewhere), added times `mult` to each of ndst
// count arrays.  The bins depend only on the lattice, so one table serves
// every field of a call and both binning passes.
// ---------------------------------------------------------------------------
struct TableArgs {
    unsigned short* tab;
    int paired;        // paired staging order (radial bins, L >= 16): one entry per (n0, -n0) pair
    long long nmodes;  // N / 2
    int log2l;         // axis-0 length
    int logTB;         // axis-0 tile width
    int ndim;
    int logM;
    int log2n[3];
    long long mult;
    int ndst;
    unsigned long long* dst[kMaxLevels + 1];
    BinParams bp;
};

}  // namespace hf
