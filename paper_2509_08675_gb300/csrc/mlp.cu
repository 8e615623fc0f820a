// mlp.cu -- the surrogate network's kernels and C ABI (include/hufield_surrogate.h):
// BF16 tensor-core GEMMs (mma.sync m16n8k16, FP32 accumulation) with the
// layer epilogues fused (bias + GELU on the way forward, GELU' on the way
// back), bias gradients, Adam, the losses, minibatch sampling and the
// parameter encoding.
//
// The network is small (173k parameters) and its GEMMs are at most a few
// thousand rows by 256 by 256: every launch is a few microseconds, so the
// kernels keep one simple tiling (64 x 64 CTA tiles, four warps of 32 x 32,
// K in steps of 32 staged through shared memory) and spend their effort on
// fusing the element-wise work into the GEMM epilogues.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/hufield.h"
#include "../../include/hufield_surrogate.h"
#include "common.cuh"

namespace hf {
namespace mlp {

constexpr int kLayers = 4;
constexpr int kIn = HUFIELD_MLP_IN;
constexpr int kInPad = 32;
constexpr int kHidden = 256;
constexpr int kOut = HUFIELD_MLP_OUT;
constexpr uint32_t kInitStream = 0x4D4C5031u;
constexpr uint32_t kGatherStream = 0x4D4C5032u;

__host__ __device__ constexpr int n_out(int l) { return l < kLayers - 1 ? kHidden : kOut; }
__host__ __device__ constexpr int n_in(int l) { return l == 0 ? kInPad : kHidden; }
__host__ __device__ constexpr int fan_in(int l) { return l == 0 ? kIn : kHidden; }
__host__ __device__ constexpr long long w_off(int l) {
    return l == 0 ? 0 : w_off(l - 1) + (long long)n_out(l - 1) * n_in(l - 1) + n_out(l - 1);
}
__host__ __device__ constexpr long long b_off(int l) { return w_off(l) + (long long)n_out(l) * n_in(l); }
constexpr long long kParams = b_off(kLayers - 1) + n_out(kLayers - 1);
static_assert(kParams == 172928, "parameter count");
static_assert(w_off(1) % 8 == 0 && w_off(2) % 8 == 0 && w_off(3) % 8 == 0, "16-byte aligned weight blocks");

using bf16 = __nv_bfloat16;

// Workspace: [X0 bf16 R x 32][Z_l f32 R x 256, X_l bf16 R x 256 for l = 1..3][dY bf16 R x 128][dZ bf16 2 x R x 256]
//            [split-K partial sums of a weight gradient: kSplits x 256 x 256 f32][of a bias gradient: kSplits x 256]
constexpr int kSplits = 16;
struct Ws {
    bf16* X[kLayers];  // X[0] = input, X[l] = output of hidden layer l
    float* Z[kLayers - 1];
    bf16* dY;
    bf16* dZ[2];
    float* part;
    float* part_b;
};
__host__ __device__ inline long long padded_rows(long long rows) { return (rows + 63) / 64 * 64; }
inline size_t ws_bytes_for(long long rows) {
    const long long R = padded_rows(rows);
    return (size_t)R * (kInPad * 2 + 3 * (kHidden * 4 + kHidden * 2) + kOut * 2 + 2 * kHidden * 2) +
           (size_t)kSplits * (kHidden * kHidden + kHidden) * 4;
}
inline Ws carve(void* ws, long long rows) {
    const long long R = padded_rows(rows);
    char* p = static_cast<char*>(ws);
    Ws w;
    w.X[0] = reinterpret_cast<bf16*>(p);
    p += R * kInPad * 2;
    for (int l = 0; l < kLayers - 1; ++l) {
        w.Z[l] = reinterpret_cast<float*>(p);
        p += R * kHidden * 4;
        w.X[l + 1] = reinterpret_cast<bf16*>(p);
        p += R * kHidden * 2;
    }
    w.dY = reinterpret_cast<bf16*>(p);
    p += R * kOut * 2;
    w.dZ[0] = reinterpret_cast<bf16*>(p);
    p += R * kHidden * 2;
    w.dZ[1] = reinterpret_cast<bf16*>(p);
    p += R * kHidden * 2;
    w.part = reinterpret_cast<float*>(p);
    p += (size_t)kSplits * kHidden * kHidden * 4;
    w.part_b = reinterpret_cast<float*>(p);
    return w;
}

// GELU(z) = z Phi(z) and its derivative Phi(z) + z phi(z) (CUDA's erff / expf).
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ---------------------------------------------------------------------------
// GEMM C[M x N] = op(A)[M x K] op(B)[K x N], BF16 operands, FP32 accumulation.
// AKM: A stored [K][M] (else [M][K]); BKN: B stored [K][N] (else [N][K]).
// M and K are multiples of 64 and 32; N a multiple of 8 (columns >= N are
// zero-filled on load and not stored).
// ---------------------------------------------------------------------------
// kEpiPartial: split K over gridDim.z; slice z stores its partial product at
// outf + z M N (row-major M x N), summed in a fixed order by k_reduce_splits.
enum Epi { kEpiHidden = 0, kEpiOut = 1, kEpiGeluBack = 2, kEpiStore = 3, kEpiPartial = 4 };

struct GemmArgs {
    const bf16* A;
    int lda;
    const bf16* B;
    int ldb;
    int M, N, K;
    const float* bias;  // kEpiHidden, kEpiOut
    float* outf;        // kEpiHidden: Z; kEpiOut, kEpiStore: result
    int ldo;
    bf16* outb;         // kEpiHidden: GELU(Z); kEpiGeluBack: dZ
    int ldb_out;
    const float* zin;   // kEpiGeluBack: Z of the layer below
    int ldz;
    int rows_valid;     // kEpiOut, kEpiStore: rows >= this are not stored
    int cols_valid;     // kEpiStore: columns >= this are not stored
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kBM = 64, kBN = 64, kBK = 32, kPadE = 8;
// K chunks in flight: chunk k + kStages - 1 loads (cp.async) while chunk k is multiplied
constexpr int kStages = 4;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
    // 16 bytes global -> shared, bypassing L1; zero-filled (nothing read) when !valid
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
                 "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <int AKM, int BKN, int EPI>
__global__ void __launch_bounds__(128) k_gemm(const GemmArgs g) {
    constexpr int AR = AKM ? kBK : kBM, AC = (AKM ? kBM : kBK) + kPadE;
    constexpr int BR = BKN ? kBK : kBN, BC = (BKN ? kBN : kBK) + kPadE;
    __shared__ __align__(16) bf16 As[kStages][AR][AC];
    __shared__ __align__(16) bf16 Bs[kStages][BR][BC];
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int q = lane >> 3, r8 = lane & 7;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;

    const int kslice = g.K / gridDim.z;
    const int kbeg = blockIdx.z * kslice;
    const int nk = kslice / kBK;
    // chunk c of this CTA's K slice into stage st: 64 x 32 tiles, 256 pieces of
    // 8 BF16 (16 bytes), two per thread; B columns >= N are zero-filled
    auto load = [&](int c, int st) {
        const int k0 = kbeg + c * kBK;
#pragma unroll
        for (int i = t; i < 256; i += 128) {
            if constexpr (!AKM) {
                const int r = i >> 2, cc = (i & 3) * 8;
                cp_async16(&As[st][r][cc], g.A + (size_t)(m0 + r) * g.lda + k0 + cc, true);
            } else {
                const int r = i >> 3, cc = (i & 7) * 8;
                cp_async16(&As[st][r][cc], g.A + (size_t)(k0 + r) * g.lda + m0 + cc, true);
            }
            if constexpr (!BKN) {
                const int r = i >> 2, cc = (i & 3) * 8;
                const bool ok = n0 + r < g.N;
                cp_async16(&Bs[st][r][cc], ok ? g.B + (size_t)(n0 + r) * g.ldb + k0 + cc : g.B, ok);
            } else {
                const int r = i >> 3, cc = (i & 7) * 8;
                const bool ok = n0 + cc < g.N;
                cp_async16(&Bs[st][r][cc], ok ? g.B + (size_t)(k0 + r) * g.ldb + n0 + cc : g.B, ok);
            }
        }
    };
#pragma unroll
    for (int c = 0; c < kStages - 1; ++c) {
        if (c < nk) load(c, c);
        cp_async_commit();  // one group per chunk, empty past the slice, so the counts stay uniform
    }
    for (int c = 0; c < nk; ++c) {
        cp_async_wait<kStages - 2>();  // chunk c has landed (this thread's part)
        __syncthreads();               // ... every thread's; and stage (c - 1) % kStages is free
        if (c + kStages - 1 < nk) load(c + kStages - 1, (c + kStages - 1) % kStages);
        cp_async_commit();
        const int st = c % kStages;
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int mb = wm + mi * 16;
                if constexpr (!AKM) {
                    // matrices (rows 0-7 | 8-15) x (k 0-7 | 8-15): lane gives row lane & 15, k (lane >> 4) 8
                    ldsm_x4(a[mi], &As[st][mb + (lane & 15)][kk + (lane >> 4) * 8]);
                } else {
                    // stored [k][m]: transposed 8x8 blocks (k 0-7, m 0-7), (k 0-7, m 8-15), (k 8-15, m 0-7), ...
                    ldsm_x4_t(a[mi], &As[st][kk + ((q >> 1) << 3) + r8][mb + ((q & 1) << 3)]);
                }
            }
#pragma unroll
            for (int nj = 0; nj < 2; ++nj) {
                const int nb = wn + nj * 16;
                uint32_t r[4];
                if constexpr (!BKN) {
                    // stored [n][k]: (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
                    ldsm_x4(r, &Bs[st][nb + ((q >> 1) << 3) + r8][kk + ((q & 1) << 3)]);
                } else {
                    // stored [k][n]: transposed (k 0-7, n 0-7), (k 8-15, n 0-7), (k 0-7, n 8-15), (k 8-15, n 8-15)
                    ldsm_x4_t(r, &Bs[st][kk + ((q & 1) << 3) + r8][nb + ((q >> 1) << 3)]);
                }
                b[2 * nj][0] = r[0];
                b[2 * nj][1] = r[1];
                b[2 * nj + 1][0] = r[2];
                b[2 * nj + 1][1] = r[3];
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni][0], b[ni][1]);
        }
    }
    cp_async_wait<0>();

    // epilogue: accumulator (mi, ni, e) is row wm + 16 mi + (lane >> 2) + 8 (e >> 1),
    // column wn + 8 ni + 2 (lane & 3) + (e & 1)
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = m0 + wm + mi * 16 + (lane >> 2) + 8 * h;
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int n = n0 + wn + ni * 8 + 2 * (lane & 3);
                if (n >= g.N) continue;
                float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
                if constexpr (EPI == kEpiHidden) {
                    v0 += g.bias[n];
                    v1 += g.bias[n + 1];
                    *reinterpret_cast<float2*>(g.outf + (size_t)m * g.ldo + n) = make_float2(v0, v1);
                    *reinterpret_cast<__nv_bfloat162*>(g.outb + (size_t)m * g.ldb_out + n) =
                        __floats2bfloat162_rn(gelu(v0), gelu(v1));
                } else if constexpr (EPI == kEpiOut) {
                    if (m < g.rows_valid)
                        *reinterpret_cast<float2*>(g.outf + (size_t)m * g.ldo + n) =
                            make_float2(v0 + g.bias[n], v1 + g.bias[n + 1]);
                } else if constexpr (EPI == kEpiGeluBack) {
                    const float2 z = *reinterpret_cast<const float2*>(g.zin + (size_t)m * g.ldz + n);
                    *reinterpret_cast<__nv_bfloat162*>(g.outb + (size_t)m * g.ldb_out + n) =
                        __floats2bfloat162_rn(v0 * gelu_grad(z.x), v1 * gelu_grad(z.y));
                } else if constexpr (EPI == kEpiPartial) {
                    *reinterpret_cast<float2*>(g.outf + (size_t)blockIdx.z * g.M * g.N + (size_t)m * g.N + n) =
                        make_float2(v0, v1);
                } else {
                    if (m < g.rows_valid) {
                        if (n < g.cols_valid) g.outf[(size_t)m * g.ldo + n] = v0;
                        if (n + 1 < g.cols_valid) g.outf[(size_t)m * g.ldo + n + 1] = v1;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Element-wise kernels.
// ---------------------------------------------------------------------------
__global__ void k_init(float* p, unsigned long long seed) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    int l = 0;
    while (l + 1 < kLayers && i >= w_off(l + 1)) ++l;
    float w = 0.0f;
    const long long rel = i - w_off(l);
    if (i < b_off(l) && (int)(rel % n_in(l)) < fan_in(l)) {
        const unsigned long long j = (unsigned long long)i >> 2;
        const uint4 x = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)(j >> 32), kInitStream, 0u), (uint32_t)seed,
                                      (uint32_t)(seed >> 32));
        const uint32_t word = (i & 3) == 0 ? x.x : (i & 3) == 1 ? x.y : (i & 3) == 2 ? x.z : x.w;
        const float u = fmaf(__uint2float_rn(word), 0x1p-32f, 0x1p-33f);
        w = (2.0f * u - 1.0f) * (1.0f / sqrtf((float)fan_in(l)));
    }
    p[i] = w;
}

__global__ void k_cast(const float* p, bf16* q, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = __float2bfloat16_rn(p[i]);
}

__global__ void k_encode(const float* th, long long rows, float* x) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const float* t = th + i * kIn;
    float* o = x + i * kIn;
    o[0] = (t[0] - 4.5f) / 3.5f;
    o[1] = log2f(t[1]);
    o[2] = log2f(t[2]);
    o[3] = 2.0f * t[3] / 3.14159265358979324f - 1.0f;
    o[4] = (t[4] - 0.225f) / 0.175f;
    o[5] = (t[5] - 0.055f) / 0.045f;
    o[6] = (t[6] - 4.0f) / 2.0f;
    o[7] = t[7];
}

__global__ void k_decode(const float* x, long long rows, float* th) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const float* v = x + i * kIn;
    float* o = th + i * kIn;
    o[0] = 4.5f + 3.5f * v[0];
    o[1] = exp2f(v[1]);
    o[2] = exp2f(v[2]);
    o[3] = 0.5f * 3.14159265358979324f * (v[3] + 1.0f);
    o[4] = 0.225f + 0.175f * v[4];
    o[5] = 0.055f + 0.045f * v[5];
    o[6] = 4.0f + 2.0f * v[6];
    o[7] = v[7];
}

// X0 = bf16(x) in 32 columns (zero beyond 8 and in the padding rows).
__global__ void k_input(const float* x, long long rows, long long R, bf16* X0) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * kInPad) return;
    const long long r = i / kInPad;
    const int c = (int)(i % kInPad);
    X0[i] = __float2bfloat16_rn(r < rows && c < kIn ? x[r * kIn + c] : 0.0f);
}

// dY = bf16(dy), zero in the padding rows.
__global__ void k_dy(const float* dy, long long rows, long long R, bf16* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * kOut) return;
    out[i] = __float2bfloat16_rn(i < rows * kOut ? dy[i] : 0.0f);
}

// out[i] = sum over z < splits of part[z n + i], in order of z.
__global__ void k_reduce_splits(const float* part, int splits, long long n, float* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += part[(long long)z * n + i];
    out[i] = s;
}

// Partial column sums of dZ [R][ncol] over the row slice z (grid.y = slices).
__global__ void k_colsum_part(const bf16* dZ, long long R, int ncol, float* part) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= ncol) return;
    const long long rs = R / gridDim.y, r0 = blockIdx.y * rs;
    float s = 0.0f;
    for (long long r = r0; r < r0 + rs; ++r) s += __bfloat162float(dZ[r * ncol + n]);
    part[(long long)blockIdx.y * ncol + n] = s;
}

__global__ void k_adam(float* p, float* m, float* v, const float* g, bf16* q, long long n, float lr, float b1,
                       float b2, float eps, float wd, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
    p[i] = pi;
    if (q) q[i] = __float2bfloat16_rn(pi);
}

// Block reduction of a double into one atomic add.
__device__ __forceinline__ void block_add(double v, double* dst) {
    __shared__ double part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(dst, v);
    }
}

__global__ void k_deviance(const float* yh, const float* S, const float* mu, const float* sg, long long rows,
                           float* dy, double* loss) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < rows * kOut) {
        const int b = (int)(i % kOut);
        const float y = fmaf(sg[b], yh[i], mu[b]);
        const float e = expf(-fminf(fmaxf(y, -30.0f), 30.0f));
        const float s = S[i];
        l = (double)y + (double)s * (double)e;
        dy[i] = sg[b] * (1.0f - s * e) / (float)(rows * kOut);
    }
    block_add(l, loss);
}

// One block per bin: mean and standard deviation of log(S + 1e-3) over n rows.
__global__ void k_label_stats(const float* S, long long n, float* mu, float* sg) {
    const int b = blockIdx.x;
    double s1 = 0.0, s2 = 0.0;
    for (long long r = threadIdx.x; r < n; r += blockDim.x) {
        const double v = log((double)S[r * kOut + b] + 1e-3);
        s1 += v;
        s2 += v * v;
    }
    __shared__ double a1[256], a2[256];
    a1[threadIdx.x] = s1;
    a2[threadIdx.x] = s2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            a1[threadIdx.x] += a1[threadIdx.x + o];
            a2[threadIdx.x] += a2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = a1[0] / (double)n;
        const double var = fmax(a2[0] / (double)n - m * m, 0.0);
        mu[b] = (float)m;
        sg[b] = (float)fmax(sqrt(var), 0.05);
    }
}

__global__ void k_spectrum(const float* yh, const float* mu, const float* sg, long long rows, float* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * kOut) return;
    const int b = (int)(i % kOut);
    out[i] = expf(fminf(fmaxf(fmaf(sg[b], yh[i], mu[b]), -30.0f), 30.0f));
}

__global__ void k_labels(const double* sums, const long long* counts, long long n, float* S) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n * kOut) S[i] = counts[i] ? (float)(sums[i] / (double)counts[i]) : 0.0f;
}

__global__ void k_gather(const float* xa, const float* Sa, long long n, long long rows, unsigned long long seed,
                         unsigned long long step, float* xo, float* So) {
    const long long r = blockIdx.x;
    if (r >= rows) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)r, (uint32_t)step, (uint32_t)(step >> 32), kGatherStream),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const long long idx = (long long)(w.x % (unsigned long long)n);
    for (int c = threadIdx.x; c < kOut; c += blockDim.x) So[r * kOut + c] = Sa[idx * kOut + c];
    if (threadIdx.x < kIn) xo[r * kIn + threadIdx.x] = xa[idx * kIn + threadIdx.x];
}

// Training-step variants that read the step counter from device memory, so a
// CUDA graph of many steps replays with the schedule advancing on the device.
struct Sched {
    float lr, lr_min_frac, b1, b2, eps, wd;
    long long total;
};

__global__ void k_gather_dev(const float* xa, const float* Sa, long long n, long long rows, unsigned long long seed,
                             const long long* step, float* xo, float* So) {
    const long long r = blockIdx.x;
    if (r >= rows) return;
    const unsigned long long s = (unsigned long long)*step;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)r, (uint32_t)s, (uint32_t)(s >> 32), kGatherStream),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const long long idx = (long long)(w.x % (unsigned long long)n);
    for (int c = threadIdx.x; c < kOut; c += blockDim.x) So[r * kOut + c] = Sa[idx * kOut + c];
    if (threadIdx.x < kIn) xo[r * kIn + threadIdx.x] = xa[idx * kIn + threadIdx.x];
}

// Adam at step t = counter + 1 with the learning rate of a half cosine from lr
// to lr * lr_min_frac over `total` steps.
__global__ void k_adam_sched(float* p, float* m, float* v, const float* g, bf16* q, long long n, const Sched sc,
                             const long long* step) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // per-step scalars in FP32 (FP64 is a slow path on this part); the same in every thread
    const long long s = *step;
    const float frac = (float)s / (float)sc.total;
    const float lr = sc.lr * (sc.lr_min_frac + (1.0f - sc.lr_min_frac) * 0.5f * (1.0f + cospif(frac)));
    const float t = (float)(s + 1);
    const float c1 = 1.0f - powf(sc.b1, t);
    const float c2 = 1.0f - powf(sc.b2, t);
    const float gi = g[i];
    const float mi = sc.b1 * m[i] + (1.0f - sc.b1) * gi;
    const float vi = sc.b2 * v[i] + (1.0f - sc.b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + sc.eps) + sc.wd * p[i]);
    p[i] = pi;
    if (q) q[i] = __float2bfloat16_rn(pi);
}

__global__ void k_step_set(long long* step, long long value) { *step = value; }
__global__ void k_step_advance(long long* step) { *step += 1; }

// One warp per row: the design loss and its gradient (4 bins per lane).
__global__ void k_design_loss(const float* yh, const float* T, const float* mu, const float* sg, long long rows,
                              float lam, float* dy, float* loss) {
    const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    float y[4], ey[4], tb[4];
    float den = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int b = lane + 32 * k;
        y[k] = fmaf(sg[b], yh[r * kOut + b], mu[b]);
        ey[k] = expf(fminf(fmaxf(y[k], -30.0f), 30.0f));
        tb[k] = T[r * kOut + b];
        if (b >= 1) den += tb[k] * tb[k];
    }
    for (int o = 16; o > 0; o >>= 1) den += __shfl_xor_sync(0xffffffffu, den, o);
    float l = 0.0f;
    const float inv_nb = 1.0f / (float)(kOut - 1);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int b = lane + 32 * k;
        float g = 0.0f;
        if (b >= 1) {
            const float d = ey[k] - tb[k];
            const float dl = y[k] - logf(tb[k]);
            l += d * d / den + lam * dl * dl * inv_nb;
            g = (2.0f * d * ey[k] / den + 2.0f * lam * dl * inv_nb) * sg[b];
        }
        dy[r * kOut + b] = g;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0 && loss) loss[r] = l;
}

__global__ void k_design_step(float* x, float* m, float* v, const float* dx, long long rows, unsigned frozen, float lr,
                              float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * kIn) return;
    if ((frozen >> (i % kIn)) & 1u) return;
    const float g = dx[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    x[i] = fminf(1.0f, fmaxf(-1.0f, x[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f)));
}

template <int AKM, int BKN, int EPI>
cudaError_t gemm(const GemmArgs& g, cudaStream_t s, int splits = 1) {
    const dim3 grid((g.N + kBN - 1) / kBN, g.M / kBM, splits);
    k_gemm<AKM, BKN, EPI><<<grid, 128, 0, s>>>(g);
    return cudaGetLastError();
}

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace mlp
}  // namespace hf

using namespace hf::mlp;

#define HF_MLP_CUDA(expr)                                    \
    do {                                                     \
        if ((expr) != cudaSuccess) return HUFIELD_ERR_CUDA;  \
    } while (0)

extern "C" {

int64_t hufield_mlp_param_count(void) { return kParams; }

size_t hufield_mlp_workspace_bytes(int64_t rows) { return rows < 1 ? 0 : ws_bytes_for(rows); }

int hufield_mlp_init(float* params, uint64_t seed, void* stream) {
    if (!params || !aligned16(params)) return HUFIELD_ERR_INVALID_ARG;
    k_init<<<blocks(kParams, 256), 256, 0, (cudaStream_t)stream>>>(params, seed);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_cast(const float* params, uint16_t* wq, void* stream) {
    if (!params || !wq || !aligned16(params) || !aligned16(wq)) return HUFIELD_ERR_INVALID_ARG;
    k_cast<<<blocks(kParams, 256), 256, 0, (cudaStream_t)stream>>>(params, reinterpret_cast<bf16*>(wq), kParams);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_encode(const float* theta, int64_t rows, float* x, void* stream) {
    if (!theta || !x || rows < 1) return HUFIELD_ERR_INVALID_ARG;
    k_encode<<<blocks(rows, 256), 256, 0, (cudaStream_t)stream>>>(theta, rows, x);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_decode(const float* x, int64_t rows, float* theta, void* stream) {
    if (!theta || !x || rows < 1) return HUFIELD_ERR_INVALID_ARG;
    k_decode<<<blocks(rows, 256), 256, 0, (cudaStream_t)stream>>>(x, rows, theta);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_forward(const float* params, const uint16_t* wq_raw, const float* x, int64_t rows, float* y, void* ws,
                        size_t ws_bytes, void* stream) {
    if (!params || !wq_raw || !x || !y || !ws || rows < 1 || rows > (1ll << 24)) return HUFIELD_ERR_INVALID_ARG;
    if (!aligned16(params) || !aligned16(wq_raw) || !aligned16(ws) || !aligned16(y)) return HUFIELD_ERR_INVALID_ARG;
    if (ws_bytes < ws_bytes_for(rows)) return HUFIELD_ERR_WS_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    const bf16* wq = reinterpret_cast<const bf16*>(wq_raw);
    const long long R = padded_rows(rows);
    Ws w = carve(ws, rows);
    k_input<<<blocks(R * kInPad, 256), 256, 0, s>>>(x, rows, R, w.X[0]);
    HF_MLP_CUDA(cudaGetLastError());
    for (int l = 0; l < kLayers; ++l) {
        GemmArgs g{};
        g.A = w.X[l];
        g.lda = n_in(l);
        g.B = wq + w_off(l);
        g.ldb = n_in(l);
        g.M = (int)R;
        g.N = n_out(l);
        g.K = n_in(l);
        g.bias = params + b_off(l);
        if (l + 1 < kLayers) {
            g.outf = w.Z[l];
            g.ldo = kHidden;
            g.outb = w.X[l + 1];
            g.ldb_out = kHidden;
            HF_MLP_CUDA((gemm<0, 0, kEpiHidden>(g, s)));
        } else {
            g.outf = y;
            g.ldo = kOut;
            g.rows_valid = (int)rows;
            HF_MLP_CUDA((gemm<0, 0, kEpiOut>(g, s)));
        }
    }
    return HUFIELD_OK;
}

int hufield_mlp_backward(const float* params, const uint16_t* wq_raw, const float* dy, int64_t rows, float* grad,
                         float* dx, void* ws, size_t ws_bytes, void* stream) {
    if (!params || !wq_raw || !dy || !ws || rows < 1 || rows > (1ll << 24) || (!grad && !dx))
        return HUFIELD_ERR_INVALID_ARG;
    if (!aligned16(wq_raw) || !aligned16(ws) || (grad && !aligned16(grad))) return HUFIELD_ERR_INVALID_ARG;
    if (ws_bytes < ws_bytes_for(rows)) return HUFIELD_ERR_WS_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    const bf16* wq = reinterpret_cast<const bf16*>(wq_raw);
    const long long R = padded_rows(rows);
    Ws w = carve(ws, rows);
    k_dy<<<blocks(R * kOut, 256), 256, 0, s>>>(dy, rows, R, w.dY);
    HF_MLP_CUDA(cudaGetLastError());
    const bf16* dz = w.dY;  // dZ of layer l, [R][n_out(l)]
    int cur = 0;
    for (int l = kLayers - 1; l >= 0; --l) {
        if (grad) {
            // dW_l = dZ_l^T X_{l-1}: A stored [R][n_out] = [K][M], B stored [R][n_in] = [K][N].
            // K = R is long and M x N small: the rows are split over `splits` CTAs per
            // tile, whose partial products are then summed in a fixed order (the
            // result does not depend on the schedule)
            const int splits = (int)std::min<long long>(kSplits, R / 64);
            GemmArgs g{};
            g.A = dz;
            g.lda = n_out(l);
            g.B = w.X[l];
            g.ldb = n_in(l);
            g.M = n_out(l);
            g.N = n_in(l);
            g.K = (int)R;
            g.outf = w.part;
            HF_MLP_CUDA((gemm<1, 1, kEpiPartial>(g, s, splits)));
            const long long mn = (long long)n_out(l) * n_in(l);
            k_reduce_splits<<<blocks(mn, 256), 256, 0, s>>>(w.part, splits, mn, grad + w_off(l));
            HF_MLP_CUDA(cudaGetLastError());
            k_colsum_part<<<dim3(blocks(n_out(l), 128), splits), 128, 0, s>>>(dz, R, n_out(l), w.part_b);
            HF_MLP_CUDA(cudaGetLastError());
            k_reduce_splits<<<blocks(n_out(l), 256), 256, 0, s>>>(w.part_b, splits, n_out(l), grad + b_off(l));
            HF_MLP_CUDA(cudaGetLastError());
        }
        // dA = dZ_l W_l: A stored [R][n_out] = [M][K], B = W_l stored [n_out][n_in] = [K][N]
        GemmArgs g{};
        g.A = dz;
        g.lda = n_out(l);
        g.B = wq + w_off(l);
        g.ldb = n_in(l);
        g.M = (int)R;
        g.N = n_in(l);
        g.K = n_out(l);
        if (l > 0) {
            g.zin = w.Z[l - 1];
            g.ldz = kHidden;
            g.outb = w.dZ[cur];
            g.ldb_out = kHidden;
            HF_MLP_CUDA((gemm<0, 1, kEpiGeluBack>(g, s)));
            dz = w.dZ[cur];
            cur ^= 1;
        } else if (dx) {
            g.outf = dx;
            g.ldo = kIn;
            g.rows_valid = (int)rows;
            g.cols_valid = kIn;
            HF_MLP_CUDA((gemm<0, 1, kEpiStore>(g, s)));
        }
    }
    return HUFIELD_OK;
}

int hufield_mlp_deviance(const float* y_hat, const float* S, const float* mu, const float* sigma, int64_t rows,
                         float* dy, double* loss_sum, void* stream) {
    if (!y_hat || !S || !mu || !sigma || !dy || !loss_sum || rows < 1) return HUFIELD_ERR_INVALID_ARG;
    k_deviance<<<blocks(rows * kOut, 256), 256, 0, (cudaStream_t)stream>>>(y_hat, S, mu, sigma, rows, dy, loss_sum);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_label_stats(const float* S, int64_t n, float* mu, float* sigma, void* stream) {
    if (!S || !mu || !sigma || n < 1) return HUFIELD_ERR_INVALID_ARG;
    k_label_stats<<<kOut, 256, 0, (cudaStream_t)stream>>>(S, n, mu, sigma);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_spectrum(const float* y_hat, const float* mu, const float* sigma, int64_t rows, float* S,
                         void* stream) {
    if (!y_hat || !mu || !sigma || !S || rows < 1) return HUFIELD_ERR_INVALID_ARG;
    k_spectrum<<<blocks(rows * kOut, 256), 256, 0, (cudaStream_t)stream>>>(y_hat, mu, sigma, rows, S);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_labels(const double* sums, const int64_t* counts, int64_t n, float* S, void* stream) {
    if (!sums || !counts || !S || n < 1) return HUFIELD_ERR_INVALID_ARG;
    k_labels<<<blocks(n * kOut, 256), 256, 0, (cudaStream_t)stream>>>(
        sums, reinterpret_cast<const long long*>(counts), n, S);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_adam(float* params, float* m, float* v, const float* grad, uint16_t* wq, int64_t n, int32_t step,
                     float lr, float beta1, float beta2, float eps, float wd, void* stream) {
    if (!params || !m || !v || !grad || n < 1 || step < 1) return HUFIELD_ERR_INVALID_ARG;
    if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return HUFIELD_ERR_INVALID_ARG;
    const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
    const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
    k_adam<<<blocks(n, 256), 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, reinterpret_cast<bf16*>(wq), n, lr,
                                                             beta1, beta2, eps, wd, c1, c2);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

// Training workspace: [256 B: step counter][xb R x 8][Sb R x 128][y R x 128][dy R x 128][forward workspace]
static size_t train_ws_bytes(long long rows) {
    const long long R = padded_rows(rows);
    return 256 + (size_t)R * 4 * (kIn + 3 * kOut) + ws_bytes_for(rows);
}

size_t hufield_mlp_train_workspace_bytes(int64_t rows) { return rows < 1 ? 0 : train_ws_bytes(rows); }

int hufield_mlp_train_reset(void* tws, int64_t step, void* stream) {
    if (!tws || !aligned16(tws) || step < 0) return HUFIELD_ERR_INVALID_ARG;
    k_step_set<<<1, 1, 0, (cudaStream_t)stream>>>(reinterpret_cast<long long*>(tws), step);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_train_step(float* params, uint16_t* wq, float* m, float* v, float* grad, const float* x_all,
                           const float* S_all, int64_t n, int64_t rows, const float* mu, const float* sigma,
                           const hufield_mlp_sched* sched, double* loss_sum, void* tws, size_t tws_bytes,
                           void* stream) {
    if (!params || !wq || !m || !v || !grad || !x_all || !S_all || !mu || !sigma || !sched || !loss_sum || !tws)
        return HUFIELD_ERR_INVALID_ARG;
    if (n < 1 || rows < 1 || rows > (1ll << 24) || !aligned16(tws) || !aligned16(params) || !aligned16(wq))
        return HUFIELD_ERR_INVALID_ARG;
    if (!(sched->lr >= 0.0f) || !(sched->lr_min_frac >= 0.0f) || !(sched->beta1 >= 0.0f && sched->beta1 < 1.0f) ||
        !(sched->beta2 >= 0.0f && sched->beta2 < 1.0f) || !(sched->eps > 0.0f) || sched->total_steps < 1)
        return HUFIELD_ERR_INVALID_ARG;
    if (tws_bytes < train_ws_bytes(rows)) return HUFIELD_ERR_WS_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    const long long R = padded_rows(rows);
    long long* step = reinterpret_cast<long long*>(tws);
    float* xb = reinterpret_cast<float*>(static_cast<char*>(tws) + 256);
    float* Sb = xb + R * kIn;
    float* y = Sb + R * kOut;
    float* dy = y + R * kOut;
    void* fws = dy + R * kOut;
    const size_t fws_bytes = ws_bytes_for(rows);
    k_gather_dev<<<(unsigned)rows, 128, 0, s>>>(x_all, S_all, n, rows, sched->seed, step, xb, Sb);
    HF_MLP_CUDA(cudaGetLastError());
    int rc = hufield_mlp_forward(params, wq, xb, rows, y, fws, fws_bytes, stream);
    if (rc) return rc;
    rc = hufield_mlp_deviance(y, Sb, mu, sigma, rows, dy, loss_sum, stream);
    if (rc) return rc;
    rc = hufield_mlp_backward(params, wq, dy, rows, grad, nullptr, fws, fws_bytes, stream);
    if (rc) return rc;
    const Sched sc{sched->lr, sched->lr_min_frac, sched->beta1, sched->beta2, sched->eps, sched->wd,
                   (long long)sched->total_steps};
    k_adam_sched<<<blocks(kParams, 256), 256, 0, s>>>(params, m, v, grad, reinterpret_cast<bf16*>(wq), kParams, sc,
                                                      step);
    HF_MLP_CUDA(cudaGetLastError());
    k_step_advance<<<1, 1, 0, s>>>(step);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_gather(const float* x_all, const float* S_all, int64_t n, int64_t rows, uint64_t seed, int64_t step,
                       float* x_out, float* S_out, void* stream) {
    if (!x_all || !S_all || !x_out || !S_out || n < 1 || rows < 1 || rows > (1ll << 31)) return HUFIELD_ERR_INVALID_ARG;
    k_gather<<<(unsigned)rows, 128, 0, (cudaStream_t)stream>>>(x_all, S_all, n, rows, seed,
                                                               (unsigned long long)step, x_out, S_out);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_design_loss(const float* y_hat, const float* T, const float* mu, const float* sigma, int64_t rows,
                            float lam, float* dy, float* loss_rows, void* stream) {
    if (!y_hat || !T || !mu || !sigma || !dy || rows < 1 || !(lam >= 0.0f)) return HUFIELD_ERR_INVALID_ARG;
    k_design_loss<<<blocks(rows, 8), 256, 0, (cudaStream_t)stream>>>(y_hat, T, mu, sigma, rows, lam, dy, loss_rows);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

int hufield_mlp_design_step(float* x, float* m, float* v, const float* dx, int64_t rows, uint32_t frozen_mask,
                            int32_t step, float lr, void* stream) {
    if (!x || !m || !v || !dx || rows < 1 || step < 1 || !(lr >= 0.0f)) return HUFIELD_ERR_INVALID_ARG;
    const float c1 = (float)(1.0 - pow(0.9, (double)step));
    const float c2 = (float)(1.0 - pow(0.999, (double)step));
    k_design_step<<<blocks(rows * kIn, 256), 256, 0, (cudaStream_t)stream>>>(x, m, v, dx, rows, frozen_mask, lr, c1,
                                                                             c2);
    HF_MLP_CUDA(cudaGetLastError());
    return HUFIELD_OK;
}

}  // extern "C"
