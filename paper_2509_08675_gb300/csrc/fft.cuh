// fft.cuh -- in-CTA FFT engine for power-of-two lengths L <= 4096.
//
// Each CTA transforms TB independent lines of length L.  A thread holds E
// complex values in registers; a stage of radix R makes every thread run E/R
// radix-R butterflies in registers, and between stages the values are
// exchanged through shared memory (Stockham autosort: natural order in and
// out, no bit reversal).  Stage s with radix R, after sub-transforms of size
// Ns have been formed, takes butterfly j's inputs at j + r L/R, multiplies
// input r by W_{Ns R}^{(j mod Ns) r}, and writes output r at
// (j / Ns) Ns R + (j mod Ns) + r Ns.
//
// The geometry (line length, lines per CTA, threads) is a compile-time
// context, so every shared-memory address reduces to a per-thread base plus
// an immediate offset.  Two thread layouts:
//   COL  line b = g mod TB, butterfly j = g / TB  (lines are adjacent columns
//        of a strided axis; lanes run over b)
//   ROW  butterfly j = g mod (L/R), line b = g / (L/R) (lines are contiguous
//        rows; lanes run over j)
// with g = t + T i for the thread's i-th butterfly.
#pragma once

#include "common.cuh"

namespace hf {

// ---------------------------------------------------------------------------
// Radix-R DFT in registers, natural order, sign DIR (-1 forward, +1 inverse).
// ---------------------------------------------------------------------------
// v * exp(DIR 2 pi i k / R) for compile-time R and k in [0, R/2)
template <int R, int DIR, int K>
__device__ __forceinline__ float2 rot_const(float2 v) {
    constexpr float kC8 = 0.70710678118654752440f;   // cos(pi/4)
    constexpr float kC16 = 0.92387953251128675613f;  // cos(pi/8)
    constexpr float kS16 = 0.38268343236508977173f;  // sin(pi/8)
    if constexpr (K == 0) {
        return v;
    } else if constexpr (4 * K == R) {
        return cmul_i<DIR>(v);
    } else if constexpr (R == 8) {
        // K = 1: (1 + DIR i)/sqrt2 ; K = 3: (-1 + DIR i)/sqrt2
        if constexpr (K == 1) {
            return DIR < 0 ? make_float2((v.x + v.y) * kC8, (v.y - v.x) * kC8)
                           : make_float2((v.x - v.y) * kC8, (v.y + v.x) * kC8);
        } else {
            return DIR < 0 ? make_float2((v.y - v.x) * kC8, -(v.x + v.y) * kC8)
                           : make_float2(-(v.x + v.y) * kC8, (v.x - v.y) * kC8);
        }
    } else {
        static_assert(R == 16, "radix");
        constexpr float c = K == 1 ? kC16 : K == 2 ? kC8 : K == 3 ? kS16 : K == 5 ? -kS16 : K == 6 ? -kC8 : -kC16;
        constexpr float s = K == 1 ? kS16 : K == 2 ? kC8 : K == 3 ? kC16 : K == 5 ? kC16 : K == 6 ? kC8 : kS16;
        return cmul(v, make_float2(c, DIR * s));
    }
}

template <int R, int DIR>
struct Dft {
    template <int K>
    __device__ __forceinline__ static void combine(float2* v, const float2* e, const float2* o) {
        if constexpr (K < R / 2) {
            const float2 t = rot_const<R, DIR, K>(o[K]);
            v[K] = cadd(e[K], t);
            v[K + R / 2] = csub(e[K], t);
            combine<K + 1>(v, e, o);
        }
    }
    __device__ __forceinline__ static void run(float2* v) {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            e[k] = v[2 * k];
            o[k] = v[2 * k + 1];
        }
        Dft<R / 2, DIR>::run(e);
        Dft<R / 2, DIR>::run(o);
        combine<0>(v, e, o);
    }
};

template <int DIR>
struct Dft<2, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int DIR>
struct Dft<4, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        const float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        const float2 a2 = cadd(v[1], v[3]), a3 = cmul_i<DIR>(csub(v[1], v[3]));
        v[0] = cadd(a0, a2);
        v[1] = cadd(a1, a3);
        v[2] = csub(a0, a2);
        v[3] = csub(a1, a3);
    }
};

// ---------------------------------------------------------------------------
// Stage plan of a length 2^LOG2L: ceil(LOG2L / 4) stages of radix <= 16,
// bits spread evenly with the larger radices last; REV reverses the order
// (the inverse transform runs the forward plan backwards so that its input
// positions are the forward transform's output positions).
// ---------------------------------------------------------------------------
template <int LOG2L, bool REV>
struct Plan {
    static constexpr int L = 1 << LOG2L;
    static constexpr int NS = (LOG2L + 3) / 4;
    static constexpr int bits_fwd(int s) { return LOG2L / NS + (s >= NS - LOG2L % NS ? 1 : 0); }
    static constexpr int bits(int s) { return REV ? bits_fwd(NS - 1 - s) : bits_fwd(s); }
    static constexpr int radix(int s) { return 1 << bits(s); }
    static constexpr int log2_before(int s) { return s == 0 ? 0 : log2_before(s - 1) + bits(s - 1); }
    static constexpr int first_radix() { return radix(0); }
    static constexpr int last_radix() { return radix(NS - 1); }
};

// Stage twiddle tables of a plan.  Stage s >= 1 (Ns = 2^log2_before(s), radix
// R) reads W_{Ns R}^{k r}, k = j mod Ns, r = 1..R-1; its table holds that value
// at [(r - 1) Ns + k] (r-major), so the lanes of a warp, which differ in k,
// read consecutive or identical words: no bank conflicts.
template <int LOG2L, bool REV>
struct TwTables {
    using P = Plan<LOG2L, REV>;
    static constexpr int stage_size(int s) { return ((1 << P::bits(s)) - 1) << P::log2_before(s); }
    static constexpr int offset(int s) { return s <= 1 ? 0 : offset(s - 1) + stage_size(s - 1); }
    static constexpr int size() { return P::NS <= 1 ? 0 : offset(P::NS - 1) + stage_size(P::NS - 1); }
};

// True when a plan and its reverse have the same stages (one table serves both).
template <int LOG2L>
constexpr bool palindromic() {
    using F = Plan<LOG2L, false>;
    for (int s = 0; s < F::NS; ++s)
        if (F::bits(s) != F::bits(F::NS - 1 - s)) return false;
    return true;
}

// Elements per thread for a line length: 16, never more than the line itself.
constexpr int elems_for(int log2l) { return log2l >= 4 ? 16 : (1 << log2l); }

// Compile-time geometry of a CTA: TB = 2^LOGTB lines of L = 2^LOG2L, E
// elements per thread, T threads.
template <int LOG2L_, int LOGTB_, bool ROW_>
struct Geo {
    static constexpr int LOG2L = LOG2L_;
    static constexpr int L = 1 << LOG2L_;
    static constexpr int LOGTB = LOGTB_;
    static constexpr int TB = 1 << LOGTB_;
    static constexpr bool ROW = ROW_;
    static constexpr int E = elems_for(LOG2L_);
    static constexpr int T = (TB * L) / E;
    static_assert(T >= 1 && T <= 512, "threads per CTA");
};

// Butterfly (line b, index j) of a thread's i-th radix-2^LR butterfly.
template <class G, int LR>
__device__ __forceinline__ void butterfly_of(int t, int i, int& b, int& j) {
    const int g = t + G::T * i;
    if constexpr (G::ROW) {
        j = g & ((1 << (G::LOG2L - LR)) - 1);
        b = g >> (G::LOG2L - LR);
    } else {
        b = g & (G::TB - 1);
        j = g >> G::LOGTB;
    }
}

// Shared-memory slot of element l of line b.  ROW lines are contiguous
// with the low four bits of l XOR-ed by the next four (bank spread for the
// stride patterns of the exchanges); COL tiles are [l][b].
template <class G>
__device__ __forceinline__ int smem_slot(int l, int b) {
    if constexpr (G::ROW) {
        return (b << G::LOG2L) + (l ^ ((l >> 4) & 15));
    } else {
        return (l << G::LOGTB) + b;
    }
}

// Slot of element l of line b in the exchange that follows a stage whose
// outputs are SH bits apart at its largest stride (SH = log2(Ns R)).  ROW:
// smem_slot.  COL: [l][b] with the bits of l that select a bank (the low
// 4 - LOGTB bits, for 8-byte elements) XOR-ed by the bits of l from SH up.
// A stage writes its outputs at (j / Ns) Ns R + (j mod Ns) + r Ns: when Ns is
// below the lanes' span of j, the lanes' positions differ only from bit SH
// up, and the XOR spreads them over the banks; the next stage reads runs of
// consecutive l, which the XOR only permutes within 2^SH.
template <class G, int SH>
__device__ __forceinline__ int exchange_slot(int l, int b) {
    if constexpr (G::ROW || G::LOGTB >= 4 || SH >= G::LOG2L) {
        return smem_slot<G>(l, b);
    } else {
        constexpr int mask = (16 >> G::LOGTB) - 1;
        return ((l ^ ((l >> SH) & mask)) << G::LOGTB) + b;
    }
}

// Element positions of the data a thread holds before stage 0 (IN) or after
// the last stage (OUT) of a plan: the i-th butterfly of radix R holds
// elements j + r L/R, r = 0..R-1, in v[i R + r].
template <class G, int R, class F>
__device__ __forceinline__ void for_each_element(int t, F&& f) {
    constexpr int LR = (R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 0);
    static_assert((1 << LR) == R, "radix");
#pragma unroll
    for (int i = 0; i < G::E / R; ++i) {
        int b, j;
        butterfly_of<G, LR>(t, i, b, j);
#pragma unroll
        for (int r = 0; r < R; ++r) f(i * R + r, b, j + r * (G::L / R));
    }
}

// Position l of element e, known only at run time, in the layout of
// for_each_element<G, R> for the COL geometry.
template <class G, int R>
__device__ __forceinline__ int col_element_l(int t, int e) {
    static_assert(!G::ROW, "column geometry");
    return ((t + G::T * (e / R)) >> G::LOGTB) + (e % R) * (G::L / R);
}

template <class G, int DIR, bool REV, int S>
struct Stages {
    using P = Plan<G::LOG2L, REV>;
    static constexpr int R = P::radix(S);
    static constexpr int LR = P::bits(S);
    static constexpr int LNS = P::log2_before(S);  // log2 Ns
    static constexpr int E = G::E;
    static_assert(E % R == 0, "E must be a multiple of every radix");

    __device__ __forceinline__ static void run(float2 (&v)[E], float2* sm, const float2* tw, int t) {
        constexpr int NB = E / R;
        if constexpr (LNS > 0) {
            // twiddles W_{Ns R}^{k r}, k = j mod Ns, from the stage's r-major table
            constexpr int off = TwTables<G::LOG2L, REV>::offset(S);
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                int b, j;
                butterfly_of<G, LR>(t, i, b, j);
                const int k = j & ((1 << LNS) - 1);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float2 w = tw[off + ((r - 1) << LNS) + k];
                    v[i * R + r] = DIR < 0 ? cmul(v[i * R + r], w) : cmulc(v[i * R + r], w);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) Dft<R, DIR>::run(&v[i * R]);
        if constexpr (S + 1 < P::NS) {
            __syncthreads();  // every thread is done reading the previous exchange
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                int b, j;
                butterfly_of<G, LR>(t, i, b, j);
                const int k = j & ((1 << LNS) - 1);
                const int base = ((j >> LNS) << (LNS + LR)) + k;
#pragma unroll
                for (int r = 0; r < R; ++r) sm[exchange_slot<G, LNS + LR>(base + (r << LNS), b)] = v[i * R + r];
            }
            __syncthreads();
            constexpr int R2 = P::radix(S + 1);
            for_each_element<G, R2>(t, [&](int e, int b, int l) { v[e] = sm[exchange_slot<G, LNS + LR>(l, b)]; });
            Stages<G, DIR, REV, S + 1>::run(v, sm, tw, t);
        }
    }
};

// Full transform.  On entry v holds the plan's IN positions, on exit its OUT
// positions.  sm (TB * L slots) holds the exchanges and tw the plan's stage
// twiddle tables (shared memory, load_stage_twiddles); contains
// __syncthreads(), so every thread of the CTA must call it.
template <class G, int DIR, bool REV>
__device__ __forceinline__ void fft(float2 (&v)[G::E], float2* sm, const float2* tw, int t) {
    Stages<G, DIR, REV, 0>::run(v, sm, tw, t);
}

// The twiddles of a packed real transform of length 2L: tw_s[k] = W_{2L}^k,
// k < L, from the plan's 4096-entry table.
template <int LOG2L>
__device__ __forceinline__ void load_half_twiddles(float2* tw_s, const float2* __restrict__ tw, int t, int T) {
    for (int k = t; k < (1 << LOG2L); k += T) tw_s[k] = __ldg(tw + (k << (kTwLog2 - LOG2L - 1)));
}

// The stage tables of plan (LOG2L, REV) from the plan's 4096-entry table.
template <int LOG2L, bool REV, int S = 1>
__device__ __forceinline__ void load_stage_twiddles(float2* tw_s, const float2* __restrict__ tw, int t, int T) {
    using P = Plan<LOG2L, REV>;
    if constexpr (S < P::NS) {
        constexpr int lns = P::log2_before(S), lr = P::bits(S);
        constexpr int off = TwTables<LOG2L, REV>::offset(S);
        for (int q = t; q < TwTables<LOG2L, REV>::stage_size(S); q += T) {
            const int r = (q >> lns) + 1, k = q & ((1 << lns) - 1);
            tw_s[off + q] = __ldg(tw + ((k * r) << (kTwLog2 - lns - lr)));
        }
        load_stage_twiddles<LOG2L, REV, S + 1>(tw_s, tw, t, T);
    }
}

// Stage tables for the forward plan and its reverse: the reverse's start at
// the returned pointer (the same tables when the plan is palindromic).
template <int LOG2L>
__device__ __forceinline__ float2* load_plan_twiddles(float2* tw_s, const float2* __restrict__ tw, int t, int T) {
    load_stage_twiddles<LOG2L, false>(tw_s, tw, t, T);
    if constexpr (palindromic<LOG2L>()) {
        return tw_s;
    } else {
        float2* rev = tw_s + TwTables<LOG2L, false>::size();
        load_stage_twiddles<LOG2L, true>(rev, tw, t, T);
        return rev;
    }
}

// Shared-memory slots of the stage tables of a plan and its reverse.
template <int LOG2L>
constexpr int plan_twiddle_slots() {
    return TwTables<LOG2L, false>::size() + (palindromic<LOG2L>() ? 0 : TwTables<LOG2L, true>::size());
}

}  // namespace hf
