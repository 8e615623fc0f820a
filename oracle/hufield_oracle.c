/*
 * hufield_oracle.c -- plain, slow FP64 CPU oracle of the spectral-filtering
 * generator of Zhong & Mao, "Ultra-Efficient Reconstruction of Anisotropic
 * Hyperuniform Continuous Random Fields in 2D and 3D via Generalized Spectral
 * Filtering" (arXiv 2509.08675), Sec. II.B.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * Every step is written in the order the paper gives it, with no blocking,
 * fusion or reordering:
 *   noise      white noise on the real lattice (Sec. II.B: i.i.d. Gaussian
 *              coefficients; a forward FFT of real white noise gives them
 *              with the Hermitian pairing a real field needs), or drawn
 *              directly as Hermitian complex Gaussian coefficients in
 *              k-space (the literal form of the same sentence)
 *   fft        own iterative radix-2 complex DFT, applied axis by axis
 *   filter     A(k) = sqrt(chi(k)), Eq. (8); chi from the generalized
 *              superellipse norm, Eq. (12), and the target spectrum, Eq. (13)
 *   inverse    f = IDFT(A * F), Eq. (9), real part
 *   normalise  f <- sigma_f (f - <f>) / sqrt(Var f), Eq. (15)
 *   threshold  sign map, Sec. II.B (last paragraph): f >= t -> +1 else -1
 *   binarise   noise-shaped binarisation (a reading of the future work of
 *              Sec. IV): sigma-delta modulation along axis 0, in FP32 (each
 *              site is a floating-point decision, taken in the kernel's
 *              precision; everything else here is FP64)
 *   spectrum   S(n) = |DFT(y)(n)|^2 / N, binned radially (and by angle in 2D)
 *   window     sigma_F^2(R), Eq. (1): variance of the field averaged over a
 *              ball of radius R, from the spectrum
 *
 * Readings of points the paper leaves open (Sec. II.B is silent on each):
 *   - noise is Philox4x32-10 (Salmon et al., SC'11) with key = seed and
 *     counter = (j lo, j hi, field_idx, 0), j = voxel >> 2, followed by
 *     Box-Muller on (x0,x1) and (x2,x3), u = (x + 1/2) 2^-32;
 *   - wavevectors are in units of the Nyquist wavenumber, kappa_i = 2 n_i/N_i;
 *   - the envelope is chi = C K^s exp(-(K-k0)^2 / (2 w^2)), the paper's
 *     Eq. (13) being the case k0 = 0, w = sigma, s = alpha; C puts the
 *     analytic maximum (at K*) at 1;
 *   - the filter is zero on every Nyquist plane and at K = 0;
 *   - variance is the population variance (1/N);
 *   - radial bin b holds b <= nr |kappa| < b+1, modes with |kappa| >= 1 are
 *     dropped; in 2D the folded angle atan2(kappa_1, kappa_0) in [0, pi) is
 *     split into ntheta half-open sectors by exact integer cross products.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the published description (Salmon, Moraes, Dror,     */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds; */
/* each round multiplies words 0 and 2 by the round multipliers, mixes the  */
/* high halves with words 1, 3 and the key, and the key is bumped by the    */
/* Weyl constants between rounds.                                           */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint64_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += weyl0;
            k[1] += weyl1;
        }
        uint64_t p0 = mult0 * (uint64_t)c[0];
        uint64_t p1 = mult1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k[0];
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k[1];
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static void noise_block(uint64_t seed, uint32_t field_idx, uint64_t j, uint32_t x[4]) {
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), field_idx, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, x);
}

/* Raw 32-bit noise words: word i of the lattice is component (i & 3) of the
 * Philox block i >> 2. */
void or_noise_bits(int64_t N, uint64_t seed, uint32_t field_idx, uint32_t *out) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (N + 3) / 4; ++j) {
        uint32_t x[4];
        noise_block(seed, field_idx, (uint64_t)j, x);
        for (int c = 0; c < 4; ++c)
            if (4 * j + c < N) out[4 * j + c] = x[c];
    }
}

/* Standard normal white noise by Box-Muller: from one block (x0,x1,x2,x3),
 * u_c = (x_c + 1/2) 2^-32, r = sqrt(-2 ln u0), z0 = r cos(2 pi u1),
 * z1 = r sin(2 pi u1), and z2, z3 likewise from (x2, x3). */
void or_noise(int64_t N, uint64_t seed, uint32_t field_idx, double *z) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (N + 3) / 4; ++j) {
        uint32_t x[4];
        double v[4];
        noise_block(seed, field_idx, (uint64_t)j, x);
        for (int pair = 0; pair < 2; ++pair) {
            double u0 = ((double)x[2 * pair] + 0.5) * ldexp(1.0, -32);
            double u1 = ((double)x[2 * pair + 1] + 0.5) * ldexp(1.0, -32);
            double r = sqrt(-2.0 * log(u0));
            v[2 * pair] = r * cos(2.0 * OR_PI * u1);
            v[2 * pair + 1] = r * sin(2.0 * OR_PI * u1);
        }
        for (int c = 0; c < 4; ++c)
            if (4 * j + c < N) z[4 * j + c] = v[c];
    }
}

/* ------------------------------------------------------------------------ */
/* DFT: X(n) = sum_x a(x) exp(-2 pi i n x / L) (dir = -1), inverse without   */
/* the 1/L factor (dir = +1).  Iterative radix-2: bit-reversal permutation,  */
/* then log2 L butterfly levels.  Data are interleaved (re, im) doubles.    */
/* ------------------------------------------------------------------------ */
static void fft1d(double *a, int64_t L, int dir, const double *cosv, const double *sinv) {
    for (int64_t i = 1, j = 0; i < L; ++i) {
        int64_t bit = L >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = a[2 * i], ti = a[2 * i + 1];
            a[2 * i] = a[2 * j]; a[2 * i + 1] = a[2 * j + 1];
            a[2 * j] = tr; a[2 * j + 1] = ti;
        }
    }
    for (int64_t len = 2; len <= L; len <<= 1) {
        int64_t half = len / 2, step = L / len;
        for (int64_t i = 0; i < L; i += len) {
            for (int64_t k = 0; k < half; ++k) {
                double wr = cosv[k * step], wi = dir * sinv[k * step];
                double *u = a + 2 * (i + k), *v = a + 2 * (i + k + half);
                double tr = v[0] * wr - v[1] * wi;
                double ti = v[0] * wi + v[1] * wr;
                v[0] = u[0] - tr; v[1] = u[1] - ti;
                u[0] += tr; u[1] += ti;
            }
        }
    }
}

/* In-place complex DFT of a C-order array of shape n[0..ndim-1] along
 * every axis; dir = -1 forward, +1 inverse (unnormalised). */
void or_fftn(int ndim, const int64_t *n, double *a, int dir) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    for (int axis = 0; axis < ndim; ++axis) {
        int64_t L = n[axis], stride = 1;
        for (int d = axis + 1; d < ndim; ++d) stride *= n[d];
        if (L < 2) continue;
        double *cosv = (double *)malloc(sizeof(double) * L / 2);
        double *sinv = (double *)malloc(sizeof(double) * L / 2);
        for (int64_t k = 0; k < L / 2; ++k) {
            cosv[k] = cos(2.0 * OR_PI * (double)k / (double)L);
            sinv[k] = sin(2.0 * OR_PI * (double)k / (double)L);
        }
        int64_t nlines = N / L;
#pragma omp parallel
        {
            double *buf = (double *)malloc(sizeof(double) * 2 * L);
#pragma omp for schedule(static)
            for (int64_t line = 0; line < nlines; ++line) {
                int64_t outer = line / stride, inner = line % stride;
                int64_t base = outer * L * stride + inner;
                for (int64_t l = 0; l < L; ++l) {
                    buf[2 * l] = a[2 * (base + l * stride)];
                    buf[2 * l + 1] = a[2 * (base + l * stride) + 1];
                }
                fft1d(buf, L, dir, cosv, sinv);
                for (int64_t l = 0; l < L; ++l) {
                    a[2 * (base + l * stride)] = buf[2 * l];
                    a[2 * (base + l * stride) + 1] = buf[2 * l + 1];
                }
            }
            free(buf);
        }
        free(cosv);
        free(sinv);
    }
}

/* ------------------------------------------------------------------------ */
/* Filter.                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    double p;        /* superellipse exponent, Eq. (12) */
    double axes[3];  /* semi-axes a, b, c of Eq. (12) */
    double rot;      /* rotation angle (radians) of the semi-axes, 2D plane 0-1 */
    double k0;       /* band centre, units of the Nyquist wavenumber */
    double width;    /* Gaussian band width w (sigma of Eq. (13)) */
    double supp;     /* small-k suppression exponent s (alpha of Eq. (13)) */
    int32_t form;    /* 0: generalised band at k0; 1: paper form, k0 = 0 */
} or_filter;

/* The analytic maximiser of K^s exp(-(K-k0)^2/(2 w^2)): s w^2 = K (K - k0). */
double or_kstar(const or_filter *f) {
    double k0 = f->form == 1 ? 0.0 : f->k0;
    return 0.5 * (k0 + sqrt(k0 * k0 + 4.0 * f->supp * f->width * f->width));
}

/* Generalized superellipse norm, Eq. (12), of the rotated wavevector. */
double or_superellipse(int ndim, const double *kappa, const or_filter *f) {
    double kr[3] = {kappa[0], ndim > 1 ? kappa[1] : 0.0, ndim > 2 ? kappa[2] : 0.0};
    if (ndim >= 2) {
        /* R(-rot): the semi-axis a points at angle rot from axis 0 toward axis 1 */
        double c = cos(f->rot), s = sin(f->rot);
        double k0r = c * kappa[0] + s * kappa[1];
        double k1r = -s * kappa[0] + c * kappa[1];
        kr[0] = k0r;
        kr[1] = k1r;
    }
    double sum = 0.0;
    for (int d = 0; d < ndim; ++d) sum += pow(fabs(kr[d]) / f->axes[d], f->p);
    return pow(sum, 1.0 / f->p);
}

/* A(k) = sqrt(chi(k)), Eqs. (8) and (13); zero on Nyquist planes and at K=0.
 * idx holds signed lattice indices n_i in [-N_i/2, N_i/2). */
double or_filter_value(int ndim, const int64_t *n, const int64_t *idx, const or_filter *f) {
    double kappa[3];
    for (int d = 0; d < ndim; ++d) {
        if (idx[d] == -n[d] / 2) return 0.0;
        kappa[d] = 2.0 * (double)idx[d] / (double)n[d];
    }
    double K = or_superellipse(ndim, kappa, f);
    if (K <= 0.0) return 0.0;
    double k0 = f->form == 1 ? 0.0 : f->k0;
    double ks = or_kstar(f);
    double w2 = f->width * f->width;
    /* s ln(K/K*); with s = 0 the factor K^s is 1 and the term vanishes, also when K* = 0 */
    double lnchi = (f->supp > 0.0 ? f->supp * log(K / ks) : 0.0) -
                   ((K - k0) * (K - k0) - (ks - k0) * (ks - k0)) / (2.0 * w2);
    return exp(0.5 * lnchi);
}

static void unravel(int ndim, const int64_t *n, int64_t lin, int64_t *idx) {
    for (int d = ndim - 1; d >= 0; --d) {
        int64_t i = lin % n[d];
        lin /= n[d];
        idx[d] = i < n[d] / 2 ? i : i - n[d];
    }
}

/* Filter on the full lattice in FFT order. */
void or_filter_grid(int ndim, const int64_t *n, const or_filter *f, double *H) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
#pragma omp parallel for schedule(static)
    for (int64_t lin = 0; lin < N; ++lin) {
        int64_t idx[3];
        unravel(ndim, n, lin, idx);
        H[lin] = or_filter_value(ndim, n, idx, f);
    }
}

/* ------------------------------------------------------------------------ */
/* Generator, Sec. II.B: noise -> DFT -> multiply by A -> inverse DFT ->    */
/* normalise (Eq. (15)).  Outputs the normalised field f (length N) and,    */
/* when spec != NULL, the filtered spectrum A F (interleaved complex).      */
/* ------------------------------------------------------------------------ */
/* Filter the spectrum a (interleaved complex, overwritten), invert and
 * normalise: the steps after the noise's coefficients are known. */
static void filter_inverse_normalise(int ndim, const int64_t *n, const or_filter *f, double sigma_f, double *a,
                                     double *out_f, double *spec) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double *H = (double *)malloc(sizeof(double) * N);
    or_filter_grid(ndim, n, f, H);
    for (int64_t i = 0; i < N; ++i) { a[2 * i] *= H[i]; a[2 * i + 1] *= H[i]; }
    free(H);
    if (spec) memcpy(spec, a, sizeof(double) * 2 * N);
    or_fftn(ndim, n, a, +1);
    /* real part of (1/N) sum F e^{+ikx}; the imaginary part is rounding noise */
    double mean = 0.0;
    for (int64_t i = 0; i < N; ++i) mean += a[2 * i] / (double)N;
    mean /= (double)N;
    double var = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double d = a[2 * i] / (double)N - mean;
        var += d * d;
    }
    var /= (double)N;
    /* Eq. (15) needs Var > 0; a filter with no power on the lattice gives g = 0,
     * and then f = 0 */
    double scale = var > 0.0 ? sigma_f / sqrt(var) : 0.0;
    for (int64_t i = 0; i < N; ++i) out_f[i] = (a[2 * i] / (double)N - mean) * scale;
}

void or_generate(int ndim, const int64_t *n, const or_filter *f, uint64_t seed, uint32_t field_idx,
                 double sigma_f, double *out_f, double *spec) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double *z = (double *)malloc(sizeof(double) * N);
    double *a = (double *)malloc(sizeof(double) * 2 * N);
    or_noise(N, seed, field_idx, z);
    for (int64_t i = 0; i < N; ++i) { a[2 * i] = z[i]; a[2 * i + 1] = 0.0; }
    free(z);
    or_fftn(ndim, n, a, -1);
    filter_inverse_normalise(ndim, n, f, sigma_f, a, out_f, spec);
    free(a);
}

/* Largest |Im| and rms of Re after the inverse DFT (realness check). */
void or_inverse_realness(int ndim, const int64_t *n, const or_filter *f, uint64_t seed, uint32_t field_idx,
                         double *max_abs_im, double *rms_re) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double *spec = (double *)malloc(sizeof(double) * 2 * N);
    double *tmp = (double *)malloc(sizeof(double) * N);
    or_generate(ndim, n, f, seed, field_idx, 1.0, tmp, spec);
    or_fftn(ndim, n, spec, +1);
    double mi = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double im = fabs(spec[2 * i + 1]);
        if (im > mi) mi = im;
        s2 += spec[2 * i] * spec[2 * i];
    }
    *max_abs_im = mi;
    *rms_re = sqrt(s2 / (double)N);
    free(spec);
    free(tmp);
}

/* Sign map, Sec. II.B: f >= t gives +1, else -1. */
void or_threshold(int64_t N, const double *f, double t, int8_t *m) {
    for (int64_t i = 0; i < N; ++i) m[i] = f[i] >= t ? (int8_t)1 : (int8_t)-1;
}

/* ------------------------------------------------------------------------ */
/* Noise-shaped binarisation.  Sec. II.B notes that the sign map generally   */
/* loses the field's hyperuniform scaling, and Sec. IV leaves binarisations  */
/* that keep it to future work without defining one.  This is the reading    */
/* built here: first-order sigma-delta modulation (one-dimensional error     */
/* diffusion) along axis 0, in strips of h consecutive rows.  With           */
/*   u(x) = clamp(g (f(x) - t), -1, 1),                                      */
/* each column of each strip runs, for rows r = 0 .. h-1 and e = 0 at the    */
/* strip's first row,                                                        */
/*   v = u + e,   m = (v >= 0 ? +1 : -1),   e <- v - m.                     */
/* Then |e| <= 1 and m - u = e_prev - e: the quantisation error is a first   */
/* difference along axis 0, so its spectrum carries 4 sin^2(pi n0 / N0),     */
/* which vanishes as k -> 0, and the map's spectrum near k = 0 follows that  */
/* of g (f - t).  g = 0 asks for g = 1 / max |f - t| (then |u| <= 1 and no   */
/* clamping); M = 0 gives u = 0.                                             */
/*                                                                           */
/* A floating-point comparison decides each site, so the decision is taken   */
/* in the precision the GPU kernel uses: every operation below is one FP32   */
/* operation rounded to nearest (this file is compiled without contraction). */
/* err, if not NULL, receives e after each site.                             */
/* ------------------------------------------------------------------------ */
float or_sd_gain(int64_t N, const float *f, float t) {
    float M = 0.0f;
    for (int64_t i = 0; i < N; ++i) {
        const float a = fabsf(f[i] - t);
        if (a > M) M = a;
    }
    return M > 0.0f ? 1.0f / M : 0.0f;
}

void or_sigma_delta(int64_t n0, int64_t cols, const float *f, float t, float g, int64_t h, int8_t *m,
                    float *err) {
    if (g == 0.0f) g = or_sd_gain(n0 * cols, f, t);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < cols; ++c) {
        for (int64_t s = 0; s < n0 / h; ++s) {
            float e = 0.0f;
            for (int64_t r = 0; r < h; ++r) {
                const int64_t i = (s * h + r) * cols + c;
                const float d = f[i] - t;
                const float y = d * g;
                const float u = fminf(fmaxf(y, -1.0f), 1.0f);
                const float v = u + e;
                const float q = v >= 0.0f ? 1.0f : -1.0f;
                m[i] = (int8_t)q;
                e = v - q;
                if (err) err[i] = e;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* k-space white noise: the Fourier coefficients of real white noise drawn   */
/* directly (Sec. II.B: i.i.d. complex Gaussian coefficients on the lattice, */
/* paired so that the field is real), instead of a forward DFT of real-space */
/* noise.  Same distribution, different numbers.                            */
/*                                                                           */
/* Half-spectrum mode (row, k_last), row the C-order index over the other   */
/* axes and k_last in [0, N_last/2] (all indices in [0, N_d)), takes Philox  */
/* block J = row (N_last/4 + 1) + (k_last >> 1) with counter (J lo, J hi,    */
/* field_idx, 1): the pair (x0, x1) for even k_last, (x2, x3) for odd,       */
/* u = (x + 1/2) 2^-32, Z = sqrt(-2 ln u_a) exp(2 pi i u_b) and              */
/* X = sqrt(N/2) Z, so E|X|^2 = N as for the DFT of unit white noise.  On    */
/* the planes k_last = 0 and k_last = N_last/2 the mode -n lies in the same  */
/* half: the one with the smaller row is drawn and the other is its          */
/* conjugate; a self-conjugate mode (every component 0 or N_d/2) is real,    */
/* sqrt(N) Re Z.  Every other mode of the full lattice is the conjugate of   */
/* its mirror in the half.                                                   */
/* ------------------------------------------------------------------------ */
static void kspace_draw(uint64_t seed, uint32_t field_idx, uint64_t row, int64_t kl, int64_t nlast, double N,
                        double *re, double *im) {
    uint64_t J = row * (uint64_t)(nlast / 4 + 1) + (uint64_t)(kl >> 1);
    uint32_t ctr[4] = {(uint32_t)J, (uint32_t)(J >> 32), field_idx, 1u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    int pair = (int)(kl & 1);
    double u0 = ((double)x[2 * pair] + 0.5) * ldexp(1.0, -32);
    double u1 = ((double)x[2 * pair + 1] + 0.5) * ldexp(1.0, -32);
    double r = sqrt(-2.0 * log(u0));
    double amp = sqrt(N / 2.0);
    *re = amp * r * cos(2.0 * OR_PI * u1);
    *im = amp * r * sin(2.0 * OR_PI * u1);
}

/* C-order index over every axis but the last. */
static uint64_t row_index(int ndim, const int64_t *n, const int64_t *idx) {
    uint64_t row = 0;
    for (int d = 0; d < ndim - 1; ++d) row = row * (uint64_t)n[d] + (uint64_t)idx[d];
    return row;
}

/* Coefficient of a mode in the half (k_last <= N_last/2). */
static void kspace_half_value(int ndim, const int64_t *n, const int64_t *idx, uint64_t seed, uint32_t field_idx,
                              double N, double *re, double *im) {
    int64_t kl = idx[ndim - 1], nlast = n[ndim - 1];
    uint64_t row = row_index(ndim, n, idx);
    if (kl != 0 && kl != nlast / 2) {
        kspace_draw(seed, field_idx, row, kl, nlast, N, re, im);
        return;
    }
    int64_t mirror[3];
    for (int d = 0; d < ndim; ++d) mirror[d] = (n[d] - idx[d]) % n[d];
    uint64_t rm = row_index(ndim, n, mirror);
    if (rm < row) {
        kspace_draw(seed, field_idx, rm, kl, nlast, N, re, im);
        *im = -*im;
    } else if (rm == row) {
        kspace_draw(seed, field_idx, row, kl, nlast, N, re, im);
        *re *= sqrt(2.0);
        *im = 0.0;
    } else {
        kspace_draw(seed, field_idx, row, kl, nlast, N, re, im);
    }
}

/* The full lattice of k-space noise coefficients, interleaved complex. */
void or_kspace_noise(int ndim, const int64_t *n, uint64_t seed, uint32_t field_idx, double *X) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
#pragma omp parallel for schedule(static)
    for (int64_t lin = 0; lin < N; ++lin) {
        int64_t idx[3] = {0, 0, 0};
        unravel(ndim, n, lin, idx);
        for (int d = 0; d < ndim; ++d) idx[d] = (idx[d] + n[d]) % n[d];  /* unsigned indices */
        double re, im;
        if (idx[ndim - 1] <= n[ndim - 1] / 2) {
            kspace_half_value(ndim, n, idx, seed, field_idx, (double)N, &re, &im);
        } else {
            int64_t mirror[3];
            for (int d = 0; d < ndim; ++d) mirror[d] = (n[d] - idx[d]) % n[d];
            kspace_half_value(ndim, n, mirror, seed, field_idx, (double)N, &re, &im);
            im = -im;
        }
        X[2 * lin] = re;
        X[2 * lin + 1] = im;
    }
}

/* or_generate with k-space noise: the coefficients above take the place of
 * the forward DFT of the real-space noise; filter, inverse and
 * normalisation are the same steps. */
void or_generate_kspace(int ndim, const int64_t *n, const or_filter *f, uint64_t seed, uint32_t field_idx,
                        double sigma_f, double *out_f, double *spec) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double *a = (double *)malloc(sizeof(double) * 2 * N);
    or_kspace_noise(ndim, n, seed, field_idx, a);
    filter_inverse_normalise(ndim, n, f, sigma_f, a, out_f, spec);
    free(a);
}

/* ------------------------------------------------------------------------ */
/* Binning.                                                                  */
/* ------------------------------------------------------------------------ */
static uint64_t isqrt_u64(uint64_t x) {
    uint64_t r = (uint64_t)sqrtl((long double)x);
    while (r > 0 && r * r > x) --r;
    while ((r + 1) * (r + 1) <= x) ++r;
    return r;
}

/* Boundary directions of the angular sectors, rounded to 2^30. */
void or_angle_table(int ntheta, int64_t *C, int64_t *S) {
    for (int j = 0; j < ntheta; ++j) {
        double th = OR_PI * (double)j / (double)ntheta;
        C[j] = llround(ldexp(cos(th), 30));
        S[j] = llround(ldexp(sin(th), 30));
    }
}

/* Bin of one mode: radial bin b with b <= nr |kappa| < b+1, |kappa|^2 =
 * sum (2 n_i / N_i)^2, tested exactly in integers after scaling by
 * Nmax^2; angular sector (2D) from the folded vector.  Returns -1 for
 * |kappa| >= 1. */
int or_bin_of(int ndim, const int64_t *n, const int64_t *idx, int nr, int ntheta,
              const int64_t *C, const int64_t *S) {
    int64_t nmax = 0;
    for (int d = 0; d < ndim; ++d) if (n[d] > nmax) nmax = n[d];
    uint64_t Q = 0;
    int64_t v[3];
    for (int d = 0; d < ndim; ++d) {
        v[d] = idx[d] * (nmax / n[d]);
        Q += (uint64_t)(4 * v[d] * v[d]);
    }
    uint64_t root = isqrt_u64((uint64_t)nr * (uint64_t)nr * Q);
    uint64_t b = root / (uint64_t)nmax;
    if (b >= (uint64_t)nr) return -1;
    int sector = 0;
    if (ntheta > 1) {
        int64_t a0 = v[0], a1 = v[1];
        if (a1 < 0 || (a1 == 0 && a0 < 0)) { a0 = -a0; a1 = -a1; }
        if (a0 != 0 || a1 != 0) {
            for (int j = 1; j < ntheta; ++j)
                if (C[j] * a1 - S[j] * a0 >= 0) sector = j;
        }
    }
    return (int)b * ntheta + sector;
}

/* Bin (or_bin_of) of every mode of the stored half spectrum: the axes before
 * the last in FFT order (index i is the signed i < n/2 ? i : i - n), the last
 * k = 0 .. n_last/2 - 1; -1 where |kappa| >= 1.  out has N/2 entries. */
void or_half_bins(int ndim, const int64_t *n, int nr, int ntheta, int32_t *out) {
    int64_t C[64], S[64];
    or_angle_table(ntheta, C, S);
    const int64_t M = n[ndim - 1] / 2;
    int64_t count = M;
    for (int d = 0; d < ndim - 1; ++d) count *= n[d];
#pragma omp parallel for schedule(static)
    for (int64_t lin = 0; lin < count; ++lin) {
        int64_t idx[3] = {0, 0, 0};
        int64_t rem = lin;
        idx[ndim - 1] = rem % M;
        rem /= M;
        for (int d = ndim - 2; d >= 0; --d) {
            const int64_t i = rem % n[d];
            rem /= n[d];
            idx[d] = i < n[d] / 2 ? i : i - n[d];
        }
        out[lin] = or_bin_of(ndim, n, idx, nr, ntheta, C, S);
    }
}

/* S(n) = |DFT(y)(n)|^2 / N over the full lattice, summed per bin; counts
 * are the number of lattice modes per bin.  Bins are overwritten. */
void or_spectrum_bins(int ndim, const int64_t *n, const double *y, int nr, int ntheta,
                      double *sums, int64_t *counts) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double *a = (double *)malloc(sizeof(double) * 2 * N);
    for (int64_t i = 0; i < N; ++i) { a[2 * i] = y[i]; a[2 * i + 1] = 0.0; }
    or_fftn(ndim, n, a, -1);
    int nb = nr * ntheta;
    for (int b = 0; b < nb; ++b) { sums[b] = 0.0; counts[b] = 0; }
    int64_t *C = (int64_t *)malloc(sizeof(int64_t) * ntheta);
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * ntheta);
    or_angle_table(ntheta, C, S);
    for (int64_t lin = 0; lin < N; ++lin) {
        int64_t idx[3];
        unravel(ndim, n, lin, idx);
        int b = or_bin_of(ndim, n, idx, nr, ntheta, C, S);
        if (b < 0) continue;
        double re = a[2 * lin], im = a[2 * lin + 1];
        sums[b] += (re * re + im * im) / (double)N;
        counts[b] += 1;
    }
    free(C);
    free(S);
    free(a);
}

/* Per-mode spectrum on the full lattice (FFT order), for small-grid pins. */
void or_spectrum_modes(int ndim, const int64_t *n, const double *y, double *S) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double *a = (double *)malloc(sizeof(double) * 2 * N);
    for (int64_t i = 0; i < N; ++i) { a[2 * i] = y[i]; a[2 * i + 1] = 0.0; }
    or_fftn(ndim, n, a, -1);
    for (int64_t i = 0; i < N; ++i) S[i] = (a[2 * i] * a[2 * i] + a[2 * i + 1] * a[2 * i + 1]) / (double)N;
    free(a);
}

/* Full pipeline: f, nlev sign maps, binned S of f and of every map; the
 * noise is drawn in real space (kspace = 0) or in k-space (kspace = 1). */
void or_pipeline_noise(int ndim, const int64_t *n, const or_filter *f, uint64_t seed, uint32_t field_idx,
                       int kspace, double sigma_f, const double *levels, int nlev, int nr, int ntheta,
                       double *out_f, int8_t *out_maps, double *sums_f, int64_t *counts_f,
                       double *sums_m, int64_t *counts_m) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    if (kspace)
        or_generate_kspace(ndim, n, f, seed, field_idx, sigma_f, out_f, NULL);
    else
        or_generate(ndim, n, f, seed, field_idx, sigma_f, out_f, NULL);
    or_spectrum_bins(ndim, n, out_f, nr, ntheta, sums_f, counts_f);
    double *mv = (double *)malloc(sizeof(double) * N);
    int nb = nr * ntheta;
    for (int t = 0; t < nlev; ++t) {
        int8_t *m = out_maps + (int64_t)t * N;
        or_threshold(N, out_f, levels[t], m);
        for (int64_t i = 0; i < N; ++i) mv[i] = (double)m[i];
        or_spectrum_bins(ndim, n, mv, nr, ntheta, sums_m + (int64_t)t * nb, counts_m + (int64_t)t * nb);
    }
    free(mv);
}

void or_pipeline(int ndim, const int64_t *n, const or_filter *f, uint64_t seed, uint32_t field_idx,
                 double sigma_f, const double *levels, int nlev, int nr, int ntheta,
                 double *out_f, int8_t *out_maps, double *sums_f, int64_t *counts_f,
                 double *sums_m, int64_t *counts_m) {
    or_pipeline_noise(ndim, n, f, seed, field_idx, 0, sigma_f, levels, nlev, nr, ntheta, out_f, out_maps, sums_f,
                      counts_f, sums_m, counts_m);
}

/* ------------------------------------------------------------------------ */
/* Window variance, Eq. (1) of Sec. II.A: sigma_F^2(R) = (1/v1(R)) int C(r)  */
/* alpha_2(r; R) dr, with alpha_2 the intersection volume of two balls of    */
/* radius R at distance r over v1(R).  That is the variance of the field     */
/* averaged over a ball of radius R; in Fourier space,                       */
/*   sigma_F^2(R) = (1/N^2) sum_{n != 0} |Y(n)|^2 m(|k_n| R)^2,             */
/* m the transform of the ball's indicator over its volume: 2 J1(x)/x in 2D, */
/* 3 (sin x - x cos x)/x^3 in 3D.  Reading: the lattice field is its         */
/* trigonometric interpolant, lengths are in lattice spacings, k_n has       */
/* components 2 pi n_d / N_d with n_d signed in [-N_d/2, N_d/2).             */
/* ------------------------------------------------------------------------ */
static double ball_transform(int ndim, double x) {
    if (x == 0.0) return 1.0;
    if (ndim == 2) return 2.0 * j1(x) / x;
    if (x < 1e-2) return 1.0 - x * x / 10.0 + x * x * x * x / 280.0;
    return 3.0 * (sin(x) - x * cos(x)) / (x * x * x);
}

static double mode_k(int ndim, const int64_t *n, const int64_t *idx) {
    double k2 = 0.0;
    for (int d = 0; d < ndim; ++d) {
        double kd = 2.0 * OR_PI * (double)idx[d] / (double)n[d];
        k2 += kd * kd;
    }
    return sqrt(k2);
}

/* sigma_F^2(R) of a lattice field y for nradii radii. */
void or_window_variance(int ndim, const int64_t *n, const double *y, int nradii, const double *R, double *out) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double *a = (double *)malloc(sizeof(double) * 2 * N);
    for (int64_t i = 0; i < N; ++i) { a[2 * i] = y[i]; a[2 * i + 1] = 0.0; }
    or_fftn(ndim, n, a, -1);
    for (int r = 0; r < nradii; ++r) out[r] = 0.0;
    for (int64_t lin = 1; lin < N; ++lin) {
        int64_t idx[3] = {0, 0, 0};
        unravel(ndim, n, lin, idx);
        double k = mode_k(ndim, n, idx);
        double p2 = a[2 * lin] * a[2 * lin] + a[2 * lin + 1] * a[2 * lin + 1];
        for (int r = 0; r < nradii; ++r) {
            double m = ball_transform(ndim, k * R[r]);
            out[r] += p2 * m * m;
        }
    }
    for (int r = 0; r < nradii; ++r) out[r] /= (double)N * (double)N;
    free(a);
}

/* Ensemble mean of sigma_F^2(R) for the generator with filter f: the field's
 * spectrum is proportional to A^2 (Eq. (8)) and its variance is sigma_f^2, so
 * E sigma_F^2(R) = sigma_f^2 sum_{n != 0} A(n)^2 m^2 / sum_{n != 0} A(n)^2. */
void or_window_variance_filter(int ndim, const int64_t *n, const or_filter *f, double sigma_f, int nradii,
                               const double *R, double *out) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    double total = 0.0;
    for (int r = 0; r < nradii; ++r) out[r] = 0.0;
    for (int64_t lin = 1; lin < N; ++lin) {
        int64_t idx[3] = {0, 0, 0};
        unravel(ndim, n, lin, idx);
        double A = or_filter_value(ndim, n, idx, f);
        double a2 = A * A;
        if (a2 == 0.0) continue;
        total += a2;
        double k = mode_k(ndim, n, idx);
        for (int r = 0; r < nradii; ++r) {
            double m = ball_transform(ndim, k * R[r]);
            out[r] += a2 * m * m;
        }
    }
    for (int r = 0; r < nradii; ++r) out[r] = total > 0.0 ? sigma_f * sigma_f * out[r] / total : 0.0;
}

/* Forward DFT of the noise at a list of modes, one by one from the
 * definition X(n) = sum_x z(x) exp(-2 pi i sum_d n_d x_d / N_d), for
 * lattices too large for the full oracle.  modes: nmodes x ndim signed. */
void or_noise_dft_at(int ndim, const int64_t *n, uint64_t seed, uint32_t field_idx,
                     int nmodes, const int64_t *modes, double *out) {
    int64_t N = 1;
    for (int d = 0; d < ndim; ++d) N *= n[d];
    for (int q = 0; q < 2 * nmodes; ++q) out[q] = 0.0;
    int64_t inner = N / n[0];
#pragma omp parallel
    {
        double *acc = (double *)calloc(2 * (size_t)nmodes, sizeof(double));
        double *z = (double *)malloc(sizeof(double) * inner);
#pragma omp for schedule(static)
        for (int64_t x0 = 0; x0 < n[0]; ++x0) {
            /* noise of slab x0, generated block by block */
            int64_t base = x0 * inner;
            for (int64_t i = 0; i < inner; i += 4) {
                uint32_t x[4];
                noise_block(seed, field_idx, (uint64_t)((base + i) >> 2), x);
                for (int pair = 0; pair < 2; ++pair) {
                    double u0 = ((double)x[2 * pair] + 0.5) * ldexp(1.0, -32);
                    double u1 = ((double)x[2 * pair + 1] + 0.5) * ldexp(1.0, -32);
                    double r = sqrt(-2.0 * log(u0));
                    if (i + 2 * pair < inner) z[i + 2 * pair] = r * cos(2.0 * OR_PI * u1);
                    if (i + 2 * pair + 1 < inner) z[i + 2 * pair + 1] = r * sin(2.0 * OR_PI * u1);
                }
            }
            for (int q = 0; q < nmodes; ++q) {
                const int64_t *m = modes + (int64_t)q * ndim;
                double sr = 0.0, si = 0.0;
                for (int64_t i = 0; i < inner; ++i) {
                    int64_t rem = i;
                    /* phase numerator modulo N_d for each axis, exact in integers */
                    double frac = 0.0;
                    for (int d = ndim - 1; d >= 1; --d) {
                        int64_t xd = rem % n[d];
                        rem /= n[d];
                        int64_t pd = ((m[d] % n[d] + n[d]) % n[d]) * xd % n[d];
                        frac += (double)pd / (double)n[d];
                    }
                    int64_t p0 = ((m[0] % n[0] + n[0]) % n[0]) * x0 % n[0];
                    frac += (double)p0 / (double)n[0];
                    frac -= floor(frac);
                    sr += z[i] * cos(2.0 * OR_PI * frac);
                    si -= z[i] * sin(2.0 * OR_PI * frac);
                }
                acc[2 * q] += sr;
                acc[2 * q + 1] += si;
            }
        }
#pragma omp critical
        for (int q = 0; q < 2 * nmodes; ++q) out[q] += acc[q];
        free(acc);
        free(z);
    }
}
