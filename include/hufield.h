/*
 * hufield.h -- C ABI of the GB300 (sm_103a) spectral-filtering generator of
 * hyperuniform random fields (Zhong & Mao, arXiv 2509.08675, Sec. II.B).
 *
 * Pipeline (Sec. II.B): seeded white noise -> forward real FFT -> multiply by
 * A(k) = sqrt(chi(k)) (Eq. 8) with chi from the generalized superellipse norm
 * (Eq. 12) and the band envelope (Eq. 13) -> inverse FFT (Eq. 9) ->
 * normalisation to zero mean and variance sigma_f^2 (Eq. 15) -> sign maps at
 * given levels (Sec. II.B, last paragraph) -> binned spectral density S(k) of
 * the field and of every map (the log S panels of Figs. 1-5).  Beside the
 * sign map, hufield_binarise gives a noise-shaped +-1 map that keeps the
 * field's suppression of S near k = 0 (Sec. IV's binarisations that keep
 * hyperuniformity, read as sigma-delta modulation along axis 0).
 *
 * Conventions shared by every call
 *   - Lattice: ndim = 2 or 3, C order, axis ndim-1 contiguous; every n[i] is a
 *     power of two with 8 <= n[i] <= 4096, and N = prod n[i] <= 2^31.
 *   - Signed index n_i in [-n[i]/2, n[i]/2); wavevector in units of the
 *     Nyquist wavenumber, kappa_i = 2 n_i / n[i] (kappa_i = +-1 is Nyquist).
 *     A physical k_i is kappa_i * pi n[i] / L.
 *   - Noise: Philox4x32-10 (Salmon et al., SC'11) with key = (seed lo, seed hi)
 *     and counter = (j lo, j hi, field_idx, 0) for the block j = voxel >> 2;
 *     its four words x0..x3 give voxels 4j..4j+3 by Box-Muller,
 *     u = (x + 1/2) 2^-32, z0 = sqrt(-2 ln u0) cos(2 pi u1),
 *     z1 = sqrt(-2 ln u0) sin(2 pi u1), z2/z3 likewise from (x2, x3).
 *   - Filter: K = (sum_i |kappa'_i / axes[i]|^p)^(1/p), kappa' = kappa rotated
 *     by -rot in the 0-1 plane; chi = C K^supp exp(-(K-k0)^2 / (2 width^2))
 *     with C putting the analytic maximum at 1; A = 0 at K = 0 and on every
 *     Nyquist plane.  form = 1 sets k0 = 0, which is the paper's Eq. (13)
 *     with alpha = supp and sigma = width.
 *   - Spectrum: S(n) = |DFT(y)(n)|^2 / N over the full lattice.  Radial bin b
 *     holds modes with b <= nr |kappa| < b + 1 (exact integer test); modes
 *     with |kappa| >= 1 are dropped.  In 2D, ntheta > 1 splits the folded
 *     angle atan2(kappa_1, kappa_0) in [0, pi) into ntheta half-open sectors
 *     whose edges are the directions round(2^30 (cos, sin)(j pi / ntheta)).
 *     Bin index = b * ntheta + sector.  sums[bin] += sum of S over its modes,
 *     counts[bin] += number of modes; the bin mean is sums / counts.
 *
 * Memory and execution
 *   - Every buffer argument named out_*, ws, sums, counts, f or y is a DEVICE
 *     pointer owned by the caller; levels is a HOST pointer.  Device buffers
 *     must be 256-byte aligned, except out_maps of hufield_threshold,
 *     hufield_pipeline and hufield_ensemble, and out_map of hufield_binarise,
 *     which need 4 bytes (a map may start at any field offset of a larger
 *     buffer, e.g. a batch item's).
 *     The library allocates device memory only in
 *     hufield_plan_create (a 32 KB twiddle table) and hufield_plan_set_bins,
 *     never on a hot call.
 *   - All hot calls are asynchronous on the given CUDA stream (a cudaStream_t
 *     passed as void*, NULL = legacy default stream) and return after
 *     enqueueing the work.  A stream-ordered caller may reuse ws once the call
 *     has completed on that stream.
 *   - Return value: HUFIELD_OK or an error code; arguments are validated before
 *     anything is enqueued, so an error return leaves every buffer untouched,
 *     except HUFIELD_ERR_CUDA (a launch failed; the stream state is that of
 *     the CUDA runtime).  No exception crosses this interface.
 *   - A plan may be used from one host thread at a time; distinct plans are
 *     independent.
 */
#ifndef HUFIELD_H
#define HUFIELD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum hufield_status {
    HUFIELD_OK = 0,
    HUFIELD_ERR_INVALID_ARG = 1,      /* NULL pointer, NaN/out-of-range parameter, bad dtype */
    HUFIELD_ERR_UNSUPPORTED_DIMS = 2, /* ndim or n[i] outside the supported set */
    HUFIELD_ERR_WS_TOO_SMALL = 3,     /* ws_bytes below hufield_workspace_bytes() */
    HUFIELD_ERR_CUDA = 4,             /* a CUDA runtime call or launch failed */
    HUFIELD_ERR_TIMEOUT = 5,          /* reserved for bounded device-side waits */
    HUFIELD_ERR_TOO_LARGE = 6,        /* lattice larger than a fixed-size static scratch */
    HUFIELD_ERR_NO_POWER = 7          /* device status: the filter is 0 at every lattice mode */
};

enum hufield_dtype { HUFIELD_F32 = 0, HUFIELD_BF16 = 1, HUFIELD_I8 = 2 };

typedef struct hufield_plan hufield_plan;

/* Plan flag: record CUDA events around every kernel launch of the plan's
 * calls (per-pass device times for profiling; see hufield_profile_read). */
#define HUFIELD_PLAN_PROFILE 1u
/* Plan flag, test hook for failure detection: the plan's strided passes never
 * issue the load of their first tile and bound each wait to ~2 ms, so every
 * such pass gives up, drains its own copies, and records a timeout in the
 * workspace status word (see hufield_workspace_status).  Outputs are then
 * undefined.  Not for production use. */
#define HUFIELD_PLAN_INJECT_TIMEOUT 2u
/* Plan flag: draw the white noise directly as its Fourier coefficients
 * (Sec. II.B: i.i.d. complex Gaussian coefficients on the lattice, paired
 * X(-n) = conj X(n) so that the field is real) instead of as real-space noise
 * followed by a forward FFT.  The field has the same distribution but other
 * numbers, and the path skips every forward pass.  Half-spectrum mode
 * (row, k_last), row the C-order index over the axes before the last, takes
 * Philox4x32-10 block J = row (n_last/4 + 1) + (k_last >> 1) with key = seed
 * and counter (J lo, J hi, field_idx, 1): words (x0, x1) for even k_last,
 * (x2, x3) for odd, u = (x + 1/2) 2^-32 and X = sqrt(N/2) sqrt(-2 ln u_a)
 * exp(2 pi i u_b).  On k_last = 0 the mode whose mirror -n has the smaller
 * row is the mirror's conjugate; a self-conjugate mode is sqrt(N) times the
 * real part of its unit draw.  Affects hufield_generate, hufield_pipeline and
 * hufield_ensemble; hufield_noise and hufield_forward keep the real-space
 * noise. */
#define HUFIELD_PLAN_KSPACE_NOISE 4u

typedef struct {
    int32_t ndim;   /* 2 or 3 */
    int32_t reserved;
    int64_t n[3];   /* lattice extent per axis; n[2] ignored in 2D */
} hufield_dims;

typedef struct {
    float p;        /* superellipse exponent, Eq. (12); 0 < p <= 1024 */
    float axes[3];  /* semi-axes a, b, c of Eq. (12); in [2^-20, 2^20] (axes[2] ignored in 2D) */
    float rot;      /* rotation of the semi-axes in the 0-1 plane, radians */
    float k0;       /* band centre in units of k_Nyquist (ignored when form = 1) */
    float width;    /* Gaussian width w (sigma of Eq. 13) in units of k_Nyquist; > 0 */
    float supp;     /* small-k exponent s (alpha of Eq. 13); >= 0 */
    float sigma_f;  /* target standard deviation of the field, Eq. (15); > 0 */
    int32_t form;   /* 0 generalised band at k0, 1 paper form (k0 = 0) */
    int32_t nyquist;/* must be 0: the filter is zero on Nyquist planes */
} hufield_filter;

/* Plan for one lattice.  Allocates the twiddle table on the current CUDA
 * device and chooses launch shapes; the plan must be used on that device.
 * flags is 0 or a combination of HUFIELD_PLAN_PROFILE,
 * HUFIELD_PLAN_INJECT_TIMEOUT and HUFIELD_PLAN_KSPACE_NOISE (any other bit:
 * HUFIELD_ERR_INVALID_ARG).  Returns HUFIELD_ERR_UNSUPPORTED_DIMS
 * for a lattice outside the set above. */
int hufield_plan_create(hufield_plan **plan, const hufield_dims *dims, uint32_t flags);
int hufield_plan_destroy(hufield_plan *plan);

/* Plan-time bins: builds, on the plan's device, the bin of every mode for
 * (nr, ntheta) and the number of modes per bin (allocating N bytes plus
 * 8 nr ntheta bytes, freed with the plan), so that later calls with the
 * same nr and ntheta reuse them instead of building them per call (the bins
 * depend only on the lattice).  nr = 0 drops them.  Synchronises the device;
 * call it outside stream capture. */
int hufield_plan_set_bins(hufield_plan *plan, int32_t nr, int32_t ntheta);

/* Autotuning of the plan's launch choices for the strided passes: their tile
 * width (hufield_plan_set_tile), resident CTAs per SM of each pass mode
 * (plain, filter, bins, k-space) and the L2 promotion of their tensor maps.
 * Times hufield_pipeline with filter f, nlev
 * levels and nr x ntheta bins on scratch it allocates and frees (best of
 * three calls per candidate, coordinate descent, a change kept only when 2%
 * faster), and keeps the fastest choice in the plan; results are the same
 * for every choice up to the order of the bin sums.  With the environment
 * variable HUFIELD_AUTOTUNE_CACHE naming a file, a choice recorded there for
 * the same device, lattice and call shape is reused without timing, and a new
 * one is appended.  Synchronises its own stream; call it outside stream
 * capture.  Errors: HUFIELD_ERR_INVALID_ARG (arguments as for
 * hufield_pipeline), HUFIELD_ERR_CUDA, HUFIELD_ERR_TIMEOUT (a bounded device
 * wait ran out); on error the plan keeps its defaults.  Not in the paper: a
 * deployment convenience. */
int hufield_plan_autotune(hufield_plan *plan, const hufield_filter *f, int32_t nlev, int32_t nr, int32_t ntheta);

/* The plan's launch choices: out[0..3] CTAs per SM of the plain, filter,
 * bins and k-space strided passes, out[4] the L2 promotion in bytes (0: 64 or
 * 128 by the tile's row width). */
int hufield_plan_tuning(const hufield_plan *plan, int32_t out[5]);

/* Tile width of the strided passes along axes of 256 or more: 0 by size (the
 * wide tile of 8192 / L or 4096 / L columns, except the two-column tile for
 * columns of 1024 or more whose wide tiles would leave SMs idle), 1 the wide
 * tile wherever the columns fill it, 2 the two-column tile.  Every choice
 * computes the same results up to the order of the bin sums.  A cached bin
 * table (hufield_plan_set_bins), which is laid out in the axis-0 tiles, is
 * rebuilt when the width of those tiles changes (synchronising the device, as
 * hufield_plan_set_bins does).  hufield_plan_tile reads the choice. */
int hufield_plan_set_tile(hufield_plan *plan, int32_t tile);
int hufield_plan_tile(const hufield_plan *plan, int32_t *tile);

/* Order in which the CTAs of the strided passes take their tiles: 0 the
 * default (interleaved: neighbouring tiles, whose box rows share DRAM sectors
 * and L2 lines, run at the same time on different CTAs), 1 contiguous chunks (CTA
 * c runs tiles c T / G .. (c + 1) T / G - 1 of T on a grid of G), 2
 * interleaved (CTA c runs tiles c, c + G, c + 2 G, ...).  Every order
 * computes the same fields and maps; bin sums may differ in their rounding
 * order.  Takes effect at the next call.  Errors: HUFIELD_ERR_INVALID_ARG.
 * hufield_plan_order reads the choice.  Not in the paper: a launch choice. */
int hufield_plan_set_order(hufield_plan *plan, int32_t order);
int hufield_plan_order(const hufield_plan *plan, int32_t *order);

/* Storage of the sign maps (the +-1 maps of Sec. II.B, last paragraph) that
 * hufield_threshold, hufield_pipeline and hufield_ensemble write through this
 * plan.  HUFIELD_MAPS_I8 (the default): one int8 per site, +1 or -1, a map of
 * N sites at out_maps + t * N.  HUFIELD_MAPS_BITS: one bit per site, site i of
 * a map at bit (i mod 32) of the 32-bit little-endian word i / 32, 1 for +1
 * and 0 for -1; a map takes N / 8 bytes, map t of field e of an ensemble at
 * byte (e * nlev + t) * N / 8.  The same maps either way, 8 times fewer
 * bytes to store or copy; the maps' spectra are unaffected (batches take the
 * format from HUFIELD_BATCH_MAPS_BITS).  Returns
 * HUFIELD_ERR_INVALID_ARG for another format; hufield_plan_maps_format reads
 * the setting. */
enum hufield_maps_format { HUFIELD_MAPS_I8 = 0, HUFIELD_MAPS_BITS = 1 };
int hufield_plan_set_maps_format(hufield_plan *plan, int32_t format);
int hufield_plan_maps_format(const hufield_plan *plan, int32_t *format);

/* Bytes of device workspace a call needs: nlev sign maps (0 for
 * hufield_generate, 1 for hufield_spectrum) and nbins = nr * ntheta bins
 * (0 when no spectrum is taken).  Returns 0 for invalid arguments. */
size_t hufield_workspace_bytes(const hufield_plan *plan, int32_t nlev, int32_t nbins);

/* Noise of field (seed, field_idx), Sec. II.B: bits (N uint32 words, word i =
 * Philox word i & 3 of block i >> 2) and/or z (N floats, Box-Muller).  Either
 * output may be NULL. */
int hufield_noise(hufield_plan *plan, uint64_t seed, uint32_t field_idx, uint32_t *bits, float *z,
                  void *stream);

/* Forward r2c DFT of the noise (diagnostic): X(n) = sum_x z(x) e^{-2 pi i n.x/N}
 * into ws at byte offset 256 (every workspace begins with a 256-byte status
 * header) as complex64 [n0][n1]...[n_last/2], i.e. the half spectrum without
 * its Nyquist plane along the last axis (k_last = 0 .. n_last/2 - 1). */
int hufield_forward(hufield_plan *plan, uint64_t seed, uint32_t field_idx, void *ws, size_t ws_bytes,
                    void *stream);

/* Steps noise -> r2c -> filter -> c2r -> normalise (Sec. II.B, Eqs. 8-15):
 * writes the field f (N values of out_dtype, HUFIELD_F32 or HUFIELD_BF16). */
int hufield_generate(hufield_plan *plan, const hufield_filter *filt, uint64_t seed, uint32_t field_idx,
                     int32_t out_dtype, void *out_f, void *ws, size_t ws_bytes, void *stream);

/* Sign maps of a field (Sec. II.B, last paragraph): out_maps[t * N + i] =
 * f[i] >= levels[t] ? +1 : -1 for t < nlev (1 <= nlev <= 8), stored as the
 * plan's maps format says (hufield_plan_set_maps_format).  dtype of f is
 * HUFIELD_F32 or HUFIELD_BF16. */
int hufield_threshold(hufield_plan *plan, const void *f, int32_t dtype, const float *levels, int32_t nlev,
                      int8_t *out_maps, void *stream);

/* Noise-shaped binarisation of a field: a +-1 map that keeps the field's
 * suppression of fluctuations near k = 0, which the sign map loses (Sec. II.B,
 * last paragraph; Sec. IV names such binarisations as future work without
 * defining one).  This is first-order sigma-delta modulation (one-dimensional
 * error diffusion) along axis 0, in strips of h rows: with
 *   u = clamp(g (f - level), -1, 1),
 * each column of each strip runs, row by row from e = 0,
 *   v = u + e,  m = (v >= 0 ? +1 : -1),  e <- v - m,
 * every operation one FP32 operation rounded to nearest.  |e| <= 1, and the
 * quantisation error m - u is a first difference along axis 0, so its
 * spectrum carries the factor 4 sin^2(pi n0 / n[0]) and vanishes as k -> 0;
 * the map's spectrum there follows that of g (f - level), and each column's
 * mean over a strip that of u to within 1 / h.
 *   f        device, N values of dtype (HUFIELD_F32 or HUFIELD_BF16), C order,
 *            256-byte aligned; not modified
 *   level    the level t (finite)
 *   gain     g > 0, or 0 for g = 1 / max |f - level| (then |u| <= 1; u = 0
 *            when f == level everywhere); negative or non-finite: invalid
 *   strip    rows per strip h: a power of two in [1, n[0]], or 0 for
 *            min(n[0], 256); strips start from e = 0 and run in parallel
 *   out_map  device, written in the plan's maps format
 *            (hufield_plan_set_maps_format): N int8, or N / 8 bytes of
 *            one-bit words (site i at bit i mod 32 of word i / 32; needs
 *            N / n[0] >= 32); 4-byte aligned
 *   ws       the workspace of hufield_generate (hufield_workspace_bytes(plan,
 *            0, 0)), used for gain = 0 only (the maximum's reduction word);
 *            may be NULL when gain > 0
 * Errors: HUFIELD_ERR_INVALID_ARG (pointers, alignment, dtype, level, gain,
 * strip, one-bit maps with N / n[0] < 32), HUFIELD_ERR_WS_TOO_SMALL,
 * HUFIELD_ERR_CUDA.  Nothing is enqueued when an argument is refused. */
int hufield_binarise(hufield_plan *plan, const void *f, int32_t dtype, float level, float gain, int32_t strip,
                     int8_t *out_map, void *ws, size_t ws_bytes, void *stream);

/* Binned spectral density of a real field y (dtype F32, BF16 or I8):
 * S(n) = |DFT(y)(n)|^2 / N.  nr in [1, 4096], ntheta in [1, 64] (2D only for
 * ntheta > 1), nr * ntheta <= 4096.  accumulate = 0 overwrites sums/counts,
 * 1 adds to them (ensembles). */
int hufield_spectrum(hufield_plan *plan, const void *y, int32_t dtype, int32_t nr, int32_t ntheta,
                     int32_t accumulate, double *sums, int64_t *counts, void *ws, size_t ws_bytes,
                     void *stream);

/* Whole path, fused: generate (as hufield_generate), then for each of nlev
 * (0..8) levels the sign map (as hufield_threshold), and the binned S of the
 * field (sums_f/counts_f) and of each map (sums_m/counts_m, nlev blocks of
 * nr * ntheta).  out_f and out_maps may be NULL (not stored).  The field's S
 * is taken from the filtered spectrum (S_f(n) = N |G(n)|^2 / sum |G|^2), which
 * equals the spectrum of the stored FP32 field up to rounding. */
int hufield_pipeline(hufield_plan *plan, const hufield_filter *filt, uint64_t seed, uint32_t field_idx,
                     int32_t out_dtype, void *out_f, const float *levels, int32_t nlev, int8_t *out_maps,
                     int32_t nr, int32_t ntheta, int32_t accumulate, double *sums_f, int64_t *counts_f,
                     double *sums_m, int64_t *counts_m, void *ws, size_t ws_bytes, void *stream);

/* Ensemble: hufield_pipeline for field_idx = field0 .. field0 + nfields - 1
 * with the same seed and filter, bins accumulated over the ensemble.  Field e
 * is written at out_f + e * N elements and its maps at out_maps + e * nlev * N
 * (bytes; e * nlev * N / 8 with one-bit maps, hufield_plan_set_maps_format)
 * (either may be NULL).  accumulate applies to the first field.  A workspace
 * of two slices, ws_bytes >= 2 * W with W = hufield_workspace_bytes(plan,
 * nlev, nr * ntheta) rounded up to a multiple of 256, runs the odd fields on
 * the plan's second stream and slice, overlapping consecutive fields; the
 * call stays ordered on `stream` (it forks and joins there), both lanes
 * report to the first slice's status word, and the bins are added in a
 * different order (the sums agree to rounding). */
int hufield_ensemble(hufield_plan *plan, const hufield_filter *filt, uint64_t seed, uint32_t field0,
                     int32_t nfields, int32_t out_dtype, void *out_f, const float *levels, int32_t nlev,
                     int8_t *out_maps, int32_t nr, int32_t ntheta, int32_t accumulate, double *sums_f,
                     int64_t *counts_f, double *sums_m, int64_t *counts_m, void *ws, size_t ws_bytes,
                     void *stream);

/* Allocation-free variant of hufield_spectrum, for callers that must not
 * allocate device memory: code running where cudaMalloc is forbidden or
 * unavailable (inside a host-managed memory budget, a plugin that may only
 * touch buffers handed to it, or a latency-critical loop that cannot afford
 * cudaMalloc's implicit device synchronisation).  The paper has no
 * counterpart; this is a deployment convenience.
 *   - No plan and no workspace: the lattice comes as dims, and the scratch
 *     (the half spectrum, 4 MiB; its bin table, 1 MiB) and the twiddle table
 *     (32 KiB) are file-scope static device arrays of the library.  Every GPU
 *     that loads the library holds them until the process exits.
 *   - Largest lattice: N = prod n[i] <= 2^20 (e.g. 1024^2, 128^2 x 64);
 *     larger lattices return HUFIELD_ERR_TOO_LARGE before anything is enqueued.
 *     Other limits and arguments as hufield_spectrum.
 *   - The first call on each device does the set-up (looks up the static
 *     arrays' device addresses, fills the twiddle table and waits for it on
 *     `stream`); make that first call before any stream capture.
 *   - Calls never call cudaMalloc, cudaFree or any allocating routine.  Every
 *     call shares the same scratch, which keeps the previous call's contents
 *     (each call overwrites all of it before reading it); calls that overlap
 *     on the GPU race, so serialise them (one stream, or events). */
int hufield_spectrum_noalloc(const hufield_dims *dims, const void *y, int32_t dtype, int32_t nr, int32_t ntheta,
                             int32_t accumulate, double *sums, int64_t *counts, void *stream);

/* Device-side status of the most recent hufield_spectrum_noalloc call on the
 * current device: the allocation-free call has no workspace, so its kernels
 * report a bounded wait that ran out in a word of the library's static
 * scratch instead.  Waits for `stream`, reads that word (no allocation) and
 * returns HUFIELD_ERR_TIMEOUT (that call's bins are undefined) or HUFIELD_OK
 * (also before any call on the device); HUFIELD_ERR_CUDA if the copy fails.
 * The word belongs to whichever call ran last, like the rest of the scratch. */
int hufield_spectrum_noalloc_status(void *stream);

/* ---- Ragged batches ------------------------------------------------------
 * Many fields of different lattices and filters in one launch: the whole
 * path (as hufield_pipeline with one level and radial bins) for every item.
 * Items are grouped by lattice into size classes, each with its own plan
 * (bins cached) and two lanes (a stream and a workspace slice each) that take
 * the class's items in turn; hufield_batch_run captures the whole batch into
 * one CUDA graph, with the lanes as parallel branches, and replays it on later
 * runs with the same buffers (one graph launch per run).
 * Outputs lie end to end in item order (see hufield_batch_layout). */
typedef struct {
    hufield_dims dims;
    hufield_filter filt;
    uint64_t seed;
    uint32_t field_idx;
    float level;    /* sign-map level */
    int32_t nr;     /* radial bins (no angular sectors) */
} hufield_batch_item;

typedef struct hufield_batch hufield_batch;

/* Batch flag: autotune every size class's plan (hufield_plan_autotune with
 * the class's first item: its filter, one level and its radial bins). */
#define HUFIELD_BATCH_AUTOTUNE 1u

/* Lanes per size class: HUFIELD_BATCH_LANES(l), 1 <= l <= 8, in the flags
 * (default 2).  Each lane is a stream and a workspace slice; more lanes let
 * many small fields, whose passes each fill only a few SMs, run side by side. */
#define HUFIELD_BATCH_LANES(l) (((uint32_t)(l) & 15u) << 8)

/* Batch flag: run every item through its own calls (hufield_ensemble of one
 * field), as for a size class whose items differ in their number of bins.
 * Without it, a class whose items share nr runs a chunk of items at a time
 * (as many as 512 MB of half spectra per lane hold) through the passes of the
 * path, each pass one launch over the whole chunk with every field's own
 * filter, seed, index and level; the filter's band edge is the chunk's
 * largest (the environment variable HUFIELD_BATCH_CHUNK_BYTES, read when the
 * batch is planned, sets another budget).  Both give the same fields and maps;
 * bin sums agree to rounding. */
#define HUFIELD_BATCH_PER_ITEM 2u

/* Batch flag: the items' parameters may be replaced after planning
 * (hufield_batch_set_params) without capturing the graph again; the filter's
 * band edge then prunes nothing. */
#define HUFIELD_BATCH_UPDATABLE 4u

/* Batch flag: sign maps one bit per site (HUFIELD_MAPS_BITS layout, see
 * hufield_plan_set_maps_format): item i's map starts at bit f_offset[i] of
 * out_maps, i.e. byte f_offset[i] / 8, and the whole buffer takes sum N_i / 8
 * bytes. */
#define HUFIELD_BATCH_MAPS_BITS 8u

/* Plan a batch of n >= 1 items on the current device (copies the items;
 * flags: HUFIELD_BATCH_AUTOTUNE, HUFIELD_BATCH_PER_ITEM, HUFIELD_BATCH_UPDATABLE,
 * HUFIELD_BATCH_MAPS_BITS and/or HUFIELD_BATCH_LANES(l)).  Allocates the size-class plans, streams and the
 * batched classes' parameter arrays. */
int hufield_batch_plan(hufield_batch **batch, const hufield_batch_item *items, int32_t n, uint32_t flags);

/* Output layout (host arrays of n entries, either may be NULL): item i's
 * field is out_f[f_offset[i] .. + N_i) (and its map the same range of
 * out_maps), its bins [bin_offset[i] .. + nr_i) of each bin array.  totals
 * (may be NULL) receives {sum of N_i, sum of nr_i, workspace bytes}. */
int hufield_batch_layout(const hufield_batch *batch, int64_t *f_offset, int64_t *bin_offset, int64_t totals[3]);

/* Run the batch (asynchronous on `stream`): out_f FP32 fields, out_maps sign
 * maps, int8 or one bit per site (HUFIELD_BATCH_MAPS_BITS) (either may be
 * NULL), field and map bins (overwritten).  A run
 * with a set of buffers (outputs, bins, workspace) that none of the last two
 * sets used captures the graph; the graphs of the two most recent sets are
 * kept, so outputs alternating between two sets replay without a capture.
 * Runs sharing a workspace must not overlap in time (one stream, or ordered). */
int hufield_batch_run(hufield_batch *batch, float *out_f, int8_t *out_maps, double *sums_f, int64_t *counts_f,
                      double *sums_m, int64_t *counts_m, void *ws, size_t ws_bytes, void *stream);

/* Kernels one hufield_batch_run launches (inside its graph): per batched
 * chunk or per item run on its own, 5 for a 2D and 8 for a 3D lattice. */
int hufield_batch_launches(const hufield_batch *batch, int64_t *launches);

/* Replace the parameters (filter, seed, field index, level) of every item of
 * a batch planned with HUFIELD_BATCH_UPDATABLE; item i keeps its lattice and
 * nr.  Copies on `stream` and waits for it; later runs use the new values
 * (a size class run item by item captures its graph again). */
int hufield_batch_set_params(hufield_batch *batch, const hufield_batch_item *items, int32_t n, void *stream);

int hufield_batch_destroy(hufield_batch *batch);

/* Window variance, Eq. (1) of Sec. II.A: sigma_F^2(R) = (1/v1(R)) int C(r)
 * alpha_2(r; R) dr, the variance of the field averaged over a ball of radius
 * R.  Computed from the spectrum as (1/N^2) sum_{n != 0} |Y(n)|^2 m(|k_n| R)^2,
 * m = 2 J1(x)/x (2D) or 3 (sin x - x cos x)/x^3 (3D), the transform of the
 * ball's indicator over its volume, with the lattice field read as its
 * trigonometric interpolant, k_n of components 2 pi n_d / N_d (n_d signed)
 * and R in lattice spacings.  Every mode is included (the Nyquist plane of
 * the last axis by a separate plain DFT).  The window terms are FP64.
 *
 * hufield_window_variance: of a stored real field y (dtype F32, BF16 or I8:
 * fields and sign maps), N elements in C order, 256-byte aligned.
 * hufield_window_variance_filter: the ensemble mean for filter f, which does
 * not depend on the noise: sigma_f^2 sum A^2 m^2 / sum A^2 (Eq. (8): the
 * spectrum is proportional to A^2).
 *
 * radii: host array of nradii in [1, 64] finite values >= 0.  out: device,
 * nradii doubles (overwritten).  ws: hufield_window_variance needs
 * hufield_workspace_bytes(plan, 3, 0) bytes, hufield_window_variance_filter
 * hufield_workspace_bytes(plan, 0, 0).  Stream-ordered and asynchronous;
 * HUFIELD_ERR_INVALID_ARG for bad arguments. */
int hufield_window_variance(hufield_plan *plan, const void *y, int32_t dtype, int32_t nradii, const float *radii,
                            double *out, void *ws, size_t ws_bytes, void *stream);
int hufield_window_variance_filter(hufield_plan *plan, const hufield_filter *f, int32_t nradii, const float *radii,
                                   double *out, void *ws, size_t ws_bytes, void *stream);

/* Per-mode spectra over the stored half spectrum, float out[n0][n1][k_last]
 * (3D) or out[n0][k_last] (2D) with k_last = 0 .. n_last/2 - 1 and the other
 * indices in FFT order (device, N/2 floats, overwritten; the other half is
 * the mirror, S(-n) = S(n)).
 * hufield_spectrum_modes: S(n) = |DFT(y)(n)|^2 / N of a stored real field y
 * (F32, BF16 or I8), ws >= hufield_workspace_bytes(plan, 1, 0).
 * hufield_filter_modes: A(n)^2, Eqs. (8), (12), (13), the filter's target
 * spectrum up to its normalisation (zero at n = 0 and on Nyquist planes). */
int hufield_spectrum_modes(hufield_plan *plan, const void *y, int32_t dtype, float *out, void *ws, size_t ws_bytes,
                           void *stream);
int hufield_filter_modes(hufield_plan *plan, const hufield_filter *f, float *out, void *stream);

/* The filter's band edge along the last axis (Eqs. 12-13, Sec. II.B): *kz
 * receives the first k_last from which every mode of the filter is exactly
 * zero in FP32 (the exponent of A is below -140, far past the FP32 underflow),
 * or n_last / 2 when there is none.  The generator's passes after the forward
 * transform skip the columns k_last >= kz; a caller can use kz to count the
 * bytes those passes move.  Host only, nothing is enqueued.  Errors:
 * HUFIELD_ERR_INVALID_ARG (null pointer or a filter hufield_generate rejects). */
int hufield_filter_band_edge(const hufield_plan *plan, const hufield_filter *f, int64_t *kz);

/* Group means of per-item bins laid out item after item (nbins each, as a
 * batch whose items share nbins lays them out): out[g][b] = (sum over the
 * group_size items of group g of sums) / (sum of their counts), FP32, 0 when
 * empty; groups x nbins entries. */
int hufield_bins_group_mean(const double *sums, const int64_t *counts, int64_t groups, int32_t group_size,
                            int32_t nbins, float *out, void *stream);

/* Bin means: out_mean[b] = counts[b] ? sums[b] / counts[b] : 0. */
int hufield_bins_mean(const double *sums, const int64_t *counts, int32_t nbins, double *out_mean,
                      void *stream);

/* Device-side status of the most recent call that used workspace `ws` (every
 * call clears the first word of its workspace when it starts, in stream
 * order, and its kernels set bits in it).  This function waits for `stream`,
 * reads the word and returns:
 *   HUFIELD_ERR_TIMEOUT   a bounded wait on a bulk copy (~1 s) ran out: the
 *                         call's outputs are undefined;
 *   HUFIELD_ERR_NO_POWER  the filter is 0 at every lattice mode (for example a
 *                         band beyond the Nyquist wavenumber): Eq. (15) has no
 *                         variance to divide by, the field was set to 0 (its
 *                         maps follow from f = 0) and no field bins were added;
 *   HUFIELD_OK            otherwise. */
int hufield_workspace_status(const void *ws, void *stream);

/* Profiling (plans created with HUFIELD_PLAN_PROFILE): waits for the events
 * recorded since the previous read and adds, per pass kind, the device time
 * in ms and the number of launches into ms[i] and launches[i] for
 * i < min(n, number of kinds).  Kind names, comma separated, in that order:
 * hufield_profile_names(). */
int hufield_profile_read(hufield_plan *plan, double *ms, int64_t *launches, int32_t n);
const char *hufield_profile_names(void);

/* Name of a status code. */
const char *hufield_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* HUFIELD_H */
