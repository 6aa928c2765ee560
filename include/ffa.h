/*
 * ffa.h -- C ABI of libffa, a GB300 (sm_103a) implementation of the FFA periodogram
 * of Morello et al. 2020 ("Optimal periodicity searching: revisiting the Fast Folding
 * Algorithm for large scale pulsar surveys", arXiv:2004.03701).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers named d_* are DEVICE pointers, h_* are HOST pointers.  All memory is
 *    owned by the caller; libffa never allocates or frees device memory.  Scratch
 *    memory comes from a caller-provided workspace (d_ws, ws_bytes) whose size is
 *    queried first.  The workspace must be 256-byte aligned.
 *  - `stream` is a cudaStream_t passed as an opaque pointer (NULL = legacy default
 *    stream).  Calls that take a stream are asynchronous on it unless stated.
 *  - Every call returns an ffa_status.  Argument errors are detected on the host
 *    before anything is launched.  ffa_last_error() returns a thread-local message
 *    for the last failing call of the calling thread.  No exception and no process
 *    exit crosses this ABI.
 *  - Device-side failures (a bounded wait that ran out) set a status word inside
 *    the workspace; ffa_check() reads it.
 *  - All arrays are dense and row-major.  float is IEEE binary32, double binary64.
 */
#ifndef FFA_H
#define FFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ffa_status;
#define FFA_OK 0
#define FFA_ERR_ARG 1         /* invalid argument (null pointer, bad size, bad range) */
#define FFA_ERR_CAPACITY 2    /* output or workspace too small                        */
#define FFA_ERR_CUDA 3        /* a CUDA runtime call failed                           */
#define FFA_ERR_TIMEOUT 4     /* a bounded device-side wait ran out                   */
#define FFA_ERR_UNSUPPORTED 5 /* size outside what this build supports                */
#define FFA_ERR_DEVICE 6      /* another device-side check failed                     */

typedef int32_t ffa_dtype;
#define FFA_F32 0 /* float                                                   */
#define FFA_F16 1 /* IEEE binary16                                           */
#define FFA_I8 2  /* int8 q, value q / 16 (normalised data clipped to +-8 sigma) */

/* Thread-local text of the last error of this thread ("" if none). */
const char* ffa_last_error(void);
/* Library version string. */
const char* ffa_version(void);

/* ------------------------------------------------------------------------------
 * Real-factor downsampling (paper Sec. 5.3 and App. A.4).
 *   out[i] = sum_j x[j] * |[j, j+1) intersect [i f, (i+1) f)|,   0 <= i < n_out,
 *   n_out = floor(n / f).  Input samples that overlap the window partially are
 *   weighted by their overlap fraction.  factor >= 1.
 * d_x:     n floats (device).   d_out: out_cap floats (device).
 * n_out:   host pointer, receives floor(n / factor) (set even on FFA_ERR_CAPACITY).
 * Workspace: ffa_downsample_workspace(n) bytes (a prefix-sum of the input).
 * Accuracy: within 1e-6 of sum_j |w_j x_j| per output sample.
 * Errors: FFA_ERR_ARG (null pointers, n <= 0, factor < 1 or not finite),
 *         FFA_ERR_CAPACITY (out_cap < n_out or workspace too small).
 * ---------------------------------------------------------------------------- */
ffa_status ffa_downsample_workspace(int64_t n, size_t* bytes);
/* n_out = floor(n / factor) of a downsampling (host only), to size d_out before the
 * call.  Errors: FFA_ERR_ARG (null n_out, n <= 0, factor < 1 or not finite). */
ffa_status ffa_downsample_length(int64_t n, double factor, int64_t* n_out);
ffa_status ffa_downsample(const float* d_x, int64_t n, double factor, float* d_out,
                          int64_t out_cap, int64_t* n_out, void* d_ws, size_t ws_bytes,
                          void* stream);

/* ------------------------------------------------------------------------------
 * Folding transform of an m x p block by the depth-first FFA (paper Sec. 2.1-2.2,
 * Eq. ffa_merge_rule).  d_in and d_out are rows x cols floats (device, row-major,
 * row r = samples [r*cols, (r+1)*cols)); out row s is the profile folded along the
 * integration path drifting s bins over the block, 0 <= s < rows.  The head of an
 * n-row block is its first floor(n/2) rows; nearest-integer rounding of the split
 * is half-up; (T << k)[x] = T[(x + k) mod cols].  The result is bit-identical to
 * the recursion evaluated with one float add per element.
 * rows >= 1, cols >= 1, rows * cols < 2^31.  d_in and d_out must not overlap.
 * Workspace: ffa_transform_workspace(rows, cols) bytes.
 * Errors: FFA_ERR_ARG, FFA_ERR_CAPACITY, FFA_ERR_UNSUPPORTED (cols > 4096).
 * ---------------------------------------------------------------------------- */
ffa_status ffa_transform_workspace(int32_t rows, int32_t cols, size_t* bytes);
ffa_status ffa_transform(const float* d_in, int32_t rows, int32_t cols, float* d_out,
                         void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------
 * ffa_transform without a workspace, for callers that cannot allocate device memory
 * (plugins whose host application manages all device allocations, pipelines that
 * forbid allocation once running, code whose device memory another runtime's pool has
 * reserved).  The paper has no counterpart: this is a deployment variant of
 * ffa_transform, with the same arguments minus the workspace and the same bit-exact
 * result.
 * Scratch: a fixed 4 MiB array inside the library (per device, held by every GPU that
 * loads the library until the process exits).  Blocks that need sub-trees may have
 * rows * cols <= 1048512 floats; larger ones return FFA_ERR_CAPACITY before anything is
 * launched.  Calls no cudaMalloc, cudaFree, event creation or library allocator.
 * The first call on a device looks up the array's device address (once per device,
 * with that device current).  With CUDA's lazy module loading that first call also
 * loads the library module holding the array, which is when the runtime allocates its
 * 4 MiB on the device: make that first call before the caller's no-allocation phase
 * (and before any stream capture).  Later calls allocate nothing.
 * All calls share the one array: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.
 * ---------------------------------------------------------------------------- */
ffa_status ffa_transform_noalloc(const float* d_in, int32_t rows, int32_t cols, float* d_out,
                                 void* stream);

/* ------------------------------------------------------------------------------
 * Boxcar matched filter S/N (paper Sec. 5.4, with the Z-statistic normalisation of
 * Sec. 3.3 and App. A.3).  For each profile row r and width w = h_widths[iw]:
 *   d_snr[r * nw + iw] = max_{0<=k<cols} C_k(w) / (stdnoise * sqrt(w)),
 *   C_k(w) = sum_{q<w} prof[r][(k + q) mod cols],
 * where stdnoise is the noise standard deviation of one profile bin (for an
 * m-row transform of a series downsampled by f: sqrt(m * V_f)).
 * d_prof: rows x cols floats (device).  h_widths: nw ints (host), 1 <= w <= cols.
 * d_snr: rows x nw floats (device).  Sums are accumulated in float.
 * Errors: FFA_ERR_ARG (null pointers, rows < 0, cols < 1, nw < 1 or > 64,
 *         bad width, stdnoise <= 0), FFA_ERR_UNSUPPORTED (cols > 4096).
 * ---------------------------------------------------------------------------- */
ffa_status ffa_boxcar_snr(const float* d_prof, int32_t rows, int32_t cols,
                          const int32_t* h_widths, int32_t nw, double stdnoise,
                          float* d_snr, void* stream);
/* Same with a choice of template: boxcar = FFA_BOXCAR_PLAIN (as above) or
 * FFA_BOXCAR_ZERO_MEAN (see ffa_plan_opts below: value a on the w bins and b on the
 * others, zero sum, unit square sum; the score is max_k (a C_k + b (T - C_k)) / stdnoise
 * with T the profile's sum; widths must be below cols). */
ffa_status ffa_boxcar_snr_template(const float* d_prof, int32_t rows, int32_t cols,
                                   const int32_t* h_widths, int32_t nw, double stdnoise,
                                   int32_t boxcar, float* d_snr, void* stream);

/* ------------------------------------------------------------------------------
 * Normalisation of a whole series (paper Sec. 3.1 and Sec. 5.2): the noise mean and
 * standard deviation are estimated once from the whole series and every sample becomes
 *   x' = (x - mean) / std,
 * mean and std (population) accumulated in double.  d_mean_std (device, 2 doubles)
 * receives {mean, std}.  d_out (device) receives n values of type out_dtype:
 * FFA_F32 float, FFA_F16 binary16, FFA_I8 int8 q = clamp(rint(16 x'), -128, 127)
 * (value q / 16, i.e. clipped at +-8 sigma).  A constant series (std = 0) gives zeros.
 * Workspace: ffa_normalise_workspace(n) bytes.  Deterministic for a given n.
 * Errors: FFA_ERR_ARG (null pointers, n <= 0, bad dtype), FFA_ERR_CAPACITY.
 * ---------------------------------------------------------------------------- */
ffa_status ffa_normalise_workspace(int64_t n, size_t* bytes);
ffa_status ffa_normalise(const float* d_x, int64_t n, void* d_out, ffa_dtype out_dtype,
                         double* d_mean_std, void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------
 * Running median (paper Sec. 5.2): the low-frequency ("red") noise of a series is
 * removed by subtracting a running median before the series is normalised.
 *   med[i] = median of x[i-h .. i+h],   width = 2h + 1 (odd),
 * where an index before the start reads x[0] and one after the end reads x[n-1]
 * (the series extended by its end samples), and
 *   y[i]   = x[i] - med[i]   (one float subtraction).
 * The median is a sample of the window, found exactly (a wavelet matrix over the
 * series: every output is a range-quantile query), for any width.
 * d_x: n floats (device), finite (NaN has no order).  d_med, d_y: n floats (device),
 * either may be NULL but not both; either may equal d_x (in place), not each other.
 * Workspace: ffa_running_median_workspace(n) bytes (about 16 n), a status word first
 * (ffa_check reads it).  Deterministic.
 * Errors: FFA_ERR_ARG (null pointers, n outside [1, 2^31 - 1], even or non-positive
 *         width, d_med == d_y), FFA_ERR_CAPACITY (workspace too small).
 * ---------------------------------------------------------------------------- */
ffa_status ffa_running_median_workspace(int64_t n, size_t* bytes);
ffa_status ffa_running_median(const float* d_x, int64_t n, int64_t width, float* d_med,
                              float* d_y, void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------------
 * Peak finding on a periodogram (paper Sec. 5.5, Fig. 6), each width on its own.
 * With nu = 1 / P the trial frequencies and T = tobs the series length in seconds:
 *   - segments of dzseg / T cover [nu_lo, nu_hi] from the lowest trial frequency;
 *     segment j holds the trials with floor((nu - nu_lo) / (dzseg / T)) = j (the
 *     highest frequency falls in the last segment);
 *   - a segment of >= min_seg trials gives the control point
 *       (nu_lo + (j + 1/2) dzseg / T,  m + nsigma * (q75 - q25) / 1.349),
 *     m, q25, q75 the 50th, 25th and 75th percentiles of its S/N, interpolated linearly
 *     between order statistics (virtual index c q + (1 - q) - 1 for c values);
 *   - the threshold is the least-squares polynomial of the given degree in ln(nu)
 *     through the control points (none, and no peaks, with fewer than degree + 1);
 *   - the trials with S/N strictly above it, taken in order of decreasing frequency,
 *     form one peak until the frequency gap to the previous one exceeds clrad / T;
 *     a peak is reported as its brightest trial (the lowest index among equal S/N).
 * d_periods: ntrials doubles (device), positive and non-decreasing (the order of every
 * periodogram of this library).  d_snr: ntrials x nw floats (device, row-major).
 * d_peaks: peak_cap records (device), written width by width and, within a width, in
 * order of increasing period; peaks beyond peak_cap are counted but not written.
 * d_npeaks: nw + 1 int64 (device): peaks per width, then their total.
 * opts: NULL for the defaults (ffa_peak_opts_default).  Workspace:
 * ffa_find_peaks_workspace bytes (about 13 bytes per trial and width, 16 per trial,
 * plus 16 * max_segments * (nw + 1)).  Asynchronous; a device-side rejection (periods not
 * positive and non-decreasing: bit 16; more than max_segments segments: bit 4; a
 * segment of more than 16384 trials: bit 8, that segment gives no control point)
 * shows in ffa_check(d_ws), and a rejected call finds no peaks.
 * Errors: FFA_ERR_ARG (null pointers, ntrials outside [1, 2^32 - 1], nw outside
 *         [1, 64], tobs <= 0, bad options), FFA_ERR_CAPACITY (workspace too small).
 * ---------------------------------------------------------------------------- */
typedef struct ffa_peak_opts {
    double dzseg;          /* segment width in units of 1/T (default 5)            */
    double nsigma;         /* k of the control points m + k sigma (default 6)       */
    double clrad;          /* peak-clustering radius in units of 1/T (default 1)    */
    int32_t degree;        /* polynomial degree, 0..6 (default 2)                   */
    int32_t min_seg;       /* trials a segment needs for a control point (8)        */
    int64_t max_segments;  /* workspace bound on the segment count (65536)          */
} ffa_peak_opts;

typedef struct ffa_peak {
    int64_t trial;   /* trial index in the periodogram                               */
    double period;   /* its period (s)                                               */
    float snr;       /* its S/N                                                      */
    int32_t iw;      /* width index                                                  */
} ffa_peak;

void ffa_peak_opts_default(ffa_peak_opts* opts);
ffa_status ffa_find_peaks_workspace(int64_t ntrials, int32_t nw, const ffa_peak_opts* opts,
                                    size_t* bytes);
ffa_status ffa_find_peaks(const double* d_periods, const float* d_snr, int64_t ntrials,
                          int32_t nw, double tobs, const ffa_peak_opts* opts,
                          ffa_peak* d_peaks, int64_t peak_cap, int64_t* d_npeaks, void* d_ws,
                          size_t ws_bytes, void* stream);
/* The intermediate results of the last ffa_find_peaks on a workspace (same ntrials, nw
 * and opts), for inspection: synchronises `stream`, then copies to host memory
 *   h_nseg: the segment count;
 *   h_ctrl: min(nseg, ctrl_cap) x nw x 2 doubles {nu_j, s_j} per segment and width,
 *           s_j NaN where the segment gave no control point;
 *   h_fits: nw x 10 doubles per width {xbar, xscale, valid, c_0 .. c_6}: where valid
 *           is 1, the threshold at frequency nu is sum_a c_a u^a with
 *           u = (ln nu - xbar) / xscale (c_a is 0 past the degree).
 * Errors: FFA_ERR_ARG (null pointers, bad sizes or options), FFA_ERR_CUDA. */
ffa_status ffa_find_peaks_fits(const void* d_ws, int64_t ntrials, int32_t nw,
                               const ffa_peak_opts* opts, int64_t* h_nseg, double* h_ctrl,
                               int64_t ctrl_cap, double* h_fits, void* stream);

/* ------------------------------------------------------------------------------
 * Periodogram search plan (paper Sec. 5.3, Fig. 4; Sec. 5.6 for the first factor).
 *   f0 = pmin / (bmin * tsamp) (must be >= 1), fg = (bmax + 1) / bmin,
 *   octave k: factor F_k = f0 * fg^k while bmin * tsamp * F_k <= pmax,
 *             N_k = floor(n / F_k) samples of length tau_k = tsamp * F_k;
 *   base periods p = bmin..bmax, m = floor(N_k / p) rows (transforms with m < 2
 *   skipped); row s is kept iff P_s < (p + 1) tau_k, i.e. s (p + 1) < p (m - 1)
 *   (Sec. 2.3); P_s = tau_k p^2 / (p - s / (m - 1)).
 * Host only.  Widths: 1 <= w < bmin, strictly increasing, at most 64.
 * ---------------------------------------------------------------------------- */
/* Options of a plan.  Zero-initialised options are the default of every call without
 * options.
 * Tile shape: the work-item sizes of the persistent FFA launch; 0 means "the largest
 * that fits shared memory".  Every tile shape gives the same results, bit for bit: the
 * merges and the S/N of each row do not depend on how rows are grouped.  The Python
 * binding's `tune` times a few shapes on the caller's data and keeps the fastest.
 *   subtree_rows  rows of a shared-memory sub-tree item, 2..1024
 *   top_levels    merge levels per gathered top pass, 1..3
 *   top_rows      output rows per top-pass item, 1..128
 * Boxcar template of the S/N (both with unit square sum, so the S/N is the
 * Z-statistic of Sec. 3.3; Sec. 3.5 leaves the choice of matched filters open):
 *   FFA_BOXCAR_PLAIN      height 1/sqrt(w) on w bins, 0 elsewhere (Sec. 5.4)
 *   FFA_BOXCAR_ZERO_MEAN  value a on w bins and b on the other p - w, zero sum:
 *                         a = sqrt((p-w)/(w p)), b = -sqrt(w/(p (p-w))); a constant
 *                         added to a profile does not change its S/N
 * Out-of-range values give FFA_ERR_ARG.  The tiles have no counterpart in the paper (its
 * CPU code recurses depth first). */
enum { FFA_BOXCAR_PLAIN = 0, FFA_BOXCAR_ZERO_MEAN = 1 };

/* Tile classes: transforms of different shapes may take different tiles.  A transform
 * (m rows of p bins) takes the first class in table order with m <= m_max and
 * p <= p_max (a 0 bound admits any value); each non-zero tile field of that class
 * replaces the plan-wide one for that transform (subtree_rows stays a cap: the smaller
 * of the class's and the plan's).  Transforms that match no class keep the plan-wide
 * tiles.  In ffa_plan_info.opts the table comes back with its bounds as given and, per
 * class, the largest sub-tree, levels per top pass and rows per top item that its
 * transforms got (all 0: no transform of the plan fell in the class). */
#define FFA_MAX_TILE_CLASSES 8
typedef struct ffa_tile_class {
    int32_t m_max;
    int32_t p_max;
    int32_t subtree_rows;
    int32_t top_levels;
    int32_t top_rows;
} ffa_tile_class;

typedef struct ffa_plan_opts {
    int32_t subtree_rows;
    int32_t top_levels;
    int32_t top_rows;
    int32_t boxcar;
    int32_t nclasses;                              /* 0 .. FFA_MAX_TILE_CLASSES */
    ffa_tile_class classes[FFA_MAX_TILE_CLASSES];  /* the first nclasses are used */
} ffa_plan_opts;

typedef struct ffa_plan_info {
    int64_t ntrials;                  /* rows of the periodogram                     */
    int32_t noctaves;                 /* pseudo-octaves                              */
    int32_t ntransforms;              /* FFA transforms (octave, p)                  */
    int32_t nwidths;                  /* boxcar widths                               */
    int32_t max_rows;                 /* largest m                                   */
    int64_t downsampled_samples;      /* sum over octaves of N_k                     */
    int64_t folded_samples;           /* sum over transforms of m * p                */
    size_t workspace_bytes;           /* for ffa_periodogram                         */
    size_t host_workspace_bytes;      /* for ffa_periodogram_host (includes I/O)     */
    ffa_plan_opts opts;               /* options in effect: largest sub-tree, levels per
                                         top pass and rows per top item of the plan,
                                         boxcar template                             */
    double ffa_adds;                  /* FP32 adds of all merges (one per element of
                                         every merged row)                           */
    double snr_ops;                   /* FP32 operations of the S/N: per kept profile
                                         p prefix adds + 2 p per width               */
} ffa_plan_info;

ffa_status ffa_periodogram_plan(int64_t n, double tsamp, double pmin, double pmax,
                                int32_t bmin, int32_t bmax, const int32_t* h_widths,
                                int32_t nw, ffa_plan_info* out);
/* Same with plan options (NULL = defaults). */
ffa_status ffa_periodogram_plan_opts(int64_t n, double tsamp, double pmin, double pmax,
                                     int32_t bmin, int32_t bmax, const int32_t* h_widths,
                                     int32_t nw, const ffa_plan_opts* opts, ffa_plan_info* out);

/* ------------------------------------------------------------------------------
 * FFA periodogram (paper Sec. 5.3, Fig. 4; Sec. 5.5 for the two-dimensional output).
 * d_x: n samples (device) of a normalised series (zero mean, unit variance, Sec. 3.1
 *      and Sec. 5.2), stored as `dtype`.
 * Outputs (device), trials in (octave, p, s) order, periods strictly increasing:
 *   d_periods[t]            trial period in seconds (double)
 *   d_foldbins[t]           base period p in samples of its octave (int32)
 *   d_snr[t * nw + iw]      boxcar S/N of width h_widths[iw] (float), normalised by
 *                           sqrt(m * w * V_f), V_f = F_k if F_k is an integer else
 *                           F_k - 1/3 (App. A.4)
 * ntrials_cap >= ffa_plan_info.ntrials.  Workspace: ffa_plan_info.workspace_bytes.
 * The plan's tables are copied into the workspace on every call (from page-locked
 * host memory owned by libffa).
 * Errors: FFA_ERR_ARG, FFA_ERR_CAPACITY, FFA_ERR_UNSUPPORTED, FFA_ERR_CUDA.
 * ---------------------------------------------------------------------------- */
ffa_status ffa_periodogram(const void* d_x, ffa_dtype dtype, int64_t n, double tsamp,
                           double pmin, double pmax, int32_t bmin, int32_t bmax,
                           const int32_t* h_widths, int32_t nw, double* d_periods,
                           int32_t* d_foldbins, float* d_snr, int64_t ntrials_cap,
                           void* d_ws, size_t ws_bytes, void* stream);
/* Same with plan options (NULL = defaults); the workspace is the one that
 * ffa_periodogram_plan_opts reports for the same options.
 * All periodogram calls: the first call of a host thread on a device also creates a
 * helper stream and two events of that thread (the top-pass records are made on it,
 * concurrently with the prefix sums and downsampling, and joined back into `stream`).
 * Make that first call outside any stream capture; later calls capture as one graph
 * with a fork and a join. */
ffa_status ffa_periodogram_opts(const void* d_x, ffa_dtype dtype, int64_t n, double tsamp,
                                double pmin, double pmax, int32_t bmin, int32_t bmax,
                                const int32_t* h_widths, int32_t nw, const ffa_plan_opts* opts,
                                double* d_periods, int32_t* d_foldbins, float* d_snr,
                                int64_t ntrials_cap, void* d_ws, size_t ws_bytes, void* stream);
/* Diagnostics of the persistent FFA launch (the paper has no counterpart): synchronises
 * `stream` and copies to host memory the work-item records that the last
 * ffa_periodogram[_opts] call with the same search and options made in d_ws, one per
 * queue position in queue order, 8 int32 each: {transform, node or block index, pass
 * (-2 whole tree, -1 sub-tree, >= 0 top pass), scratch batch (-1: none), counter waited
 * for (-1: none), count needed, counter released on completion (-1: none), sub-tree
 * depth}.  min(cap, items) records are written; *nitems receives the item count.  Every
 * wait ends if the items releasing a counter come before its waiters in the queue (CTAs
 * claim positions in order).  Errors: FFA_ERR_ARG, FFA_ERR_CAPACITY (workspace smaller
 * than the plan's), FFA_ERR_CUDA. */
ffa_status ffa_periodogram_queue(int64_t n, double tsamp, double pmin, double pmax, int32_t bmin,
                                 int32_t bmax, const int32_t* h_widths, int32_t nw,
                                 const ffa_plan_opts* opts, const void* d_ws, size_t ws_bytes,
                                 int32_t* h_out, int64_t cap, int64_t* nitems, void* stream);

/* ------------------------------------------------------------------------------
 * Batched periodograms (many series, e.g. the dedispersed DM trials of an observation,
 * searched like the paper's pipeline does per DM trial, Sec. 5.7).  Series i is
 * samples [offset, offset + n) of d_x and has its own sampling time, period range and
 * bins range; the widths are shared (each below every series' bmin).  Outputs are the
 * periodograms of the series one after another (h_trial_offsets[i] = first trial of
 * series i, h_trial_offsets[nseries] = total).  The series are cut into consecutive
 * chunks whose workspace each fits ws_budget bytes (a series alone may exceed it);
 * each chunk runs as prefix sums, downsampling and one persistent FFA launch over all
 * its transforms, in the chunk order on `stream`, reusing one workspace of
 * ffa_batch_info.workspace_bytes.  d_x must span max(offset + n) elements of dtype.
 * ---------------------------------------------------------------------------- */
typedef struct ffa_series {
    int64_t offset;   /* first sample of the series in d_x (elements) */
    int64_t n;        /* samples */
    double tsamp;     /* seconds */
    double pmin, pmax;
    int32_t bmin, bmax;
} ffa_series;

typedef struct ffa_batch_info {
    int64_t ntrials;          /* rows of all periodograms              */
    int32_t nchunks;          /* launch sequences                      */
    int32_t ntransforms;      /* FFA transforms over all series        */
    int64_t folded_samples;   /* sum of m * p                          */
    int64_t input_samples;    /* sum of n                              */
    size_t workspace_bytes;   /* for ffa_periodogram_batch             */
} ffa_batch_info;

ffa_status ffa_batch_plan(const ffa_series* h_series, int32_t nseries, const int32_t* h_widths,
                          int32_t nw, size_t ws_budget, int64_t* h_trial_offsets,
                          ffa_batch_info* out);
ffa_status ffa_periodogram_batch(const void* d_x, ffa_dtype dtype, const ffa_series* h_series,
                                 int32_t nseries, const int32_t* h_widths, int32_t nw,
                                 size_t ws_budget, double* d_periods, int32_t* d_foldbins,
                                 float* d_snr, int64_t ntrials_cap, void* d_ws, size_t ws_bytes,
                                 void* stream);
/* Same two calls with plan options for every chunk (NULL = defaults). */
ffa_status ffa_batch_plan_opts(const ffa_series* h_series, int32_t nseries,
                               const int32_t* h_widths, int32_t nw, size_t ws_budget,
                               const ffa_plan_opts* opts, int64_t* h_trial_offsets,
                               ffa_batch_info* out);
ffa_status ffa_periodogram_batch_opts(const void* d_x, ffa_dtype dtype,
                                      const ffa_series* h_series, int32_t nseries,
                                      const int32_t* h_widths, int32_t nw, size_t ws_budget,
                                      const ffa_plan_opts* opts, double* d_periods,
                                      int32_t* d_foldbins, float* d_snr, int64_t ntrials_cap,
                                      void* d_ws, size_t ws_bytes, void* stream);

/* Plans (single-series and batch) are built on first use and cached by their parameters
 * for the life of the process: their page-locked tables are what the table copy of
 * every call, and of every CUDA graph that captured a call, reads.  This releases them
 * all; call it only when no call is in flight and no captured graph that contains one
 * will be launched again. */
ffa_status ffa_plan_cache_clear(void);

/* Same search, end to end from and to HOST buffers: copies h_x (n floats) to the
 * device, runs the periodogram, copies the three outputs back, and synchronises
 * `stream` before returning.  Host buffers should be page-locked for speed.
 * Workspace: ffa_plan_info.host_workspace_bytes. */
ffa_status ffa_periodogram_host(const float* h_x, int64_t n, double tsamp, double pmin,
                                double pmax, int32_t bmin, int32_t bmax,
                                const int32_t* h_widths, int32_t nw, double* h_periods,
                                int32_t* h_foldbins, float* h_snr, int64_t ntrials_cap,
                                void* d_ws, size_t ws_bytes, void* stream);

/* Synchronises `stream`, reads and clears the device status word of a workspace used
 * by ffa_periodogram / ffa_transform / ffa_downsample / ffa_running_median /
 * ffa_find_peaks.  FFA_OK if no
 * device-side check failed, else FFA_ERR_TIMEOUT or FFA_ERR_DEVICE (the message names
 * the failed checks). */
ffa_status ffa_check(void* d_ws, void* stream);

/* Bounds-checked debug build.  The library compiled with FFA_CHECKED (built beside the
 * normal one as libffa_checked.so; same entry points, same results) checks every
 * shared-memory range and global index its kernels compute from runtime data before
 * use: a violation skips the access (or the whole work item) and sets bit 32 in the
 * status word, which ffa_check reports as FFA_ERR_DEVICE ("an index out of range").
 * *checked: 1 in that build, 0 in the normal one.  *bits: synchronises the device and
 * returns (and clears) bit 32 if any kernel of the library found a violation since the
 * last call, whatever workspace (or none, as for the standalone boxcar S/N) the launch
 * had; always 0 in the normal build.  Errors: FFA_ERR_ARG (null pointer), FFA_ERR_CUDA. */
ffa_status ffa_checked_status(int32_t* checked, uint32_t* bits);

/* Limit of every device-side wait of a periodogram launch (a CTA waiting for the items
 * an item depends on, or for its own bulk copies), in milliseconds of SM clock at the
 * maximum clock; default 1000.  A wait that runs out sets FFA_ERR_TIMEOUT in the status
 * word and the launch ends early (its outputs are then incomplete).  Process-wide; takes
 * effect from the next call.  Errors: FFA_ERR_ARG (ms <= 0 or ms > 60000).
 *
 * Fault injection for tests: the environment variable FFA_FAULT, read at every call,
 * makes calls fail on purpose, always without a device fault: "plan" (plan building:
 * FFA_ERR_UNSUPPORTED), "alloc" (the page-locked table allocation: FFA_ERR_CUDA),
 * "launch" (the launch sequence, before any CUDA call: FFA_ERR_CUDA), "stage" (one
 * transform's second stage waits for one item more than exist: the wait runs out after
 * the wait limit and ffa_check reports FFA_ERR_TIMEOUT). */
ffa_status ffa_set_wait_limit_ms(double ms);

/* ------------------------------------------------------------------------------
 * Launch accounting and per-kernel timing (for benchmarks).  When enabled, every
 * kernel launch of this library is bracketed by CUDA events on its stream.
 * Not to be enabled while a stream is being captured into a graph.
 * ---------------------------------------------------------------------------- */
int64_t ffa_launch_count(void);          /* kernels launched by this process so far */
int32_t ffa_kernel_kinds(void);          /* number of kernel kinds                  */
const char* ffa_kernel_name(int32_t kind);
ffa_status ffa_profile_enable(int32_t on);
ffa_status ffa_profile_reset(void);
/* Synchronises the recorded events; returns launches, summed device time (ms) and
 * summed algorithmic bytes (reads + writes of the data the method must touch) of
 * one kernel kind since the last reset. */
ffa_status ffa_profile_query(int32_t kind, int64_t* launches, double* total_ms,
                             double* alg_bytes);

#ifdef __cplusplus
}
#endif
#endif /* FFA_H */
