/*
 * ffa_oracle.c -- plain, slow, single-threaded CPU oracle of the FFA periodogram
 * (Morello et al. 2020, "Optimal periodicity searching: revisiting the Fast
 * Folding Algorithm for large scale pulsar surveys").
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * Everything is written straight from the paper, with no blocking, fusion or
 * reordering:
 *   - search plan (pseudo-octaves)      Sec. 5.3, Sec. 5.6 (tau = Pmin / bmin)
 *   - real-factor downsampling           Sec. 5.3, Appendix A.4
 *   - depth-first FFA                    Sec. 2.2, Eq. "ffa_merge_rule"
 *   - trial periods, redundant rows      Sec. 2.3, Eqs. for nu_s and P_s
 *   - boxcar S/N                         Sec. 5.4, Sec. 3.3 (Z-statistic), App. A.3
 *   - normalisation                      Sec. 3.1, Sec. 5.2 (whole-series mean/std)
 *   - running-median de-reddening        Sec. 5.2 (data whitening)
 *
 * Readings where the paper is silent (each is shared with the CUDA path as a
 * written convention, never as code):
 *   - head size  m_h = floor(m/2), tail m_t = m - m_h                (Sec. 2.2)
 *   - nearest-integer rounding is half-up, done exactly in integers  (Sec. 2.2)
 *   - "rotate towards the left by k":  (T << k)[x] = T[(x + k) mod p] (Sec. 2.2)
 *   - downsampled length is floor(n / f) complete windows            (App. A.4)
 *   - window edges i*f and (i+1)*f computed in double                (App. A.4)
 *   - octaves continue while bmin * tau_k <= Pmax; f0 < 1 is an error (Sec. 5.3)
 *   - a row s is kept iff P_s < (p+1) tau_k, i.e. s(p+1) < p(m-1)     (Sec. 2.3)
 *   - transforms with m < 2 are skipped (P_s undefined)
 *   - boxcar S/N = max_k C_k / sqrt(m * w * V_f), with V_f = f for an integer
 *     factor and f - 1/3 otherwise                                    (Sec. 5.3, App. A.4)
 *   - running median: odd window w = 2h + 1 centred on the sample; indices outside
 *     [0, n) take the nearest end sample                              (Sec. 5.2)
 */
#include "ffa_oracle_api.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Search plan (Sec. 5.3): geometric pseudo-octaves from the raw series.       */
/* ------------------------------------------------------------------------- */

static int plan_args_ok(int64_t n, double tsamp, double pmin, double pmax,
                        int bmin, int bmax)
{
    if (n <= 0 || !(tsamp > 0.0) || !(pmin > 0.0) || !(pmax > pmin)) return 0;
    if (bmin < 2 || bmax < bmin) return 0;
    /* The first factor brings the sampling time to Pmin / bmin (Sec. 5.6). */
    if (pmin / ((double)bmin * tsamp) < 1.0) return 0;
    return 1;
}

/* Downsampling factor of octave k: f0 * fg^k, fg = (bmax + 1) / bmin.        */
static double octave_factor(double tsamp, double pmin, int bmin, int bmax, int k)
{
    double f0 = pmin / ((double)bmin * tsamp);
    double fg = ((double)bmax + 1.0) / (double)bmin;
    return f0 * pow(fg, (double)k);
}

/* Number of rows s of an m-row transform with period P_s < (p+1) tau.        */
static int64_t kept_rows(int64_t m, int64_t p)
{
    int64_t s, kept = 0;
    for (s = 0; s < m; ++s)
        if (s * (p + 1) < p * (m - 1)) ++kept;
    return kept;
}

int oracle_plan(int64_t n, double tsamp, double pmin, double pmax, int bmin, int bmax,
                int max_octaves, double* oct_factor, int64_t* oct_len,
                int max_transforms, int* tr_octave, int* tr_p, int64_t* tr_m,
                int64_t* tr_kept, int64_t* tr_first_trial,
                int* n_octaves, int* n_transforms, int64_t* n_trials)
{
    int k, p, nt = 0;
    int64_t trials = 0;
    if (!plan_args_ok(n, tsamp, pmin, pmax, bmin, bmax)) return -1;
    for (k = 0;; ++k) {
        double f = octave_factor(tsamp, pmin, bmin, bmax, k);
        int64_t nk;
        if ((double)bmin * tsamp * f > pmax) break;
        nk = (int64_t)floor((double)n / f);
        if (k < max_octaves) {
            oct_factor[k] = f;
            oct_len[k] = nk;
        }
        for (p = bmin; p <= bmax; ++p) {
            int64_t m = nk / p;
            if (m < 2) continue;
            if (nt < max_transforms) {
                tr_octave[nt] = k;
                tr_p[nt] = p;
                tr_m[nt] = m;
                tr_kept[nt] = kept_rows(m, p);
                tr_first_trial[nt] = trials;
            }
            trials += kept_rows(m, p);
            ++nt;
        }
    }
    *n_octaves = k;
    *n_transforms = nt;
    *n_trials = trials;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Downsampling by a real factor f (App. A.4): output sample i adds the input  */
/* samples overlapping the window [i f, (i+1) f), each weighted by the length  */
/* of its overlap with the window.                                            */
/* ------------------------------------------------------------------------- */

int64_t oracle_downsampled_length(int64_t n, double f)
{
    if (n <= 0 || !(f >= 1.0)) return -1;
    return (int64_t)floor((double)n / f);
}

int oracle_downsample(const float* x, int64_t n, double f, double* out, int64_t nout)
{
    int64_t i, j;
    if (nout != oracle_downsampled_length(n, f)) return -1;
    for (i = 0; i < nout; ++i) {
        double a = (double)i * f;         /* window start */
        double b = (double)(i + 1) * f;   /* window end   */
        double acc = 0.0;
        for (j = (int64_t)floor(a); j < n && (double)j < b; ++j) {
            double lo = (double)j > a ? (double)j : a;
            double hi = (double)(j + 1) < b ? (double)(j + 1) : b;
            if (hi > lo) acc += (hi - lo) * (double)x[j];
        }
        out[i] = acc;
    }
    return 0;
}

/* Per-bin noise variance of a downsampled series (Sec. 5.3, App. A.4).       */
double oracle_downsampled_variance(double f)
{
    return (f == floor(f)) ? f : f - 1.0 / 3.0;
}

/* ------------------------------------------------------------------------- */
/* Depth-first FFA (Sec. 2.2).  The folding transform F of an m x p block is   */
/* built from the transforms H (first m_h rows) and T (last m_t rows):         */
/*     i = nint((m_h - 1) s / (m - 1)),  j = nint((m_t - 1) s / (m - 1)),      */
/*     b = s - (i + j),                  F_s = H_i + (T_j << (i + b)).          */
/* A one-row block is its own transform.                                       */
/* ------------------------------------------------------------------------- */

/* nint(a / d) for a >= 0, d > 0, ties rounded up, in exact integer arithmetic. */
static int64_t nint_ratio(int64_t a, int64_t d)
{
    return (2 * a + d) / (2 * d);
}

void oracle_ffa_split(int64_t m, int64_t s, int64_t* i, int64_t* j, int64_t* b)
{
    int64_t mh = m / 2, mt = m - mh;
    *i = nint_ratio((mh - 1) * s, m - 1);
    *j = nint_ratio((mt - 1) * s, m - 1);
    *b = s - (*i + *j);
}

static void ffa_f64(const double* in, int64_t m, int64_t p, double* out)
{
    int64_t mh, mt, s, x;
    double *H, *T;
    if (m == 1) {
        memcpy(out, in, (size_t)p * sizeof(double));
        return;
    }
    mh = m / 2;
    mt = m - mh;
    H = (double*)malloc((size_t)(mh * p) * sizeof(double));
    T = (double*)malloc((size_t)(mt * p) * sizeof(double));
    ffa_f64(in, mh, p, H);            /* left sub-tree first (post-order) */
    ffa_f64(in + mh * p, mt, p, T);   /* then the right sub-tree          */
    for (s = 0; s < m; ++s) {
        int64_t i, j, b, k;
        oracle_ffa_split(m, s, &i, &j, &b);
        k = (i + b) % p;
        for (x = 0; x < p; ++x)
            out[s * p + x] = H[i * p + x] + T[j * p + (x + k) % p];
    }
    free(H);
    free(T);
}

/* Same recursion with single-precision storage and one float add per element:
 * the exact sequence of additions that a bit-exact FP32 implementation must
 * reproduce. */
static void ffa_f32(const float* in, int64_t m, int64_t p, float* out)
{
    int64_t mh, mt, s, x;
    float *H, *T;
    if (m == 1) {
        memcpy(out, in, (size_t)p * sizeof(float));
        return;
    }
    mh = m / 2;
    mt = m - mh;
    H = (float*)malloc((size_t)(mh * p) * sizeof(float));
    T = (float*)malloc((size_t)(mt * p) * sizeof(float));
    ffa_f32(in, mh, p, H);
    ffa_f32(in + mh * p, mt, p, T);
    for (s = 0; s < m; ++s) {
        int64_t i, j, b, k;
        oracle_ffa_split(m, s, &i, &j, &b);
        k = (i + b) % p;
        for (x = 0; x < p; ++x)
            out[s * p + x] = H[i * p + x] + T[j * p + (x + k) % p];
    }
    free(H);
    free(T);
}

int oracle_ffa_f64(const double* in, int64_t m, int64_t p, double* out)
{
    if (m < 1 || p < 1) return -1;
    ffa_f64(in, m, p, out);
    return 0;
}

int oracle_ffa_f32(const float* in, int64_t m, int64_t p, float* out)
{
    if (m < 1 || p < 1) return -1;
    ffa_f32(in, m, p, out);
    return 0;
}

/* Trial period of row s of an m-row transform with base period p samples of
 * length tau (Sec. 2.3): P_s = p^2 / (p - s / (m - 1)) * tau. */
double oracle_trial_period(double tau, int64_t p, int64_t m, int64_t s)
{
    return tau * (double)p * (double)p / ((double)p - (double)s / (double)(m - 1));
}

/* ------------------------------------------------------------------------- */
/* Boxcar matched filter (Sec. 5.4): for every row and width w, the largest    */
/* circular boxcar sum C_k = sum_{q<w} P[(k + q) mod p] over phases k, scaled   */
/* to a unit-square-sum template over noise of standard deviation stdnoise per */
/* bin, i.e. S/N = max_k C_k / (stdnoise * sqrt(w)) (Sec. 3.3, App. A.3).      */
/* Sums are formed directly, not through prefix sums.                         */
/* ------------------------------------------------------------------------- */

int oracle_boxcar_snr(const double* prof, int64_t rows, int64_t p, const int* widths,
                      int nw, double stdnoise, double* snr)
{
    return oracle_boxcar_snr_kind(prof, rows, p, widths, nw, stdnoise, 0, snr);
}

/* kind 0: the plain boxcar (height 1/sqrt(w) on w bins, 0 elsewhere; Sec. 5.4).
 * kind 1: the zero-mean boxcar, another template with unit square sum, so that its
 *   Z-statistic (Sec. 3.3) is again N(0, 1) under pure noise (Sec. 3.5 leaves the
 *   choice of matched filters open): value a on the w on-pulse bins and b on the p - w
 *   others, with zero sum and unit square sum, i.e. a = sqrt((p - w) / (w p)),
 *   b = -sqrt(w / (p (p - w))).  The statistic at phase k is the template's dot product
 *   with the profile, a * (on-pulse sum) + b * (off-pulse sum), over the per-bin noise
 *   std; a constant added to the profile does not change it.  Needs w < p.
 * Both take the maximum over the p phases; sums are direct (no prefix sums). */
int oracle_boxcar_snr_kind(const double* prof, int64_t rows, int64_t p, const int* widths,
                           int nw, double stdnoise, int kind, double* snr)
{
    int64_t r, k, x;
    int iw;
    if (rows < 0 || p < 1 || nw < 1 || !(stdnoise > 0.0) || kind < 0 || kind > 1) return -1;
    for (iw = 0; iw < nw; ++iw)
        if (widths[iw] < 1 || widths[iw] > p || (kind == 1 && widths[iw] >= p)) return -1;
    for (r = 0; r < rows; ++r) {
        const double* P = prof + r * p;
        double total = 0.0;
        for (x = 0; x < p; ++x) total += P[x];
        for (iw = 0; iw < nw; ++iw) {
            int w = widths[iw];
            double best = -INFINITY;
            double a = 1.0 / sqrt((double)w), b = 0.0;
            if (kind == 1) {
                a = sqrt((double)(p - w) / ((double)w * (double)p));
                b = -sqrt((double)w / ((double)p * (double)(p - w)));
            }
            for (k = 0; k < p; ++k) {
                double on = 0.0, z;
                int q;
                for (q = 0; q < w; ++q) on += P[(k + q) % p];
                z = a * on + b * (total - on);
                if (z > best) best = z;
            }
            snr[r * nw + iw] = best / stdnoise;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Normalisation (Sec. 3.1, Sec. 5.2): the series is brought to zero mean and  */
/* unit standard deviation once, from statistics of the whole series.          */
/* Two passes in FP64; population standard deviation.                          */
/* ------------------------------------------------------------------------- */

int oracle_normalise(const float* x, int64_t n, double* mean, double* stdev, double* out)
{
    int64_t i;
    double s = 0.0, q = 0.0;
    if (n <= 0) return -1;
    for (i = 0; i < n; ++i) s += (double)x[i];
    *mean = s / (double)n;
    for (i = 0; i < n; ++i) {
        double d = (double)x[i] - *mean;
        q += d * d;
    }
    *stdev = sqrt(q / (double)n);
    if (out)
        for (i = 0; i < n; ++i)
            out[i] = *stdev > 0.0 ? ((double)x[i] - *mean) / *stdev : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Running median (Sec. 5.2): the low-frequency noise is removed by subtracting */
/* a running median from the series before it is normalised.  med[i] is the    */
/* median of the w = 2h + 1 samples x[i-h .. i+h]; an index before the start   */
/* reads x[0] and one after the end reads x[n-1].  The window is copied out,    */
/* sorted, and its middle element taken.                                       */
/* ------------------------------------------------------------------------- */

static int cmp_float(const void* a, const void* b)
{
    float u = *(const float*)a, v = *(const float*)b;
    return (u > v) - (u < v);
}

static float window_median(const float* x, int64_t n, int64_t h, int64_t i, float* buf)
{
    int64_t j;
    for (j = -h; j <= h; ++j) {
        int64_t t = i + j;
        buf[j + h] = x[t < 0 ? 0 : (t >= n ? n - 1 : t)];
    }
    qsort(buf, (size_t)(2 * h + 1), sizeof(float), cmp_float);
    return buf[h];
}

int oracle_running_median_at(const float* x, int64_t n, int64_t w, const int64_t* idx,
                             int64_t nidx, float* med)
{
    int64_t k;
    float* buf;
    if (n <= 0 || w < 1 || (w & 1) == 0 || nidx < 0) return -1;
    buf = (float*)malloc((size_t)w * sizeof(float));
    if (!buf) return -2;
    for (k = 0; k < nidx; ++k) {
        if (idx[k] < 0 || idx[k] >= n) { free(buf); return -1; }
        med[k] = window_median(x, n, w / 2, idx[k], buf);
    }
    free(buf);
    return 0;
}

int oracle_running_median(const float* x, int64_t n, int64_t w, float* med)
{
    int64_t i;
    float* buf;
    if (n <= 0 || w < 1 || (w & 1) == 0) return -1;
    buf = (float*)malloc((size_t)w * sizeof(float));
    if (!buf) return -2;
    for (i = 0; i < n; ++i) med[i] = window_median(x, n, w / 2, i, buf);
    free(buf);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Periodogram (Sec. 5.3, Fig. 4): for each octave, downsample the raw series, */
/* fold it at every base period p in [bmin, bmax] with the FFA, keep the rows   */
/* below the next base period, score them with every boxcar width.             */
/* Trials are emitted in (octave, p, s) order.                                 */
/*                                                                            */
/* `select` (may be NULL) is a per-transform 0/1 mask: only selected            */
/* transforms are computed, and their trials are written compactly in plan     */
/* order.  Returns the number of trials written, or -1 on error.               */
/* ------------------------------------------------------------------------- */

int64_t oracle_periodogram(const float* x, int64_t n, double tsamp, double pmin,
                           double pmax, int bmin, int bmax, const int* widths, int nw,
                           const unsigned char* select, double* periods, int* foldbins,
                           double* snr, int64_t cap)
{
    return oracle_periodogram_kind(x, n, tsamp, pmin, pmax, bmin, bmax, widths, nw, 0,
                                   select, periods, foldbins, snr, cap);
}

int64_t oracle_periodogram_kind(const float* x, int64_t n, double tsamp, double pmin,
                                double pmax, int bmin, int bmax, const int* widths, int nw,
                                int kind, const unsigned char* select, double* periods,
                                int* foldbins, double* snr, int64_t cap)
{
    int k, p, t = 0, iw;
    int64_t written = 0;
    if (!plan_args_ok(n, tsamp, pmin, pmax, bmin, bmax) || nw < 1) return -1;
    for (iw = 0; iw < nw; ++iw)
        if (widths[iw] < 1 || widths[iw] >= bmin) return -1;
    for (k = 0;; ++k) {
        double f = octave_factor(tsamp, pmin, bmin, bmax, k);
        double tau_k = tsamp * f;
        double var_f = oracle_downsampled_variance(f);
        int64_t nk;
        double* ds = NULL;
        if ((double)bmin * tsamp * f > pmax) break;
        nk = oracle_downsampled_length(n, f);
        for (p = bmin; p <= bmax; ++p) {
            int64_t m = nk / p, kept, s;
            double *fold, *s_n;
            if (m < 2) continue;
            if (select && !select[t]) { ++t; continue; }
            ++t;
            if (!ds) {
                ds = (double*)malloc((size_t)nk * sizeof(double));
                oracle_downsample(x, n, f, ds, nk);
            }
            kept = kept_rows(m, p);
            if (written + kept > cap) { free(ds); return -1; }
            fold = (double*)malloc((size_t)(m * p) * sizeof(double));
            s_n = (double*)malloc((size_t)(kept * nw) * sizeof(double));
            oracle_ffa_f64(ds, m, p, fold);
            oracle_boxcar_snr_kind(fold, kept, p, widths, nw, sqrt((double)m * var_f), kind,
                                   s_n);
            for (s = 0; s < kept; ++s) {
                periods[written + s] = oracle_trial_period(tau_k, p, m, s);
                foldbins[written + s] = p;
                memcpy(snr + (written + s) * nw, s_n + s * nw, (size_t)nw * sizeof(double));
            }
            written += kept;
            free(fold);
            free(s_n);
        }
        free(ds);
    }
    return written;
}
