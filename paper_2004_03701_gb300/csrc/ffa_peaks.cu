// ffa_peaks.cu -- peak finding on a periodogram (paper Sec. 5.5, Fig. 6) for sm_103a.
//
// Each width's S/N column is searched on its own.  The trial-frequency range is cut
// into segments of dzseg / T; the median m and sigma = IQR / 1.349 of the S/N in each
// segment give a control point (nu_j, m + k sigma); a least-squares polynomial in
// ln(nu) through the control points is the selection threshold; trials above it are
// grouped into peaks along decreasing frequency, a new peak starting where the
// frequency gap to the previous selected trial exceeds clrad / T, and each peak is
// reported as its brightest trial.
//
// Launches (all on the caller's stream, no host synchronisation):
//   pk_prep_kernel     per trial: input checks, nu = 1 / P and ln nu, once (FP64 divides
//                      and logarithms are slow on this GPU: nothing later repeats them);
//   pk_range_kernel    one thread: frequency range (the ends of the sorted trials) and
//                      segment count;
//   pk_bounds_kernel   per segment, its first trial (binary search: the segments fall
//                      with the trial index, periods being non-decreasing);
//   pk_segment_kernel  one CTA per (segment, 4 widths): the S/N values of each width are
//                      sorted in shared memory (bitonic) and the quartiles interpolated
//                      linearly between order statistics;
//   pk_fit_kernel      one CTA per width: normal equations of the polynomial in the
//                      centred and scaled log frequency, solved by Gaussian elimination
//                      with partial pivoting, in FP64;
//   pk_count_kernel,   selection of the trials above the threshold, in chunks of 4096
//   pk_offsets_kernel, trials per (chunk, width): flags and counts, their prefix per
//   pk_write_kernel    width, and the selected trials written in order;
//   pk_cluster_kernel  one CTA per width: peaks along the selected trials (block scans)
//                      and the brightest trial of every peak;
//   pk_output_kernel   one CTA: widths' peaks packed width by width into the output.
// The control points are computed with the same FP64 operations, in the same order, as
// a plain evaluation (no fused multiply-adds), so they are reproducible bit for bit.
#include "ffa.h"
#include "ffa_internal.h"
#include "ffa_kinds.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

namespace ffa {
ffa_status set_error(ffa_status st, const char* msg);
}

namespace {

using ffa::LaunchScope;

constexpr int kPrepThreads = 256;
constexpr int kSegThreads = 512;
constexpr int kSortCap = 16384;  // trials of one segment sorted in shared memory
constexpr int kFitThreads = 256;
constexpr int kSelThreads = 1024;
constexpr int kSelPer = 4;                      // trials per thread of a selection chunk
constexpr int kSelTile = kSelThreads * kSelPer;
constexpr int kMaxDegree = 6;
constexpr int kSegGrid = 152 * 8;
constexpr int kGroupW = 4;       // widths per segment work item

// device status bits of the peak finder (first word of its workspace)
constexpr unsigned kPkTooManySegments = 4u;
constexpr unsigned kPkSegmentTooLarge = 8u;
constexpr unsigned kPkBadPeriods = 16u;

struct Hdr {
    double nu_lo, width;
    long long nseg;  // 0 when the input was rejected on the device
};

struct Fit {
    double xbar, xscale, inv_xscale;
    double c[kMaxDegree + 1];  // threshold = sum_a c[a] u^a, u = (ln nu - xbar) / xscale
    int valid;
};

struct Params {
    const double* periods;
    double* nu;          // [ntrials]: 1 / P
    double* lnnu;        // [ntrials]: ln(1 / P)
    uint8_t* flags;      // [ntrials][nw]: selected (the S/N's layout)
    long long* first;    // [max_segments]: first trial of segment <= j
    const float* snr;
    long long ntrials;
    int nw;
    double width, nsigma, gap;
    int degree, min_seg;
    long long max_segments;
    unsigned* status;
    Hdr* hdr;
    double2* ctrl;       // [max_segments][nw]: {nu_j, s_j}, s_j NaN without a point
    Fit* fit;            // [nw]
    uint32_t* list;      // [nw][ntrials]: selected trials, in order
    uint64_t* best;      // [nw][ntrials]: per peak, the brightest trial's key
    long long* counts;   // [nw][2]: selected trials, peaks
    long long nchunks;   // selection chunks of kSelTile trials
    long long* ccount;   // [nw][nchunks]: selected trials per chunk
    long long* coff;     // [nw][nchunks]: their exclusive prefix
};

// Checked builds: false (and the status bit set) when `ok` fails.
__device__ __forceinline__ bool ck(bool ok, unsigned* status) {
    if (!ffa::kChecked || ok) return true;
    ffa::bounds_violation(status);
    return false;
}

__device__ __forceinline__ long long seg_of(double nu, const Hdr& h) {
    const long long j = (long long)floor(__ddiv_rn(__dsub_rn(nu, h.nu_lo), h.width));
    return j < h.nseg - 1 ? j : h.nseg - 1;
}

// reduction over the block; `id` is the identity of `op` (fills the missing warps)
template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T id, T* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nwarps ? sh[lane] : id;
        for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sh[0] = v;
    }
    __syncthreads();
    const T r = sh[0];
    __syncthreads();
    return r;
}

// exclusive block scan of one value per thread
__device__ long long block_scan(long long v, long long* sh, long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    __syncthreads();
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < nwarps ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        sh[lane] = w;
    }
    __syncthreads();
    const long long ex = inc - v + (warp ? sh[warp - 1] : 0);
    *total = sh[nwarps - 1];
    __syncthreads();
    return ex;
}

struct AddOp {
    __device__ double operator()(double a, double b) const { return a + b; }
};

__global__ void __launch_bounds__(kPrepThreads) pk_prep_kernel(Params p) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.ntrials) return;
    const double P = p.periods[t];
    bool bad = !(P > 0.0) || !isfinite(P);
    if (t + 1 < p.ntrials && !(P <= p.periods[t + 1])) bad = true;
    if (bad) atomicOr(p.status, kPkBadPeriods);
    const double nu = __ddiv_rn(1.0, P);
    p.nu[t] = nu;
    p.lnnu[t] = log(nu);
}

// The trial frequencies fall with the trial index (periods checked non-decreasing), so
// the range is their two ends.
__global__ void pk_range_kernel(Params p) {
    if (threadIdx.x != 0) return;
    const double lo = p.nu[p.ntrials - 1], hi = p.nu[0];
    const double q = ceil(__ddiv_rn(__dsub_rn(hi, lo), p.width));
    long long nseg = q > 1.0 ? (long long)q : 1;
    if (*p.status & kPkBadPeriods) {
        nseg = 0;
    } else if (!(q <= (double)p.max_segments)) {
        atomicOr(p.status, kPkTooManySegments);
        nseg = 0;
    }
    p.hdr->nu_lo = lo;
    p.hdr->width = p.width;
    p.hdr->nseg = nseg;
}

// Linear interpolation between order statistics, as the "linear" sample quantile of
// Hyndman and Fan (their definition 7): virtual index c q + (1 - q) - 1.
__device__ double quantile(const float* v, long long c, double q) {
    const double vi = __dsub_rn(__dadd_rn(__dmul_rn((double)c, q), __dsub_rn(1.0, q)), 1.0);
    const double prev = floor(vi);
    long long i0 = (long long)prev, i1 = i0 + 1;
    if (i0 > c - 1) i0 = c - 1;
    if (i1 > c - 1) i1 = c - 1;
    const double g = __dsub_rn(vi, prev);
    const double a = (double)v[i0], b = (double)v[i1];
    const double d = __dsub_rn(b, a);
    return g >= 0.5 ? __dsub_rn(b, __dmul_rn(d, __dsub_rn(1.0, g))) : __dadd_rn(a, __dmul_rn(d, g));
}

// first[j] = the first trial whose segment is <= j (segments fall with the trial index),
// so segment j is [first[j], first[j - 1]) with first[-1] = ntrials.
__global__ void __launch_bounds__(256) pk_bounds_kernel(Params p) {
    const Hdr h = *p.hdr;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < h.nseg;
         j += (long long)gridDim.x * blockDim.x) {
        long long a = 0, b = p.ntrials;
        while (a < b) {
            const long long m = (a + b) >> 1;
            if (seg_of(p.nu[m], h) <= j)
                b = m;
            else
                a = m + 1;
        }
        if (ck(j < p.max_segments, p.status)) p.first[j] = a;
    }
}

// Work items of (segment, group of kGroupW widths): the rows of the segment are read
// once per group (coalesced across its widths), as many widths as fit shared memory are
// sorted together (independent bitonic networks, one comparator per thread and step),
// and one thread per width interpolates its quartiles.
__global__ void __launch_bounds__(kSegThreads) pk_segment_kernel(Params p) {
    extern __shared__ float v[];
    const Hdr h = *p.hdr;
    const int nw = p.nw;
    const int ngroups = (nw + kGroupW - 1) / kGroupW;
    const long long nitems = h.nseg * ngroups;
    for (long long q = blockIdx.x; q < nitems; q += gridDim.x) {
        const long long j = q / ngroups;
        const int wa = (int)(q - j * ngroups) * kGroupW;
        const int wb = wa + kGroupW < nw ? wa + kGroupW : nw;
        const long long t0 = p.first[j], t1 = j ? p.first[j - 1] : p.ntrials;
        const long long c = t1 - t0;
        if (ffa::kChecked &&  // uniform
            !ck(j < p.max_segments && t0 >= 0 && t0 <= t1 && t1 <= p.ntrials, threadIdx.x ? nullptr : p.status))
            continue;
        const double nu_c = __dadd_rn(h.nu_lo, __dmul_rn((double)j + 0.5, h.width));
        if (c < p.min_seg || c > kSortCap) {
            if (threadIdx.x == 0 && c > kSortCap) atomicOr(p.status, kPkSegmentTooLarge);
            for (int iw = wa + threadIdx.x; iw < wb; iw += blockDim.x)
                p.ctrl[j * nw + iw] = make_double2(nu_c, __longlong_as_double(0x7ff8000000000000LL));
            continue;
        }
        int lm = 0;
        while ((1LL << lm) < c) ++lm;
        const int m = 1 << lm;
        const int G = kSortCap >> lm;  // widths per pass
        if (ffa::kChecked &&
            !ck((long long)G * m <= ffa::dyn_smem_floats(), threadIdx.x ? nullptr : p.status))
            continue;
        for (int w0 = wa; w0 < wb; w0 += G) {
            const int gn = wb - w0 < G ? wb - w0 : G;
            __syncthreads();  // the previous pass's quartiles are read
            for (int e = threadIdx.x; e < gn * m; e += blockDim.x) {
                const int i = e / gn, g = e - i * gn;
                v[g * m + i] = i < c ? p.snr[(t0 + i) * nw + w0 + g] : INFINITY;
            }
            __syncthreads();
            const int half = m >> 1, ncmp = gn * half;
            for (int k = 2; k <= m; k <<= 1) {
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    for (int cq = threadIdx.x; cq < ncmp; cq += blockDim.x) {
                        const int g = cq >> (lm - 1), r = cq & (half - 1);
                        const int i = ((r & ~(jj - 1)) << 1) | (r & (jj - 1));  // bit jj clear
                        float* w = v + g * m;
                        const float x = w[i], y = w[i + jj];
                        if ((x > y) == ((i & k) == 0)) {
                            w[i] = y;
                            w[i + jj] = x;
                        }
                    }
                    __syncthreads();
                }
            }
            if (threadIdx.x < gn) {
                const float* w = v + threadIdx.x * m;
                const double q25 = quantile(w, c, 0.25), q50 = quantile(w, c, 0.5),
                             q75 = quantile(w, c, 0.75);
                const double sigma = __ddiv_rn(__dsub_rn(q75, q25), 1.349);
                p.ctrl[j * nw + w0 + threadIdx.x] =
                    make_double2(nu_c, __dadd_rn(q50, __dmul_rn(p.nsigma, sigma)));
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kFitThreads) pk_fit_kernel(Params p) {
    __shared__ double shd[32];
    __shared__ double s_sum[3 * kMaxDegree + 3];
    const int iw = blockIdx.x;
    const long long nseg = p.hdr->nseg;
    const int d = p.degree, na = d + 1;
    // pass 1: count, mean and spread of x = ln(nu) over the control points
    double cnt = 0.0, sx = 0.0;
    for (long long j = threadIdx.x; j < nseg; j += blockDim.x) {
        const double2 c = p.ctrl[j * p.nw + iw];
        if (!isnan(c.y)) {
            cnt += 1.0;
            sx += log(c.x);
        }
    }
    cnt = block_reduce(cnt, AddOp(), 0.0, shd);
    sx = block_reduce(sx, AddOp(), 0.0, shd);
    Fit* f = p.fit + iw;
    if (cnt < (double)na) {
        if (threadIdx.x == 0) f->valid = 0;
        return;
    }
    const double xbar = sx / cnt;
    double sq = 0.0;
    for (long long j = threadIdx.x; j < nseg; j += blockDim.x) {
        const double2 c = p.ctrl[j * p.nw + iw];
        if (!isnan(c.y)) {
            const double u = log(c.x) - xbar;
            sq += u * u;
        }
    }
    sq = block_reduce(sq, AddOp(), 0.0, shd);
    const double xs = sq > 0.0 ? sqrt(sq / cnt) : 1.0;
    // pass 2: sums of u^a (a <= 2d) and u^a s (a <= d)
    double acc[3 * kMaxDegree + 3];
    for (int a = 0; a < 3 * kMaxDegree + 3; ++a) acc[a] = 0.0;
    for (long long j = threadIdx.x; j < nseg; j += blockDim.x) {
        const double2 c = p.ctrl[j * p.nw + iw];
        if (isnan(c.y)) continue;
        const double u = (log(c.x) - xbar) / xs;
        double pw = 1.0;
        for (int a = 0; a <= 2 * d; ++a) {
            acc[a] += pw;
            if (a <= d) acc[2 * kMaxDegree + 1 + a] += pw * c.y;
            pw *= u;
        }
    }
    for (int a = 0; a < 3 * kMaxDegree + 3; ++a) {
        const bool used = a <= 2 * d || (a >= 2 * kMaxDegree + 1 && a <= 2 * kMaxDegree + 1 + d);
        if (!used) continue;
        const double t = block_reduce(acc[a], AddOp(), 0.0, shd);
        if (threadIdx.x == 0) s_sum[a] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // normal equations A c = r, A[i][k] = sum u^(i+k), r[i] = sum u^i s
    double A[kMaxDegree + 1][kMaxDegree + 2];
    for (int i = 0; i < na; ++i) {
        for (int k = 0; k < na; ++k) A[i][k] = s_sum[i + k];
        A[i][na] = s_sum[2 * kMaxDegree + 1 + i];
    }
    for (int col = 0; col < na; ++col) {
        int piv = col;
        for (int r = col + 1; r < na; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int k = 0; k <= na; ++k) {
                const double t = A[col][k];
                A[col][k] = A[piv][k];
                A[piv][k] = t;
            }
        if (A[col][col] == 0.0) {
            f->valid = 0;
            return;
        }
        for (int r = col + 1; r < na; ++r) {
            const double m = A[r][col] / A[col][col];
            for (int k = col; k <= na; ++k) A[r][k] -= m * A[col][k];
        }
    }
    for (int i = na - 1; i >= 0; --i) {
        double s = A[i][na];
        for (int k = i + 1; k < na; ++k) s -= A[i][k] * f->c[k];
        f->c[i] = s / A[i][i];
    }
    f->xbar = xbar;
    f->xscale = xs;
    f->inv_xscale = 1.0 / xs;
    f->valid = 1;
}

__device__ __forceinline__ double threshold(const Fit& f, int d, double lnnu) {
    const double u = (lnnu - f.xbar) * f.inv_xscale;
    double t = f.c[d];
    for (int a = d - 1; a >= 0; --a) t = t * u + f.c[a];
    return t;
}

// order-preserving key of a float S/N, with the lower trial index winning ties
__device__ __forceinline__ uint64_t best_key(float s, long long t) {
    uint32_t u = __float_as_uint(s);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((uint64_t)u << 32) | (uint64_t)(0xffffffffu - (uint32_t)t);
}

// Selection over chunks of kSelTile consecutive trials, all widths per CTA, one trial
// per thread and step (its S/N row read whole): a trial is selected for a width when
// its S/N is strictly above that width's threshold.  The threshold is first evaluated in
// FP32; only an S/N within a guard band of it (1e-3 (1 + |threshold|), far above the
// FP32 evaluation's error) is decided by the FP64 polynomial, so every decision is the
// FP64 one.  Flags are kept in the S/N's layout; counts per (chunk, width).
struct Fit32 {
    float xbar, inv, c[kMaxDegree + 1];
};

__global__ void __launch_bounds__(kSelThreads) pk_count_kernel(Params p) {
    __shared__ Fit s_fit[ffa::kMaxWidths];
    __shared__ Fit32 s_f32[ffa::kMaxWidths];
    __shared__ unsigned s_cnt[ffa::kMaxWidths];
    const int nw = p.nw, d = p.degree;
    const bool live = p.hdr->nseg != 0;
    for (int iw = threadIdx.x; iw < nw; iw += blockDim.x) {
        const Fit f = p.fit[iw];
        s_fit[iw] = f;
        Fit32 g;
        g.xbar = (float)f.xbar;
        g.inv = (float)f.inv_xscale;
        for (int a = 0; a <= kMaxDegree; ++a) g.c[a] = (float)f.c[a];
        s_f32[iw] = g;
        s_cnt[iw] = 0;
    }
    __syncthreads();
    const long long t0 = (long long)blockIdx.x * kSelTile;
    const long long t1 = t0 + kSelTile < p.ntrials ? t0 + kSelTile : p.ntrials;
    for (long long t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const double ln = p.lnnu[t];
        const float l32 = (float)ln;
        const float* S = p.snr + t * nw;
        uint8_t* fl = p.flags + t * nw;
        for (int iw = 0; iw < nw; ++iw) {
            const float s = S[iw];
            bool sel = false;
            if (live && s_fit[iw].valid) {
                const Fit32& g = s_f32[iw];
                const float u = (l32 - g.xbar) * g.inv;
                float th = g.c[d];
                for (int a = d - 1; a >= 0; --a) th = fmaf(th, u, g.c[a]);
                const float guard = 1e-3f * (1.0f + fabsf(th));
                if (s > th + guard)
                    sel = true;
                else if (s >= th - guard)
                    sel = (double)s > threshold(s_fit[iw], d, ln);
            }
            fl[iw] = sel;
            if (sel) atomicAdd(s_cnt + iw, 1u);
        }
    }
    __syncthreads();
    for (int iw = threadIdx.x; iw < nw; iw += blockDim.x)
        p.ccount[(size_t)iw * p.nchunks + blockIdx.x] = s_cnt[iw];
}

__global__ void __launch_bounds__(kSelThreads) pk_offsets_kernel(Params p) {
    __shared__ long long shl[32];
    const int iw = blockIdx.x;
    long long* cnt = p.counts + 2 * iw;
    if (p.hdr->nseg == 0 || !p.fit[iw].valid) {
        if (threadIdx.x == 0) cnt[0] = cnt[1] = 0;
        return;
    }
    const long long n = p.nchunks;
    const long long per = (n + blockDim.x - 1) / blockDim.x;
    const long long a0 = threadIdx.x * per, a1 = a0 + per < n ? a0 + per : n;
    const long long* cc = p.ccount + (size_t)iw * n;
    long long* co = p.coff + (size_t)iw * n;
    long long mine = 0;
    for (long long i = a0; i < a1; ++i) mine += cc[i];
    long long total;
    long long run = block_scan(mine, shl, &total);
    for (long long i = a0; i < a1; ++i) {
        co[i] = run;
        run += cc[i];
    }
    if (threadIdx.x == 0) cnt[0] = total;
}

__global__ void __launch_bounds__(kSelThreads) pk_write_kernel(Params p) {
    __shared__ long long shl[32];
    const int iw = blockIdx.y;
    const Fit f = p.fit[iw];
    if (p.hdr->nseg == 0 || !f.valid) return;
    bool sel[kSelPer];
    long long k = 0;
#pragma unroll
    for (int u = 0; u < kSelPer; ++u) {
        const long long t = (long long)blockIdx.x * kSelTile + (long long)threadIdx.x * kSelPer + u;
        sel[u] = t < p.ntrials && p.flags[t * p.nw + iw];
        k += sel[u];
    }
    long long tot;
    long long off = p.coff[(size_t)iw * p.nchunks + blockIdx.x] + block_scan(k, shl, &tot);
    uint32_t* L = p.list + (size_t)iw * p.ntrials;
#pragma unroll
    for (int u = 0; u < kSelPer; ++u)
        if (sel[u] && ck(off >= 0 && off < p.ntrials, p.status))
            L[off++] = (uint32_t)((long long)blockIdx.x * kSelTile + threadIdx.x * kSelPer + u);
}

// Peaks of one width: the selected trials in order (decreasing frequency) split where the
// frequency gap exceeds clrad / T; each peak keeps its brightest trial.
__global__ void __launch_bounds__(kSelThreads) pk_cluster_kernel(Params p) {
    __shared__ long long shl[32];
    const int iw = blockIdx.x;
    long long* cnt = p.counts + 2 * iw;
    if (p.hdr->nseg == 0 || !p.fit[iw].valid) return;
    const long long nsel = cnt[0];
    if (ffa::kChecked && !ck(nsel >= 0 && nsel <= p.ntrials, threadIdx.x ? nullptr : p.status))
        return;  // uniform
    const uint32_t* L = p.list + (size_t)iw * p.ntrials;
    uint64_t* B = p.best + (size_t)iw * p.ntrials;
    const long long per = (nsel + blockDim.x - 1) / blockDim.x;
    const long long e0 = threadIdx.x * per, e1 = e0 + per < nsel ? e0 + per : nsel;
    auto starts = [&](long long e) {
        if (e == 0) return true;
        if (ffa::kChecked && !ck(L[e - 1] < p.ntrials && L[e] < p.ntrials, p.status)) return false;
        const double gp = __dsub_rn(p.nu[L[e - 1]], p.nu[L[e]]);
        return gp > p.gap;
    };
    long long ns = 0;
    for (long long e = e0; e < e1; ++e) ns += starts(e);
    long long npk;
    const long long cbase = block_scan(ns, shl, &npk);
    for (long long c = threadIdx.x; c < npk; c += blockDim.x) B[c] = 0;
    __syncthreads();
    // a running maximum per thread, flushed when its peak changes
    long long cid = cbase - 1;
    uint64_t run = 0;
    for (long long e = e0; e < e1; ++e) {
        if (starts(e)) {
            if (cid >= 0 && run) atomicMax((unsigned long long*)(B + cid), (unsigned long long)run);
            ++cid;
            run = 0;
        }
        const long long t = L[e];
        if (ffa::kChecked && !(ck(t < p.ntrials, p.status) && ck(cid >= 0 && cid < npk, p.status)))
            continue;
        const uint64_t k = best_key(p.snr[t * p.nw + iw], t);
        run = k > run ? k : run;
    }
    if (cid >= 0 && run) atomicMax((unsigned long long*)(B + cid), (unsigned long long)run);
    if (threadIdx.x == 0) cnt[1] = npk;
}

__global__ void __launch_bounds__(1024) pk_output_kernel(Params p, ffa_peak* out, long long cap,
                                                         long long* npeaks) {
    long long base = 0;
    for (int iw = 0; iw < p.nw; ++iw) {
        const long long np = p.counts[2 * iw + 1];
        const uint64_t* B = p.best + (size_t)iw * p.ntrials;
        for (long long c = threadIdx.x; c < np; c += blockDim.x) {
            if (base + c >= cap) break;
            const long long t = (long long)(0xffffffffu - (uint32_t)(B[c] & 0xffffffffu));
            if (ffa::kChecked && !ck(c < p.ntrials && t < p.ntrials, p.status)) continue;
            ffa_peak pk;
            pk.trial = t;
            pk.period = p.periods[t];
            pk.snr = p.snr[t * p.nw + iw];
            pk.iw = iw;
            out[base + c] = pk;
        }
        if (threadIdx.x == 0) npeaks[iw] = np;
        base += np;
    }
    if (threadIdx.x == 0) npeaks[p.nw] = base;
}

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
    size_t status, hdr, ctrl, fit, list, best, counts, ccount, coff, nu, lnnu, flags, first, bytes;
};

Layout layout(long long ntrials, int nw, long long max_segments) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off += up256(b);
        return o;
    };
    L.status = take(sizeof(unsigned));
    L.hdr = take(sizeof(Hdr));
    L.ctrl = take(sizeof(double2) * (size_t)max_segments * nw);
    L.fit = take(sizeof(Fit) * nw);
    L.list = take(sizeof(uint32_t) * (size_t)ntrials * nw);
    L.best = take(sizeof(uint64_t) * (size_t)ntrials * nw);
    L.counts = take(sizeof(long long) * 2 * nw);
    const size_t nchunks = (size_t)((ntrials + kSelTile - 1) / kSelTile);
    L.ccount = take(sizeof(long long) * nchunks * nw);
    L.coff = take(sizeof(long long) * nchunks * nw);
    L.nu = take(sizeof(double) * (size_t)ntrials);
    L.lnnu = take(sizeof(double) * (size_t)ntrials);
    L.flags = take((size_t)ntrials * nw);
    L.first = take(sizeof(long long) * (size_t)max_segments);
    L.bytes = off;
    return L;
}

ffa_peak_opts defaults() {
    ffa_peak_opts o;
    o.dzseg = 5.0;
    o.nsigma = 6.0;
    o.clrad = 1.0;
    o.degree = 2;
    o.min_seg = 8;
    o.max_segments = 1 << 16;
    return o;
}

ffa_status check_opts(const ffa_peak_opts& o) {
    if (!(o.dzseg > 0.0) || !std::isfinite(o.dzseg))
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: dzseg must be > 0");
    if (!std::isfinite(o.nsigma))
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: nsigma must be finite");
    if (!(o.clrad >= 0.0) || !std::isfinite(o.clrad))
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: clrad must be >= 0");
    if (o.degree < 0 || o.degree > kMaxDegree)
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: degree must be in [0, 6]");
    if (o.min_seg < 1 || o.min_seg > kSortCap)
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: min_seg must be in [1, 16384]");
    if (o.max_segments < 1 || o.max_segments > (1LL << 26))
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: max_segments must be in [1, 2^26]");
    return FFA_OK;
}

}  // namespace

extern "C" void ffa_peak_opts_default(ffa_peak_opts* opts) {
    if (opts) *opts = defaults();
}

extern "C" ffa_status ffa_find_peaks_workspace(int64_t ntrials, int32_t nw,
                                               const ffa_peak_opts* opts, size_t* bytes) {
    if (!bytes) return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks_workspace: bytes is null");
    if (ntrials < 1 || ntrials > 0xffffffffLL || nw < 1 || nw > ffa::kMaxWidths)
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks_workspace: ntrials must be in "
                                           "[1, 2^32 - 1] and nw in [1, 64]");
    const ffa_peak_opts o = opts ? *opts : defaults();
    const ffa_status st = check_opts(o);
    if (st != FFA_OK) return st;
    *bytes = layout(ntrials, nw, o.max_segments).bytes;
    return FFA_OK;
}

extern "C" ffa_status ffa_find_peaks(const double* d_periods, const float* d_snr, int64_t ntrials,
                                     int32_t nw, double tobs, const ffa_peak_opts* opts,
                                     ffa_peak* d_peaks, int64_t peak_cap, int64_t* d_npeaks,
                                     void* d_ws, size_t ws_bytes, void* stream) {
    if (!d_periods || !d_snr || !d_npeaks || !d_ws || (peak_cap > 0 && !d_peaks))
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: null pointer");
    if (ntrials < 1 || ntrials > 0xffffffffLL || nw < 1 || nw > ffa::kMaxWidths)
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: ntrials must be in [1, 2^32 - 1] "
                                           "and nw in [1, 64]");
    if (!(tobs > 0.0) || !std::isfinite(tobs))
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: tobs must be > 0");
    if (peak_cap < 0) return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: peak_cap < 0");
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks: workspace must be 256-byte aligned");
    const ffa_peak_opts o = opts ? *opts : defaults();
    ffa_status st = check_opts(o);
    if (st != FFA_OK) return st;
    const Layout L = layout(ntrials, nw, o.max_segments);
    if (ws_bytes < L.bytes)
        return ffa::set_error(FFA_ERR_CAPACITY, "ffa_find_peaks: workspace too small");
    char* ws = static_cast<char*>(d_ws);
    Params p;
    p.periods = d_periods;
    p.snr = d_snr;
    p.ntrials = ntrials;
    p.nw = nw;
    p.width = o.dzseg / tobs;
    p.nsigma = o.nsigma;
    p.gap = o.clrad / tobs;
    p.degree = o.degree;
    p.min_seg = o.min_seg;
    p.max_segments = o.max_segments;
    p.status = reinterpret_cast<unsigned*>(ws + L.status);
    p.hdr = reinterpret_cast<Hdr*>(ws + L.hdr);
    p.ctrl = reinterpret_cast<double2*>(ws + L.ctrl);
    p.fit = reinterpret_cast<Fit*>(ws + L.fit);
    p.list = reinterpret_cast<uint32_t*>(ws + L.list);
    p.best = reinterpret_cast<uint64_t*>(ws + L.best);
    p.counts = reinterpret_cast<long long*>(ws + L.counts);
    p.nchunks = (ntrials + kSelTile - 1) / kSelTile;
    p.ccount = reinterpret_cast<long long*>(ws + L.ccount);
    p.coff = reinterpret_cast<long long*>(ws + L.coff);
    p.nu = reinterpret_cast<double*>(ws + L.nu);
    p.lnnu = reinterpret_cast<double*>(ws + L.lnnu);
    p.flags = reinterpret_cast<uint8_t*>(ws + L.flags);
    p.first = reinterpret_cast<long long*>(ws + L.first);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the segment kernel's shared-memory size, once per device (setting it twice from two
    // threads is harmless)
    static std::atomic<unsigned char> attr_done[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return ffa::set_error(FFA_ERR_CUDA, "ffa_find_peaks: no current device");
    }
    if (dev < 0 || dev >= 64 || !attr_done[dev].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(pk_segment_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSortCap * (int)sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return ffa::set_error(FFA_ERR_CUDA, "ffa_find_peaks: shared-memory attribute");
        }
        if (dev >= 0 && dev < 64) attr_done[dev].store(1, std::memory_order_release);
    }
    {
        LaunchScope ls(ffa::kPeaks, 4.0 * (double)ntrials * nw + 8.0 * ntrials, s);
        if (cudaMemsetAsync(p.status, 0, sizeof(unsigned), s) != cudaSuccess) {
            cudaGetLastError();
            return ffa::set_error(FFA_ERR_CUDA, "ffa_find_peaks: status reset");
        }
        pk_prep_kernel<<<(unsigned)((ntrials + kPrepThreads - 1) / kPrepThreads), kPrepThreads, 0,
                         s>>>(p);
        pk_range_kernel<<<1, 32, 0, s>>>(p);
        pk_bounds_kernel<<<152, 256, 0, s>>>(p);
        pk_segment_kernel<<<kSegGrid, kSegThreads, kSortCap * sizeof(float), s>>>(p);
        pk_fit_kernel<<<nw, kFitThreads, 0, s>>>(p);
        const dim3 grid((unsigned)p.nchunks, (unsigned)nw);
        pk_count_kernel<<<(unsigned)p.nchunks, kSelThreads, 0, s>>>(p);
        pk_offsets_kernel<<<nw, kSelThreads, 0, s>>>(p);
        pk_write_kernel<<<grid, kSelThreads, 0, s>>>(p);
        pk_cluster_kernel<<<nw, kSelThreads, 0, s>>>(p);
        pk_output_kernel<<<1, 1024, 0, s>>>(p, d_peaks, peak_cap, reinterpret_cast<long long*>(d_npeaks));
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[200];
        snprintf(buf, sizeof buf, "ffa_find_peaks: launch: %s", cudaGetErrorString(e));
        return ffa::set_error(FFA_ERR_CUDA, buf);
    }
    return FFA_OK;
}

extern "C" ffa_status ffa_find_peaks_fits(const void* d_ws, int64_t ntrials, int32_t nw,
                                          const ffa_peak_opts* opts, int64_t* h_nseg,
                                          double* h_ctrl, int64_t ctrl_cap, double* h_fits,
                                          void* stream) {
    if (!d_ws || !h_nseg || !h_fits || (ctrl_cap > 0 && !h_ctrl) || ctrl_cap < 0)
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks_fits: null pointer or bad capacity");
    if (ntrials < 1 || ntrials > 0xffffffffLL || nw < 1 || nw > ffa::kMaxWidths)
        return ffa::set_error(FFA_ERR_ARG, "ffa_find_peaks_fits: ntrials must be in "
                                           "[1, 2^32 - 1] and nw in [1, 64]");
    const ffa_peak_opts o = opts ? *opts : defaults();
    ffa_status st = check_opts(o);
    if (st != FFA_OK) return st;
    const Layout L = layout(ntrials, nw, o.max_segments);
    const char* ws = static_cast<const char*>(d_ws);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Hdr h{};
    std::vector<Fit> fits(nw);
    if (cudaMemcpyAsync(&h, ws + L.hdr, sizeof(Hdr), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(fits.data(), ws + L.fit, sizeof(Fit) * nw, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return ffa::set_error(FFA_ERR_CUDA, "ffa_find_peaks_fits: copy");
    }
    *h_nseg = h.nseg;
    const long long nc = std::min<long long>(std::min<long long>(h.nseg, o.max_segments), ctrl_cap);
    if (nc > 0) {
        if (cudaMemcpyAsync(h_ctrl, ws + L.ctrl, sizeof(double2) * (size_t)nc * nw,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return ffa::set_error(FFA_ERR_CUDA, "ffa_find_peaks_fits: copy");
        }
    }
    for (int iw = 0; iw < nw; ++iw) {
        double* f = h_fits + 10 * iw;
        f[0] = fits[iw].xbar;
        f[1] = fits[iw].xscale;
        f[2] = fits[iw].valid ? 1.0 : 0.0;
        for (int a = 0; a <= kMaxDegree; ++a)  // 0 past the degree
            f[3 + a] = fits[iw].valid && a <= o.degree ? fits[iw].c[a] : 0.0;
    }
    return FFA_OK;
}

cudaError_t ffa::bounds_seen_peaks(unsigned* bits) {
    unsigned v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, ffa::g_bounds_seen, sizeof(v));
    if (e != cudaSuccess) return e;
    *bits = v;
    v = 0;
    return cudaMemcpyToSymbol(ffa::g_bounds_seen, &v, sizeof(v));
}
