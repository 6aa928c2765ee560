// ffa_internal.h -- structures shared by the host plan and the sm_103a kernels of
// libffa.  Not part of the public ABI (include/ffa.h is).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace ffa {

constexpr int kMaxWidths = 64;       // boxcar widths per search
constexpr int kMaxCols = 4096;       // base period (bins) limit of this build
constexpr int kSmemBytes = 232448;   // dynamic shared memory per CTA on sm_103 (227 KB)
// Shared-memory budgets of the two FFA kernels: the whole CTA maximum (one CTA per SM)
// or a fraction of it (several CTAs per SM hide each other's barriers and load waits).
#ifndef FFA_BOTTOM_SMEM
#define FFA_BOTTOM_SMEM 232448
#endif
#ifndef FFA_TOP_SMEM
#define FFA_TOP_SMEM 232448
#endif
#ifndef FFA_BOTTOM_MINB
#define FFA_BOTTOM_MINB 1
#endif
#ifndef FFA_TOP_MINB
#define FFA_TOP_MINB 1
#endif
constexpr int kBottomSmemBytes = FFA_BOTTOM_SMEM;
constexpr int kTopSmemBytes = FFA_TOP_SMEM;
constexpr int kBottomMinBlocks = FFA_BOTTOM_MINB;  // resident CTAs per SM to allow for
constexpr int kTopMinBlocks = FFA_TOP_MINB;
#ifndef FFA_BOTTOM_THREADS
#define FFA_BOTTOM_THREADS 512
#endif
#ifndef FFA_TOP_THREADS
#define FFA_TOP_THREADS 512
#endif
constexpr int kBottomThreads = FFA_BOTTOM_THREADS;  // CTA of the shared-memory sub-tree kernel
constexpr int kTopThreads = FFA_TOP_THREADS;        // CTA of the gathered top-level kernel
constexpr int kTopMaxLevels = 3;     // merge levels per top pass
constexpr int kTopMaxRows = 128;     // output rows per top CTA

// Device status word bits (first word of every workspace).
constexpr unsigned kDevTimeout = 1u;
constexpr unsigned kDevBadItem = 2u;
constexpr unsigned kDevBounds = 32u;  // a checked build found an index out of range

// Checked build (compiled with FFA_CHECKED): every shared-memory range and global index
// the kernels compute from runtime data is checked before use; a violation sets
// kDevBounds in the status word and the access (or the whole work item) is skipped.
#ifdef FFA_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
#ifdef __CUDACC__
// Checked builds also record every violation here, one word per translation unit, so
// that it is seen whatever status word (or none) the launch had; bounds_seen_*() read
// and clear it.
static __device__ unsigned g_bounds_seen;
__device__ __forceinline__ void bounds_violation(unsigned* status) {
    if (status) atomicOr(status, kDevBounds);
    atomicOr(&g_bounds_seen, kDevBounds);
}
// [i, i + len) inside [0, cap); in an unchecked build always true.
__device__ __forceinline__ bool in_range(long long i, long long len, long long cap,
                                         unsigned* status) {
    if (!kChecked) return true;
    if (i >= 0 && len >= 0 && i + len <= cap) return true;
    bounds_violation(status);
    return false;
}
// Floats of the launch's dynamic shared memory.
__device__ __forceinline__ long long dyn_smem_floats() {
    unsigned r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return (long long)(r / 4);
}
#endif

// nint(a / d), ties up, for a >= 0, d > 0 (Sec. 2.2: i and j of the merge rule).
__host__ __device__ inline int nint_div(long long a, long long d) {
    long long num = 2 * a + d, den = 2 * d;
    if (num < 4294967296LL) return (int)((unsigned)num / (unsigned)den);
    return (int)(num / den);
}

// Merge rule for output row s of an n-row node: head row i, tail row j, shift i + b.
struct Split {
    int i, j, shift;
};
__host__ __device__ inline Split merge_split(int n, int s) {
    int nh = n >> 1, nt = n - nh;
    Split r;
    r.i = nint_div((long long)(nh - 1) * s, n - 1);
    r.j = nint_div((long long)(nt - 1) * s, n - 1);
    r.shift = s - r.j;  // i + b = s - j
    return r;
}

// Interval table of a top-pass work item, heap order (node e at level l is 2^l - 1 + j,
// children 2e + 1 and 2e + 2): node e at t[8 e]: {absolute start row, rows, lo, hi},
// where rows lo..hi of the node are the ones the item needs.  Node 0 is the output
// block.
//
// The item's record (kTopRecInts ints, built on the device before the FFA launch)
// is that table with the shared-memory layout added: t[8 e + 4] = float offset of the
// node's row lo in shared memory; at kRecLvl the first row descriptor of each level
// L-1 .. 0 and their end; at kRecBytes the bytes its bulk copies move.
constexpr int kTopRecInts = 128;
constexpr int kRecLvl = 120;
constexpr int kRecBytes = 125;
__host__ __device__ inline void top_intervals(int st0, int n0, int lo0, int hi0, int L, int* t) {
    t[0] = st0; t[1] = n0; t[2] = lo0; t[3] = hi0;
    for (int l = 0; l < L; ++l) {
        for (int j = 0; j < (1 << l); ++j) {
            const int e = (1 << l) - 1 + j;
            const int st = t[8 * e], n = t[8 * e + 1], lo = t[8 * e + 2], hi = t[8 * e + 3];
            const int nh = n >> 1;
            const Split a = merge_split(n, lo), z = merge_split(n, hi);
            int* h = t + 8 * (2 * e + 1);
            int* q = t + 8 * (2 * e + 2);
            h[0] = st; h[1] = nh; h[2] = a.i; h[3] = z.i;
            q[0] = st + nh; q[1] = n - nh; q[2] = a.j; q[3] = z.j;
        }
    }
}

// One FFA transform of a search: base period p (bins), m rows of the octave series.
struct TransformDesc {
    int64_t src_off;      // float offset of row 0 in the source buffer
    int64_t scratch_off;  // float offset of row 0 in the scratch buffers (its ring slot)
    int64_t trial0;       // index of its first trial in the periodogram
    double tau;           // sampling time of its octave (s)
    int32_t p;            // bins per row
    int32_t m;            // rows
    int32_t kept;         // rows s with P_s < (p + 1) tau  (Sec. 2.3)
    int32_t depth;        // depth of the shared-memory sub-trees (0 = whole tree)
    float inv_std;        // 1 / sqrt(m V_f): noise std of one folded bin, inverted
    int32_t chunk;        // merge levels per top pass (1..kTopMaxLevels)
    int32_t batch;        // scratch batch of the transform (-1: whole tree, no scratch)
    int32_t pad;
};
static_assert(sizeof(TransformDesc) == 64, "TransformDesc layout");

// A CTA's share of a launch: transform index, node / row-block index, and for the
// top kernel the pass index and the rows per block.
struct WorkItem {
    int32_t tr;
    int32_t idx;
    int16_t pass;
    int16_t rows;
    int32_t pad;
};
static_assert(sizeof(WorkItem) == 16, "WorkItem layout");

// Passes of the top of an FFA tree whose shared-memory sub-trees sit at depth D:
// chunks of `chunk` levels from the bottom, the last one reaching the root.
__host__ __device__ inline int top_passes(int depth, int chunk) {
    return (depth + chunk - 1) / chunk;
}
__host__ __device__ inline int top_pass_in_depth(int depth, int chunk, int pass) {
    return depth - chunk * pass;
}
__host__ __device__ inline int top_pass_out_depth(int depth, int chunk, int pass) {
    const int d = depth - chunk * (pass + 1);
    return d > 0 ? d : 0;
}

// Shared-memory layout (in floats) of a top-kernel CTA merging L levels for K output
// rows of p bins.  Rows of level l (0 = output) number at most K + 3 (2^l - 1).
struct TopLayout {
    int table;      // interval table (ints): 15 nodes x 8 ints
    int desc;       // row descriptors (int4), desc_cap of them
    int desc_cap;
    int buf_a;      // levels L, L-2, ...   (level L with per-interval alignment slack)
    int buf_b;      // levels L-1, L-3, ...
    int sbuf;       // per-warp prefix-sum rows of the boxcar S/N (scoring passes)
    int sbuf_warp;  // floats per warp
    int total;      // floats
};
__host__ __device__ inline int round4(int v) { return (v + 3) & ~3; }

// Shared memory of the boxcar S/N.  Profiles of p <= kSnrHalfMaxP bins are scored two
// per warp, one per half-warp: lane h of a half owns the Q = snr_q(p) consecutive
// phases Q h .. Q h + Q - 1 (Q odd and 16 Q >= p, so that the 16 lanes' rows of reads
// fall in 16 different banks), and the half's prefix-sum row holds 16 Q + wmax floats.
// The second half's row starts snr_half_stride floats after the first: 16 more than a
// multiple of 32, so that the two halves never share a bank either.  Longer profiles
// are scored one per warp, with a row of p + wmax + 1 floats.
constexpr int kSnrMaxQ = 35;
constexpr int kSnrHalfMaxP = 16 * kSnrMaxQ;  // 560 bins
__host__ __device__ inline int snr_q(int p) { return ((p + 15) / 16) | 1; }
__host__ __device__ inline int snr_half_stride(int p, int wmax) {
    const int need = 16 * snr_q(p) + wmax;
    return need + (((16 - need) % 32) + 32) % 32;
}
__host__ __device__ inline int snr_warp_floats(int p, int wmax) {
    return p <= kSnrHalfMaxP ? 2 * snr_half_stride(p, wmax) : round4(p + wmax + 1);
}

// Shared-memory layout (in floats) of a sub-tree CTA: barrier and two ints, the row
// descriptors of every shared-memory merge level (nmax int2 per level, all made while
// the rows are in flight), the register-stage node list (nmax ints), and two ping-pong
// row buffers of buf_floats.
constexpr int kBottomMaxRows = 1024;
constexpr int kRegLevels = 4;  // merge levels done in registers: nodes of <= 16 rows
__host__ __device__ inline int height_of(int n) {
    int h = 0;
    while ((1 << h) < n) ++h;
    return h;
}
__host__ __device__ inline int bottom_smem_levels(int nmax) {
    const int l = height_of(nmax) - kRegLevels;
    return l > 0 ? l : 0;
}
struct BottomLayout {
    int desc;
    int nodes;
    int buf_a;
    int buf_b;
    int buf_floats;
    int total;
};
__host__ __device__ inline BottomLayout bottom_layout(int nmax, int elems_max, int snr_need) {
    BottomLayout b;
    b.desc = 4;
    b.nodes = b.desc + 2 * bottom_smem_levels(nmax) * nmax;
    b.buf_a = round4(b.nodes + nmax);
    int need = elems_max + 4;
    if (snr_need > need) need = snr_need;
    b.buf_floats = round4(need);
    b.buf_b = b.buf_a + b.buf_floats;
    b.total = b.buf_b + b.buf_floats;
    return b;
}
__host__ __device__ inline TopLayout top_layout(int K, int L, int p, int wmax, bool snr) {
    TopLayout t;
    int off = 4;  // mbarrier
    t.table = off;
    off += 128;
    t.desc = off;
    t.desc_cap = L * K + 3 * (1 << L) + 8;
    off += 4 * t.desc_cap;
    int cap_a = 0, cap_b = 0;
    for (int l = 0; l <= L; ++l) {
        int sz = (K + 3 * ((1 << l) - 1)) * p + (l == L ? 8 * (1 << L) : 0);
        if (((L - l) & 1) == 0) cap_a = cap_a > sz ? cap_a : sz;
        else cap_b = cap_b > sz ? cap_b : sz;
    }
    t.sbuf_warp = snr ? snr_warp_floats(p, wmax) : 0;
    const int s_need = (kTopThreads / 32) * t.sbuf_warp;
    // half-warp scoring reads level 0 straight from level 1 (level 0 is never stored):
    // its buffer, whose earlier contents are consumed by then, holds the S rows
    const bool fused = snr && p <= kSnrHalfMaxP;
    const bool zero_in_a = (L & 1) == 0;
    if (fused) {
        if (zero_in_a) cap_a = cap_a > s_need ? cap_a : s_need;
        else cap_b = cap_b > s_need ? cap_b : s_need;
    }
    t.buf_a = off;
    off += round4(cap_a);
    t.buf_b = off;
    off += round4(cap_b);
    if (fused) {
        t.sbuf = zero_in_a ? t.buf_a : t.buf_b;
    } else {
        t.sbuf = off;
        off += s_need;
    }
    t.total = off;
    return t;
}

// Downsampling of one octave: factor f in 64.64 fixed point (exact for a double).
struct OctaveDesc {
    int64_t out_off;   // float offset of the octave's series in the series buffer
    int64_t nk;        // samples: floor(n / f)
    int64_t x_off;     // first raw sample of its series in the input
    int64_t x_n;       // raw samples of its series
    int64_t pre_off;   // first prefix sum of its series
    uint64_t f_int;    // floor(f)
    uint64_t f_frac;   // (f - floor(f)) * 2^64, exact
};

struct Widths {
    int32_t nw;
    int32_t wmax;
    int32_t boxcar;  // template: 0 plain (1/sqrt(w) on w bins), 1 zero-mean (zero sum)
    int32_t w[kMaxWidths];
    float inv_sqrt_w[kMaxWidths];
};

// Kernel kinds for launch accounting and profiling.
enum KernelKind : int {
    kPrefixPartial = 0,
    kPrefixTop,
    kPrefixFinal,
    kDownsample,
    kFfaBottom,
    kFfaBottomSnr,
    kFfaTop,
    kBoxcarSnr,
    kNormalise,
    kFfaPersistent,
    kItemRecs,
    kNumKinds
};

// ------------------------------------------------------------------------------
// Launch parameter blocks.
// ------------------------------------------------------------------------------
// One series of the prefix-sum pass.  Its prefix sums depend on its own samples only
// (the scan restarts at every series), so a series downsamples to the same values
// wherever it sits in the input and whatever else is searched with it.
struct PrefixSeg {
    int64_t x_off;    // first sample of the series in the input
    int64_t pre_off;  // its n + 1 exclusive prefix sums start here
    int64_t n;        // samples
    int64_t blk0;     // its first chunk (CTA of the partial and final passes)
};

struct PrefixParams {
    const void* x;
    int dtype;              // ffa_dtype
    const PrefixSeg* segs;  // device table of nsegs series, or nullptr: `single`
    const int* blk_seg;     // series of each chunk (nullptr: series 0)
    PrefixSeg single;
    int nsegs;
    float2* partial;        // per-chunk double-float sums, then their per-series scan
    float2* prefix;         // double-float exclusive prefix sums
    int64_t nchunks;        // chunks over all series
    int64_t total;          // samples over all series
    int64_t x_cap, prefix_cap;  // elements of x and of prefix (checks)
    unsigned* status;
};

constexpr int kDownsampleThreads = 256;
constexpr int kDownsamplePerBlock = 1024;  // output samples per CTA (4 per thread)

struct DownsampleParams {
    const void* x;
    int dtype;
    int64_t n;
    const float2* prefix;
    const OctaveDesc* oct;          // null: one octave, `single`
    OctaveDesc single;
    const int2* blocks;             // per CTA: {octave, first output}; null: octave 0
    int nblocks;
    int64_t total;        // sum of nk (algorithmic accounting)
    float* out;           // series buffer
    int64_t x_cap, prefix_cap, out_cap;  // elements of x, prefix and out (checks)
    unsigned* status;
};

struct BottomParams {
    const float* src;               // octave series buffer or the caller's block
    float* dst;                     // sub-trees of transforms with an even number of top
    float* dst_odd;                 // passes go to dst, the others to dst_odd
    const TransformDesc* trs;       // null: use `single`
    const WorkItem* items;          // null: item = {0, blockIdx.x}
    TransformDesc single;
    Widths widths;
    double* periods;
    int32_t* foldbins;
    float* snr;
    unsigned* status;
    int nmax;                       // largest sub-tree (rows) of the launch
    int elems_max;                  // largest sub-tree (floats) of the launch
    int snr_warps;                  // warps that score rows (fused S/N mode)
    int snr_floats;                 // shared floats those warps need (0 otherwise)
    long long src_cap, dst_cap;     // floats of src and of each of dst, dst_odd (checks)
    long long ntrials;              // trials of the S/N outputs (checks)
};

struct TopParams {
    float* buf0;                    // the two scratch buffers: pass j of a transform with
    float* buf1;                    // P passes reads buf[(P-j)&1], writes buf[(P-j-1)&1]
    const TransformDesc* trs;
    const WorkItem* items;
    TransformDesc single;           // used when trs is null
    Widths widths;
    double* periods;
    int32_t* foldbins;
    float* snr;                     // null: the last pass stores the transform instead
    unsigned* status;
    int single_pass;                // pass and rows per block when items is null
    int single_rows;
    long long buf_cap;              // floats of each of buf0, buf1 (checks)
    long long ntrials;              // trials of the S/N outputs (checks)
};

constexpr int kMaxStages = 16;  // sub-trees + up to 15 top passes per transform

// Everything a persistent CTA needs to start the item at one queue position, fetched by
// one bulk copy two items ahead: the work item (for a top pass, WorkItem::pad indexes its
// interval table, kTopRecInts ints fetched one item ahead), its transform, the completion
// counter it waits for and the count that counter must reach, and the counter the item
// releases when it completes.  Counters: per (transform, stage), the items of that stage
// completed; per scratch batch, its last-pass items completed (the batch's ring slot is
// free for the batch `ring` places later once all of them have read it).
struct ItemHead {
    WorkItem item;
    TransformDesc tr;
    int32_t wait;                   // counter index (-1: none)
    int32_t need;
    int32_t rel[2];                 // counter released on completion (-1: none); rel[1] unused
};
static_assert(sizeof(ItemHead) == 96, "ItemHead layout (a multiple of 16 bytes)");
constexpr int kTopRecBytes = kTopRecInts * 4;
// Shared memory of the persistent kernel after the item layouts: the queue slot (16 B),
// five barriers (three heads, two tables; 48 B with padding), three heads and two tables.
constexpr int kPersistExtraBytes = 64 + 3 * (int)sizeof(ItemHead) + 2 * kTopRecBytes;

struct PersistentParams {
    BottomParams bottom;            // sub-tree items (pass -1)
    BottomParams bottom_snr;        // whole-tree items scored directly (pass -2)
    TopParams top;                  // top-pass items (pass >= 0)
    const ItemHead* heads;          // one per queue position
    const int* tables;              // kTopRecInts per top-pass item (WorkItem::pad)
    int nitems;
    int* queue;                     // dispatch counter, zero at launch
    int* done;                      // completion counters, zero at launch
    int smem_floats;                // dynamic shared floats before the queue slot (a multiple of 4)
    long long wait_cycles;          // limit of every wait of a CTA, SM clock cycles
    int ncounters;                  // completion counters (checks)
    int ntables;                    // top-pass tables (checks)
};

// The per-item records of a queue, made on the device before the FFA launch.
struct RecParams {
    TopParams top;                  // items, transforms, scratch buffers (for the tables)
    const int* stage_count;         // per transform and stage: items listed
    const int* batch_top;           // per scratch batch: its last-pass items
    int nitems;
    int ring;                       // scratch ring slots (a batch reuses slot batch % ring)
    int nbatches;
    int batch_base;                 // index of batch 0's counter among the counters
    int inject_tr;                  // fault injection (tests): this transform's stage 1 waits
                                    // for one item more than exist (-1: none)
    ItemHead* heads;
    int* tables;
    int ntables;                    // top-pass tables (checks)
    unsigned* status;
};

struct SnrParams {
    const float* prof;
    int64_t rows;
    int cols;
    Widths widths;
    float inv_std;
    float* snr;
    int warp_floats;
    unsigned* status;     // (checks; may be null)
};

struct NormaliseParams {
    const float* x;
    int64_t n;
    double* partial;                // per-CTA FP64 partial sums
    int nblocks;
    double* stats;                  // [0] mean, [1] standard deviation (device)
    void* out;
    int out_dtype;                  // ffa_dtype
};

// Launchers (ffa_kernels.cu).  Each returns the cudaError_t of the launch.
cudaError_t launch_prefix(const PrefixParams& P, cudaStream_t s);
cudaError_t launch_downsample(const DownsampleParams& P, cudaStream_t s);
cudaError_t launch_bottom(const BottomParams& P, int nblocks, int smem_bytes, bool snr_mode,
                          cudaStream_t s);
cudaError_t launch_top(const TopParams& P, int nblocks, int smem_bytes, cudaStream_t s);
cudaError_t launch_persistent(const PersistentParams& P, int smem_bytes, cudaStream_t s);
// Read and clear the violations recorded by the kernels of ffa_kernels.cu, ffa_median.cu
// and ffa_peaks.cu (checked builds).
cudaError_t bounds_seen_kernels(unsigned* bits);
cudaError_t bounds_seen_median(unsigned* bits);
cudaError_t bounds_seen_peaks(unsigned* bits);
cudaError_t launch_item_recs(const RecParams& R, cudaStream_t s);
cudaError_t launch_snr(const SnrParams& P, cudaStream_t s);
cudaError_t launch_normalise(const NormaliseParams& P, cudaStream_t s);
constexpr int kNormaliseBlocks = 1216;  // 8 CTAs per SM

// Launch accounting (ffa_api.cu): brackets one launch with profiling events.
struct LaunchScope {
    LaunchScope(int kind, double alg_bytes, cudaStream_t s);
    ~LaunchScope();
    int kind;
    double bytes;
    cudaStream_t stream;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

int prefix_chunk();  // elements per CTA of the prefix kernels

}  // namespace ffa
