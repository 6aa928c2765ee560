// ffa_api.cu -- host side of libffa: argument checking, the search plan (Sec. 5.3 of
// Morello et al. 2020), workspace layout, launch sequencing and launch accounting,
// behind the C ABI declared in include/ffa.h.
#include "ffa.h"
#include "ffa_internal.h"
#include "ffa_kinds.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

namespace ffa {
namespace {

// ---------------------------------------------------------------------------------
// Errors.
// ---------------------------------------------------------------------------------
thread_local std::string g_err;

ffa_status fail(ffa_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

ffa_status cuda_fail(cudaError_t e, const char* what) {
    return fail(FFA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Fault injection for tests, by the environment variable FFA_FAULT: "plan" makes plan
// building fail, "alloc" the page-locked table allocation and "launch" the start of the
// launch sequence (each before any CUDA call of the call); "stage" makes the second stage of one transform
// wait for one item more than exist, so that the wait runs out on the device and the
// call reports FFA_ERR_TIMEOUT through ffa_check.
bool fault(const char* what) {
    const char* f = std::getenv("FFA_FAULT");
    return f && std::strcmp(f, what) == 0;
}

// Limit of every device-side wait of the persistent launch, in milliseconds of SM clock
// (at the maximum clock; a wait at a lower clock lasts proportionally longer).
std::atomic<double> g_wait_ms{1000.0};
constexpr double kCyclesPerMs = 2.1e6;

#define FFA_CUDA(call, what)                      \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------------------------
// Launch accounting.
// ---------------------------------------------------------------------------------
struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double bytes;
};
struct ProfAcc {
    int64_t launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
};

std::atomic<int64_t> g_launches{0};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_pending;
std::vector<cudaEvent_t> g_pool;
ProfAcc g_acc[kAllKinds];

const char* kKindNames[kAllKinds] = {"prefix_partial", "prefix_top",     "prefix_final",
                                     "downsample",     "ffa_bottom",     "ffa_bottom_snr",
                                     "ffa_top",        "boxcar_snr",     "normalise",
                                     "ffa_persistent", "item_records",   "median_build",
                                     "median_query",   "peaks"};

cudaEvent_t pool_get() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drain_pending() {
    for (auto& r : g_pending) {
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        g_acc[r.kind].launches += 1;
        g_acc[r.kind].ms += ms;
        g_acc[r.kind].bytes += r.bytes;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_pending.clear();
}

// ---------------------------------------------------------------------------------
// Search plan.
// ---------------------------------------------------------------------------------
// One series of a search: samples [x_off, x_off + n) of the input.
struct SeriesSpec {
    int64_t x_off, n;
    double tsamp, pmin, pmax;
    int bmin, bmax;
    bool operator<(const SeriesSpec& o) const {
        return std::tie(x_off, n, tsamp, pmin, pmax, bmin, bmax) <
               std::tie(o.x_off, o.n, o.tsamp, o.pmin, o.pmax, o.bmin, o.bmax);
    }
};

// Options of a plan: tile shape (0 = the largest that fits shared memory) and the boxcar
// template of the S/N.
// A class of transforms (m <= m_max, p <= p_max; 0: any) with its own tiles (0: the
// plan-wide value).
struct TileClass {
    int m_max = 0, p_max = 0, subtree_rows = 0, top_levels = 0, top_rows = 0;
    std::array<int, 5> key() const { return {m_max, p_max, subtree_rows, top_levels, top_rows}; }
};
struct Tiles {
    int subtree_rows = 0, top_levels = 0, top_rows = 0, boxcar = 0;
    std::vector<TileClass> classes;
    bool operator<(const Tiles& o) const {
        if (std::tie(subtree_rows, top_levels, top_rows, boxcar) !=
            std::tie(o.subtree_rows, o.top_levels, o.top_rows, o.boxcar))
            return std::tie(subtree_rows, top_levels, top_rows, boxcar) <
                   std::tie(o.subtree_rows, o.top_levels, o.top_rows, o.boxcar);
        return std::lexicographical_compare(
            classes.begin(), classes.end(), o.classes.begin(), o.classes.end(),
            [](const TileClass& a, const TileClass& b) { return a.key() < b.key(); });
    }
    // the class of a transform of m rows and p bins, or -1
    int class_of(int m, int p) const {
        for (size_t c = 0; c < classes.size(); ++c)
            if ((!classes[c].m_max || m <= classes[c].m_max) &&
                (!classes[c].p_max || p <= classes[c].p_max))
                return (int)c;
        return -1;
    }
};

ffa_status read_tiles(const ffa_plan_opts* t, Tiles* out) {
    *out = Tiles{};
    if (!t) return FFA_OK;
    if (t->subtree_rows < 0 || t->subtree_rows == 1 || t->subtree_rows > kBottomMaxRows)
        return fail(FFA_ERR_ARG, "subtree_rows must be 0 or 2..%d", kBottomMaxRows);
    if (t->top_levels < 0 || t->top_levels > kTopMaxLevels)
        return fail(FFA_ERR_ARG, "top_levels must be 0..%d", kTopMaxLevels);
    if (t->top_rows < 0 || t->top_rows > kTopMaxRows)
        return fail(FFA_ERR_ARG, "top_rows must be 0..%d", kTopMaxRows);
    if (t->boxcar != FFA_BOXCAR_PLAIN && t->boxcar != FFA_BOXCAR_ZERO_MEAN)
        return fail(FFA_ERR_ARG, "boxcar must be FFA_BOXCAR_PLAIN or FFA_BOXCAR_ZERO_MEAN");
    if (t->nclasses < 0 || t->nclasses > FFA_MAX_TILE_CLASSES)
        return fail(FFA_ERR_ARG, "nclasses must be 0..%d", FFA_MAX_TILE_CLASSES);
    *out = Tiles{t->subtree_rows, t->top_levels, t->top_rows, t->boxcar, {}};
    for (int c = 0; c < t->nclasses; ++c) {
        const ffa_tile_class& k = t->classes[c];
        if (k.m_max < 0 || k.p_max < 0) return fail(FFA_ERR_ARG, "class %d: negative bound", c);
        if (k.subtree_rows < 0 || k.subtree_rows == 1 || k.subtree_rows > kBottomMaxRows)
            return fail(FFA_ERR_ARG, "class %d: subtree_rows must be 0 or 2..%d", c, kBottomMaxRows);
        if (k.top_levels < 0 || k.top_levels > kTopMaxLevels)
            return fail(FFA_ERR_ARG, "class %d: top_levels must be 0..%d", c, kTopMaxLevels);
        if (k.top_rows < 0 || k.top_rows > kTopMaxRows)
            return fail(FFA_ERR_ARG, "class %d: top_rows must be 0..%d", c, kTopMaxRows);
        out->classes.push_back(TileClass{k.m_max, k.p_max, k.subtree_rows, k.top_levels, k.top_rows});
    }
    return FFA_OK;
}

struct Plan {
    Tiles tiles;
    // parameters
    std::vector<SeriesSpec> series;
    int64_t n = 0;       // input span: max over series of x_off + n
    std::vector<int> widths;
    std::vector<int64_t> series_trial0;  // first trial of each series, + total
    // derived
    Widths W{};
    std::vector<OctaveDesc> oct;
    std::vector<TransformDesc> trs;
    std::vector<WorkItem> items;
    std::vector<int2> ds_blocks;  // downsampling CTAs: {octave, first output}
    std::vector<PrefixSeg> segs;  // prefix-sum pass: one per series
    std::vector<int> blk_seg;     // series of each prefix chunk
    int bottom0_nmax = 0, bottom0_elems = 0, bottom0_snr_warps = 0;
    int bottom0_snr_floats = 0;
    int row_cap = kBottomMaxRows;  // sub-tree row limit (lowered if a launch's mix overflows)
    std::vector<int> stage_count;
    std::vector<int> tr_class;    // tile class of each transform (-1: none)
    std::vector<int> batch_top;   // per scratch batch: its last-pass items
    int ring = 1, nbatches = 0;   // scratch ring slots; batch b uses slot b % ring
    int64_t slot_floats = 0;      // floats of one ring slot (per scratch buffer)
    int ntop = 0;                 // top-pass items (tables made on the device)
    int bottom_nmax = 0, bottom_elems = 0;
    int smem_floats = 0;
    int nitems = 0;
    double ffa_bytes = 0;  // algorithmic bytes of the FFA + S/N: per transform 4 m p + 4 nw kept
    double ffa_adds = 0, snr_ops = 0;  // arithmetic of the method (FP32 operations)
    size_t o_counters = 0, counter_bytes = 0;
    int64_t ntrials = 0, ds_total = 0, ds_floats = 0, scratch_floats = 0, folded = 0;
    int max_rows = 0, max_p = 0;
    int64_t nchunks = 0, prefix_len = 0, input_total = 0;
    // workspace layout (bytes)
    size_t o_tables = 0, o_oct = 0, o_trs = 0, o_items = 0, o_dsblk = 0, o_stcnt = 0, o_btop = 0;
    size_t o_heads = 0, o_toptab = 0;
    size_t o_segs = 0, o_blkseg = 0;
    size_t tables_bytes = 0;
    size_t o_prefix = 0, o_partial = 0, o_ds = 0, o_s0 = 0, o_s1 = 0, ws_bytes = 0;
    size_t o_hx = 0, o_hper = 0, o_hfb = 0, o_hsnr = 0, ws_host_bytes = 0;
    void* pinned = nullptr;
    ~Plan() {
        if (pinned) cudaFreeHost(pinned);
    }
};

constexpr size_t kStatusBytes = 256;
constexpr ffa_status kRetrySmaller = -1;  // internal: a launch's sub-tree mix overflows
std::mutex g_plan_mu;
// Folded samples per scratch batch of transforms.  The queue lists stage s of batch b on
// diagonal b + kStageStride * s, so that the items of a stage are listed about two
// diagonals (several batches of work) after the items they wait for.  The scratch is a
// ring of slots, one batch in each, reused by the batch `ring` places later, with ring =
// kStageStride * (the most stages of any transform): the sub-trees that overwrite a slot
// are then listed about kStageStride diagonals after the last reads of the batch it held.
// With 3M floats per batch the ring of two buffers is 144 MB for three stages (about the
// 126 MB L2; the slots last written are the ones read next).
#ifndef FFA_BATCH_MFLOATS
#define FFA_BATCH_MFLOATS 3
#endif
#ifndef FFA_STAGE_STRIDE
#define FFA_STAGE_STRIDE 2
#endif
constexpr int64_t kBatchFloats = int64_t(FFA_BATCH_MFLOATS) << 20;
constexpr int kStageStride = FFA_STAGE_STRIDE;

// Rows of one shared-memory sub-tree of p bins: the most (at most row_cap) whose
// layout fits in shared memory.
int max_subtree_rows(int p, int row_cap) {
    int n = std::min(row_cap, kBottomMaxRows);
    // + the persistent kernel's queue slot and item records after the layout
    while (n > 1 && bottom_layout(n, n * p, 0).total * 4 + kPersistExtraBytes > kBottomSmemBytes) --n;
    return std::max(n, 1);
}
int depth_for(int m, int p, int row_cap = kBottomMaxRows) {
    const int R = max_subtree_rows(p, row_cap);
    int d = 0;
    while (((int64_t)m + (int64_t(1) << d) - 1) >> d > R) ++d;
    return d;
}

// Rows per top-kernel CTA: the most that fit in shared memory (at most kTopMaxRows).
int top_rows(int p, int L, bool score, int wmax) {
    for (int K = kTopMaxRows; K >= 1; --K)
        if (top_layout(K, L, p, wmax, score).total * 4 + kPersistExtraBytes <= kTopSmemBytes) return K;
    return 0;
}

// Merge levels per top pass for base period p: the most (up to kTopMaxLevels) for which
// at least one row per CTA fits when stored and, if `score`, when scored.
int top_chunk(int p, int wmax, bool score) {
    for (int c = kTopMaxLevels; c >= 1; --c)
        if (top_rows(p, c, false, wmax) >= 1 && (!score || top_rows(p, c, true, wmax) >= 1))
            return c;
    return 0;
}

ffa_status make_widths(const int32_t* h_widths, int32_t nw, int limit, Widths* W,
                       int boxcar = FFA_BOXCAR_PLAIN) {
    if (!h_widths) return fail(FFA_ERR_ARG, "widths is null");
    if (nw < 1 || nw > kMaxWidths) return fail(FFA_ERR_ARG, "nw must be in [1, %d]", kMaxWidths);
    std::memset(W, 0, sizeof(*W));
    W->nw = nw;
    for (int i = 0; i < nw; ++i) {
        const int w = h_widths[i];
        if (w < 1 || w > limit) return fail(FFA_ERR_ARG, "width %d outside [1, %d]", w, limit);
        if (i && w <= h_widths[i - 1]) return fail(FFA_ERR_ARG, "widths must increase strictly");
        W->w[i] = w;
        W->inv_sqrt_w[i] = (float)(1.0 / std::sqrt((double)w));
        if (w > W->wmax) W->wmax = w;
    }
    W->boxcar = boxcar;
    return FFA_OK;
}

ffa_status check_search(int64_t n, double tsamp, double pmin, double pmax, int bmin, int bmax) {
    if (n <= 0) return fail(FFA_ERR_ARG, "n must be positive");
    if (!(tsamp > 0.0) || !std::isfinite(tsamp)) return fail(FFA_ERR_ARG, "tsamp must be > 0");
    if (!(pmin > 0.0) || !(pmax > pmin) || !std::isfinite(pmax))
        return fail(FFA_ERR_ARG, "need 0 < pmin < pmax");
    if (bmin < 2 || bmax < bmin) return fail(FFA_ERR_ARG, "need 2 <= bmin <= bmax");
    if (bmax > kMaxCols) return fail(FFA_ERR_UNSUPPORTED, "bmax above %d", kMaxCols);
    if (pmin / ((double)bmin * tsamp) < 1.0)
        return fail(FFA_ERR_ARG, "pmin / (bmin tsamp) < 1: first downsampling factor below 1");
    if (n > (int64_t(1) << 40)) return fail(FFA_ERR_UNSUPPORTED, "n too large");
    return FFA_OK;
}

void fixed_point(double f, uint64_t* fi, uint64_t* ff) {
    const double fl = std::floor(f);
    *fi = (uint64_t)fl;
    // f - floor(f) is exact in double; scale by 2^64 exactly via ldexp
    *ff = (uint64_t)std::ldexp(f - fl, 64);
}

// Rows produced by all merges of an n-row transform: every node of two or more rows
// produces all of its rows (head ⌊n/2⌋, tail n - ⌊n/2⌋, Sec. 2.2).
double merged_rows(int n) {
    static thread_local std::map<int, double> memo;
    if (n < 2) return 0.0;
    auto it = memo.find(n);
    if (it != memo.end()) return it->second;
    const double r = n + merged_rows(n >> 1) + merged_rows(n - (n >> 1));
    memo[n] = r;
    return r;
}

ffa_status build_plan(Plan& pl) {
    int64_t ds_off = 0, first = 0, trial = 0;
    pl.series_trial0.clear();
    pl.segs.clear();
    pl.blk_seg.clear();
    pl.prefix_len = 0;
    pl.input_total = 0;
    for (const SeriesSpec& sp : pl.series) {
        PrefixSeg sg{sp.x_off, pl.prefix_len, sp.n, (int64_t)pl.blk_seg.size()};
        const int64_t nb = (sp.n + prefix_chunk() - 1) / prefix_chunk();
        if ((int64_t)pl.blk_seg.size() + nb > INT32_MAX) return fail(FFA_ERR_UNSUPPORTED, "input too long");
        pl.blk_seg.insert(pl.blk_seg.end(), (size_t)nb, (int)pl.segs.size());
        pl.segs.push_back(sg);
        pl.prefix_len += sp.n + 1;
        pl.input_total += sp.n;
        const double tsamp = sp.tsamp;
        const double f0 = sp.pmin / ((double)sp.bmin * tsamp);        // Sec. 5.6: tau = Pmin / bmin
        const double fg = ((double)sp.bmax + 1.0) / (double)sp.bmin;  // Sec. 5.3
        const size_t oct0 = pl.oct.size();
        std::vector<double> fac;
        for (int k = 0;; ++k) {
            const double f = f0 * std::pow(fg, (double)k);
            if ((double)sp.bmin * tsamp * f > sp.pmax) break;
            if (k > 4096) return fail(FFA_ERR_UNSUPPORTED, "too many octaves");
            OctaveDesc od{};
            od.nk = (int64_t)std::floor((double)sp.n / f);
            od.out_off = ds_off;
            od.x_off = sp.x_off;
            od.x_n = sp.n;
            od.pre_off = sg.pre_off;
            fixed_point(f, &od.f_int, &od.f_frac);
            pl.oct.push_back(od);
            fac.push_back(f);
            ds_off += (int64_t)align_up((size_t)std::max<int64_t>(od.nk, 0), 4) + 4;
            first += od.nk;
        }
        pl.series_trial0.push_back(trial);
        // Transforms in (octave, p) order (Sec. 5.3, Fig. 4).
        for (size_t kk = 0; kk < fac.size(); ++kk) {
            const OctaveDesc& od = pl.oct[oct0 + kk];
            const double f = fac[kk];
            const double var = (f == std::floor(f)) ? f : f - 1.0 / 3.0;  // App. A.4
            for (int p = sp.bmin; p <= sp.bmax; ++p) {
                const int64_t m64 = od.nk / p;
                if (m64 < 2) continue;
                if (m64 * p >= (int64_t(1) << 31))
                    return fail(FFA_ERR_UNSUPPORTED, "transform too large");
                const int m = (int)m64;
                int64_t kept = 0;  // rows with s (p + 1) < p (m - 1)  (Sec. 2.3)
                kept = (int64_t)p * (m - 1) > 0 ? ((int64_t)p * (m - 1) - 1) / (p + 1) + 1 : 0;
                if (kept > m) kept = m;
                TransformDesc t{};
                t.src_off = od.out_off;
                t.scratch_off = 0;
                t.trial0 = trial;
                t.tau = tsamp * f;
                t.p = p;
                t.m = m;
                t.kept = (int)kept;
                // tiles: the transform's class, else the plan-wide values
                const int ci = pl.tiles.class_of(m, p);
                const TileClass* tc = ci >= 0 ? &pl.tiles.classes[ci] : nullptr;
                const int rcap = tc && tc->subtree_rows ? std::min(pl.row_cap, tc->subtree_rows)
                                                        : pl.row_cap;
                const int lv = tc && tc->top_levels ? tc->top_levels : pl.tiles.top_levels;
                t.depth = depth_for(m, p, rcap);
                t.chunk = top_chunk(p, pl.W.wmax, true);
                if (lv) t.chunk = std::min(t.chunk, lv);
                pl.tr_class.push_back(ci);
                if (t.chunk < 1) return fail(FFA_ERR_UNSUPPORTED, "profile too long");
                t.inv_std = (float)(1.0 / std::sqrt((double)m * var));
                pl.trs.push_back(t);
                trial += kept;
                pl.folded += (int64_t)m * p;
                // arithmetic of the method: one add per element of every merged row
                // (Eq. ffa_merge_rule), then per kept profile p prefix adds and, per
                // width and phase, one subtract and one max (Sec. 5.4)
                pl.ffa_adds += (double)merged_rows(m) * p;
                pl.snr_ops += (double)kept * p * (1.0 + 2.0 * pl.W.nw);
                pl.max_rows = std::max(pl.max_rows, m);
                pl.max_p = std::max(pl.max_p, p);
            }
        }
    }
    pl.series_trial0.push_back(trial);
    pl.ds_total = first;
    pl.ds_floats = ds_off;
    for (size_t k = 0; k < pl.oct.size(); ++k)
        for (int64_t s = 0; s < pl.oct[k].nk; s += kDownsamplePerBlock) {
            if (s > INT32_MAX) return fail(FFA_ERR_UNSUPPORTED, "octave too long");
            pl.ds_blocks.push_back(make_int2((int)k, (int)s));
        }
    pl.ntrials = trial;
    const int wmax = pl.W.wmax;
    const int nw = pl.W.nw;

    // ---- persistent work queue.  Whole-tree transforms (scored inside one CTA) come
    //      first; the others are cut into batches of consecutive transforms, and the
    //      stages of the batches (sub-trees, then top passes) are listed along
    //      diagonals, so that an item's inputs were listed about one batch-stage earlier.
    pl.stage_count.assign(pl.trs.size() * kMaxStages, 0);
    int p0 = 0;
    for (size_t t = 0; t < pl.trs.size(); ++t) {
        const TransformDesc& d = pl.trs[t];
        if (d.depth != 0) continue;
        pl.items.push_back(WorkItem{(int32_t)t, 0, -2, 0, 0});
        pl.stage_count[t * kMaxStages] = 1;
        pl.bottom0_nmax = std::max(pl.bottom0_nmax, d.m);
        pl.bottom0_elems = std::max(pl.bottom0_elems, d.m * d.p);
        p0 = std::max(p0, d.p);
        pl.ffa_bytes += 4.0 * d.m * d.p + 4.0 * nw * d.kept;
    }
    if (pl.bottom0_nmax) {
        const int per_warp = snr_warp_floats(p0, wmax);
        const BottomLayout l0 = bottom_layout(pl.bottom0_nmax, pl.bottom0_elems, 0);
        pl.bottom0_snr_warps = std::min(kBottomThreads / 32, l0.buf_floats / per_warp);
        if (pl.bottom0_snr_warps < 1) pl.bottom0_snr_warps = 1;
        pl.bottom0_snr_floats = pl.bottom0_snr_warps * per_warp;
        pl.smem_floats = std::max(
            pl.smem_floats,
            bottom_layout(pl.bottom0_nmax, pl.bottom0_elems, pl.bottom0_snr_floats).total);
    }
    std::vector<std::vector<int>> batches;
    {
        int64_t bf = 0;
        std::vector<int64_t> off;  // offset of each transform within its batch
        off.assign(pl.trs.size(), 0);
        for (size_t t = 0; t < pl.trs.size(); ++t) {
            TransformDesc& d = pl.trs[t];
            d.batch = -1;
            if (d.depth == 0) continue;
            const int64_t need = (int64_t)d.m * d.p;
            if (batches.empty() || bf + need > kBatchFloats) {
                batches.emplace_back();
                bf = 0;
            }
            batches.back().push_back((int)t);
            d.batch = (int)batches.size() - 1;
            off[t] = bf;
            bf += (int64_t)align_up((size_t)need, 4);
            pl.slot_floats = std::max(pl.slot_floats, bf);
        }
        pl.nbatches = (int)batches.size();
        for (size_t t = 0; t < pl.trs.size(); ++t) pl.trs[t].scratch_off = off[t];  // + slot, below
    }
    // items of each (batch, stage)
    std::vector<std::vector<std::vector<WorkItem>>> st_items(batches.size());
    pl.batch_top.assign(batches.size(), 0);
    int max_stage = 0;
    for (size_t b = 0; b < batches.size(); ++b) {
        auto& sv = st_items[b];
        sv.emplace_back();
        for (int t : batches[b]) {
            const TransformDesc& d = pl.trs[t];
            for (int c = 0; c < (1 << d.depth); ++c) sv[0].push_back(WorkItem{t, c, -1, 0, 0});
            pl.stage_count[(size_t)t * kMaxStages] = 1 << d.depth;
            const int rows = (d.m + (1 << d.depth) - 1) >> d.depth;
            pl.bottom_nmax = std::max(pl.bottom_nmax, rows);
            pl.bottom_elems = std::max(pl.bottom_elems, rows * d.p);
            pl.ffa_bytes += 4.0 * d.m * d.p + 4.0 * nw * d.kept;
            const int np = top_passes(d.depth, d.chunk);
            if (np + 1 > kMaxStages) return fail(FFA_ERR_UNSUPPORTED, "tree too deep");
            for (int j = 0; j < np; ++j) {
                if ((int)sv.size() < j + 2) sv.emplace_back();
                const int dout = top_pass_out_depth(d.depth, d.chunk, j);
                const int L = top_pass_in_depth(d.depth, d.chunk, j) - dout;
                const bool score = j == np - 1;
                int K = top_rows(d.p, L, score, wmax);
                const int ci = pl.tr_class[t];
                const int kr = ci >= 0 && pl.tiles.classes[ci].top_rows ? pl.tiles.classes[ci].top_rows
                                                                         : pl.tiles.top_rows;
                if (kr) K = std::min(K, kr);
                if (K < 1) return fail(FFA_ERR_UNSUPPORTED, "profile too long");
                pl.smem_floats = std::max(pl.smem_floats, top_layout(K, L, d.p, wmax, score).total);
                const int nmax = (d.m + (1 << dout) - 1) >> dout;
                const int lim = score ? d.kept : nmax;
                const int nb = (lim + K - 1) / K;
                const int cnt = score ? nb : (1 << dout) * nb;
                for (int i = 0; i < cnt; ++i)  // pad: the item's table (made on the device)
                    sv[j + 1].push_back(WorkItem{t, i, (int16_t)j, (int16_t)K, pl.ntop++});
                pl.stage_count[(size_t)t * kMaxStages + j + 1] = cnt;
                if (score) pl.batch_top[b] += cnt;
            }
        }
        max_stage = std::max(max_stage, (int)sv.size());
    }
    // The ring: batch b writes slot b % ring once batch b - ring has finished reading it.
    // Batch b's sub-trees are listed on diagonal b, after every item of batch b - ring
    // (diagonals up to b - ring + kStageStride (max_stage - 1) < b), so the wait always
    // ends; within a diagonal the later stages come first.
#ifdef FFA_RING_SLOTS
    pl.ring = std::max(1, std::min(std::max(FFA_RING_SLOTS, kStageStride * max_stage), std::max(pl.nbatches, 1)));
#else
    pl.ring = std::max(1, std::min(kStageStride * max_stage, std::max(pl.nbatches, 1)));
#endif
    for (TransformDesc& d : pl.trs)
        if (d.batch >= 0) d.scratch_off += (int64_t)(d.batch % pl.ring) * pl.slot_floats;
    pl.scratch_floats = (int64_t)pl.ring * pl.slot_floats;
    for (int diag = 0; diag < (int)batches.size() + kStageStride * max_stage; ++diag)
        for (int s = max_stage - 1; s >= 0; --s) {
            const int b = diag - kStageStride * s;
            if (b < 0 || b >= (int)batches.size() || s >= (int)st_items[b].size()) continue;
            pl.items.insert(pl.items.end(), st_items[b][s].begin(), st_items[b][s].end());
        }
    if (pl.bottom_nmax)
        pl.smem_floats =
            std::max(pl.smem_floats, bottom_layout(pl.bottom_nmax, pl.bottom_elems, 0).total);
    pl.smem_floats = (int)round4(pl.smem_floats);  // the queue slot after it is 16-byte aligned
    if (pl.smem_floats * 4 + kPersistExtraBytes > kSmemBytes) return kRetrySmaller;
    pl.nitems = (int)pl.items.size();

    // Tables: octaves | transforms | items | downsampling CTAs | stage counts | batch
    // top-pass counts | prefix series | prefix chunks, each 256-byte aligned.
    size_t o = 0;
    pl.o_oct = o;
    o = align_up(o + pl.oct.size() * sizeof(OctaveDesc), 256);
    pl.o_trs = o;
    o = align_up(o + pl.trs.size() * sizeof(TransformDesc), 256);
    pl.o_items = o;
    o = align_up(o + pl.items.size() * sizeof(WorkItem), 256);
    pl.o_dsblk = o;
    o = align_up(o + pl.ds_blocks.size() * sizeof(int2), 256);
    pl.o_stcnt = o;
    o = align_up(o + pl.stage_count.size() * sizeof(int), 256);
    pl.o_btop = o;
    o = align_up(o + pl.batch_top.size() * sizeof(int), 256);
    pl.o_segs = o;
    o = align_up(o + pl.segs.size() * sizeof(PrefixSeg), 256);
    pl.o_blkseg = o;
    o = align_up(o + pl.blk_seg.size() * sizeof(int), 256);
    pl.tables_bytes = std::max<size_t>(o, 256);

    // Workspace: status | tables | prefix | chunk sums | octave series | scratch ring 0 |
    // scratch ring 1 | completion counters | item heads | top-pass tables
    pl.nchunks = (int64_t)pl.blk_seg.size();
    size_t w = kStatusBytes;
    pl.o_tables = w;
    w = align_up(w + pl.tables_bytes, 256);
    pl.o_prefix = w;
    w = align_up(w + (size_t)pl.prefix_len * sizeof(float2), 256);
    pl.o_partial = w;
    w = align_up(w + (size_t)pl.nchunks * sizeof(float2), 256);
    pl.o_ds = w;
    w = align_up(w + (size_t)pl.ds_floats * 4, 256);
    pl.o_s0 = w;
    w = align_up(w + (size_t)pl.scratch_floats * 4, 256);
    pl.o_s1 = w;
    w = align_up(w + (size_t)pl.scratch_floats * 4, 256);
    pl.o_counters = w;  // queue counter, then per (transform, stage) and per batch completions
    pl.counter_bytes = (1 + pl.trs.size() * kMaxStages + pl.batch_top.size()) * sizeof(int);
    w = align_up(w + pl.counter_bytes, 256);
    pl.o_heads = w;  // one head per queue position (made on the device)
    w = align_up(w + (size_t)pl.nitems * sizeof(ItemHead), 256);
    pl.o_toptab = w;  // one table per top-pass item (made on the device)
    w = align_up(w + (size_t)pl.ntop * kTopRecBytes, 256);
    pl.ws_bytes = w;
    // host-buffer variant: + input and outputs
    pl.o_hx = w;
    w = align_up(w + (size_t)pl.n * 4, 256);
    pl.o_hper = w;
    w = align_up(w + (size_t)pl.ntrials * 8, 256);
    pl.o_hfb = w;
    w = align_up(w + (size_t)pl.ntrials * 4, 256);
    pl.o_hsnr = w;
    w = align_up(w + (size_t)pl.ntrials * nw * 4, 256);
    pl.ws_host_bytes = w;

    return FFA_OK;
}

// Page-locked copy of the plan's tables, made on first execution (planning alone needs
// no CUDA device).  Copied into the workspace on every call.
ffa_status ensure_pinned(Plan& pl) {
    if (fault("alloc")) return fail(FFA_ERR_CUDA, "injected fault: alloc");
    if (fault("launch")) return fail(FFA_ERR_CUDA, "injected fault: launch");
    std::lock_guard<std::mutex> lk(g_plan_mu);
    if (pl.pinned) return FFA_OK;
    void* p = nullptr;
    FFA_CUDA(cudaHostAlloc(&p, pl.tables_bytes, cudaHostAllocDefault), "cudaHostAlloc");
    char* h = static_cast<char*>(p);
    std::memset(h, 0, pl.tables_bytes);
    std::memcpy(h + pl.o_oct, pl.oct.data(), pl.oct.size() * sizeof(OctaveDesc));
    std::memcpy(h + pl.o_trs, pl.trs.data(), pl.trs.size() * sizeof(TransformDesc));
    std::memcpy(h + pl.o_items, pl.items.data(), pl.items.size() * sizeof(WorkItem));
    std::memcpy(h + pl.o_dsblk, pl.ds_blocks.data(), pl.ds_blocks.size() * sizeof(int2));
    std::memcpy(h + pl.o_stcnt, pl.stage_count.data(), pl.stage_count.size() * sizeof(int));
    std::memcpy(h + pl.o_btop, pl.batch_top.data(), pl.batch_top.size() * sizeof(int));
    std::memcpy(h + pl.o_segs, pl.segs.data(), pl.segs.size() * sizeof(PrefixSeg));
    std::memcpy(h + pl.o_blkseg, pl.blk_seg.data(), pl.blk_seg.size() * sizeof(int));
    pl.pinned = p;
    return FFA_OK;
}

// Plan of a list of series, built afresh.  Widths must lie below every series' bmin.
ffa_status make_plan_series(const std::vector<SeriesSpec>& series, const int32_t* h_widths,
                            int32_t nw, const Tiles& tiles, std::unique_ptr<Plan>* out) {
    if (series.empty()) return fail(FFA_ERR_ARG, "no series");
    int bmin_all = INT32_MAX;
    int64_t span = 0;
    for (const SeriesSpec& s : series) {
        ffa_status st = check_search(s.n, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax);
        if (st != FFA_OK) return st;
        if (s.x_off < 0) return fail(FFA_ERR_ARG, "negative series offset");
        bmin_all = std::min(bmin_all, s.bmin);
        span = std::max(span, s.x_off + s.n);
    }
    Widths W;
    ffa_status st = make_widths(h_widths, nw, bmin_all - 1, &W,  // below the smallest base period
                                tiles.boxcar);
    if (st != FFA_OK) return st;
    std::unique_ptr<Plan> pl;
    for (int cap = tiles.subtree_rows ? tiles.subtree_rows : kBottomMaxRows;;) {
        pl = std::make_unique<Plan>();
        pl->tiles = tiles;
        pl->series = series;
        pl->n = span;
        pl->widths.assign(h_widths, h_widths + nw);
        pl->W = W;
        pl->row_cap = cap;
        st = build_plan(*pl);
        if (st != kRetrySmaller) break;
        // sub-trees of different widths share one launch: lower the row limit below the
        // largest sub-tree of this plan and replan
        cap = std::min(cap, std::max(pl->bottom_nmax, pl->bottom0_nmax)) - 1;
        if (cap < 2) return fail(FFA_ERR_UNSUPPORTED, "profile too long");
    }
    if (st != FFA_OK) return st;
    *out = std::move(pl);
    return FFA_OK;
}

// Plans are cached by parameters for the life of the process (or until
// ffa_plan_cache_clear): their page-locked tables are the source of copies that a
// captured CUDA graph replays, so they are never evicted behind the caller's back.
using PlanKey = std::tuple<std::vector<SeriesSpec>, std::vector<int>, Tiles>;
std::map<PlanKey, std::unique_ptr<Plan>> g_plans;

ffa_status get_plan_series(const std::vector<SeriesSpec>& series, const int32_t* h_widths,
                           int32_t nw, const Tiles& tiles, Plan** out) {
    if (fault("plan")) return fail(FFA_ERR_UNSUPPORTED, "injected fault: plan");
    if (nw > 0 && !h_widths) return fail(FFA_ERR_ARG, "widths is null");
    PlanKey key{series, std::vector<int>(h_widths, h_widths + std::max(nw, 0)), tiles};
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        auto it = g_plans.find(key);
        if (it != g_plans.end()) {
            *out = it->second.get();
            return FFA_OK;
        }
    }
    std::unique_ptr<Plan> pl;
    ffa_status st = make_plan_series(series, h_widths, nw, tiles, &pl);
    if (st != FFA_OK) return st;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto ins = g_plans.emplace(key, std::move(pl));  // a concurrent twin keeps the first
    *out = ins.first->second.get();
    return FFA_OK;
}

ffa_status get_plan(int64_t n, double tsamp, double pmin, double pmax, int bmin, int bmax,
                    const int32_t* h_widths, int32_t nw, const Tiles& tiles, Plan** out) {
    return get_plan_series({SeriesSpec{0, n, tsamp, pmin, pmax, bmin, bmax}}, h_widths, nw, tiles,
                           out);
}

// A batch of series cut into chunks that each run as one periodogram launch sequence
// within a workspace budget.
struct BatchChunk {
    int first, count;   // series [first, first + count)
    int64_t x_lo;       // input offset of the chunk (its series' offsets are relative)
    int64_t trial0;     // first trial of the chunk in the batch output
    std::shared_ptr<Plan> plan;  // chunks of the same shape share one plan
};
struct Batch {
    std::vector<BatchChunk> chunks;
    std::vector<int64_t> trial0;  // per series, + total
    size_t ws_bytes = 0;
    int ntransforms = 0;
    int64_t folded = 0, input = 0;
};
using BatchKey = std::tuple<std::vector<SeriesSpec>, std::vector<int>, size_t, Tiles>;
std::map<BatchKey, std::unique_ptr<Batch>> g_batches;

ffa_status get_batch(const ffa_series* h_series, int32_t nseries, const int32_t* h_widths,
                     int32_t nw, size_t budget, const Tiles& tiles, Batch** out) {
    if (fault("plan")) return fail(FFA_ERR_UNSUPPORTED, "injected fault: plan");
    if (!h_series || nseries < 1) return fail(FFA_ERR_ARG, "no series");
    if (nw > 0 && !h_widths) return fail(FFA_ERR_ARG, "widths is null");
    std::vector<SeriesSpec> all(nseries);
    for (int i = 0; i < nseries; ++i) {
        const ffa_series& s = h_series[i];
        if (s.offset < 0) return fail(FFA_ERR_ARG, "series %d has a negative offset", i);
        all[i] = SeriesSpec{s.offset, s.n, s.tsamp, s.pmin, s.pmax, s.bmin, s.bmax};
    }
    BatchKey key{all, std::vector<int>(h_widths, h_widths + std::max(nw, 0)), budget, tiles};
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        auto it = g_batches.find(key);
        if (it != g_batches.end()) {
            *out = it->second.get();
            return FFA_OK;
        }
    }
    auto B = std::make_unique<Batch>();
    // workspace of each series searched alone, the unit of the chunk budget: its own
    // part (tables, prefix sums, octave series, records) and its scratch ring, which the
    // series of a chunk share (a chunk's ring is about the largest of theirs)
    std::vector<size_t> est(nseries), ring(nseries);
    std::map<SeriesSpec, std::pair<size_t, size_t>> alone;  // series of the same shape plan alike
    for (int i = 0; i < nseries; ++i) {
        SeriesSpec s = all[i];
        s.x_off = 0;
        auto it = alone.find(s);
        if (it == alone.end()) {
            std::unique_ptr<Plan> p1;
            ffa_status st = make_plan_series({s}, h_widths, nw, tiles, &p1);
            if (st != FFA_OK) return st;
            const size_t r = 2 * (size_t)p1->scratch_floats * 4;
            it = alone.emplace(s, std::make_pair(p1->ws_bytes - std::min(r, p1->ws_bytes), r)).first;
        }
        est[i] = it->second.first;
        ring[i] = it->second.second;
    }
    std::map<std::vector<SeriesSpec>, std::shared_ptr<Plan>> shapes;
    int64_t trial = 0;
    for (int i = 0; i < nseries;) {
        int j = i;
        size_t acc = 0, rmax = 0;
        while (j < nseries && (j == i || acc + est[j] + std::max(rmax, ring[j]) <= budget)) {
            acc += est[j];
            rmax = std::max(rmax, ring[j]);
            ++j;
        }
        std::vector<SeriesSpec> part(all.begin() + i, all.begin() + j);
        int64_t lo = part[0].x_off;
        for (const SeriesSpec& s : part) lo = std::min(lo, s.x_off);
        for (SeriesSpec& s : part) s.x_off -= lo;
        BatchChunk c{i, j - i, lo, trial, nullptr};
        auto sh = shapes.find(part);
        if (sh == shapes.end()) {
            std::unique_ptr<Plan> pc;
            ffa_status st = make_plan_series(part, h_widths, nw, tiles, &pc);
            if (st != FFA_OK) return st;
            sh = shapes.emplace(part, std::shared_ptr<Plan>(std::move(pc))).first;
        }
        c.plan = sh->second;
        for (int q = 0; q < j - i; ++q) B->trial0.push_back(trial + c.plan->series_trial0[q]);
        trial += c.plan->ntrials;
        B->ws_bytes = std::max(B->ws_bytes, c.plan->ws_bytes);
        B->ntransforms += (int)c.plan->trs.size();
        B->folded += c.plan->folded;
        for (const SeriesSpec& s : part) B->input += s.n;
        B->chunks.push_back(std::move(c));
        i = j;
    }
    B->trial0.push_back(trial);
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto ins = g_batches.emplace(key, std::move(B));
    *out = ins.first->second.get();
    return FFA_OK;
}

// Issues the whole periodogram on `st`: tables upload, prefix, downsampling, then
// the FFA + S/N launches group by group.
// A second stream per host thread and device, with a fork and a join event: the
// item records are made on it while the prefix sums and downsampling run.  Made on
// a thread's first periodogram call on a device (so that call should precede any stream
// capture); if it cannot be made, everything runs on the caller's stream.
struct SideStream {
    int dev = -1;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

constexpr int kMaxDevices = 64;
SideStream* side_stream() {
    thread_local SideStream t[kMaxDevices];  // one per device, made once per (thread, device)
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    if (t[dev].dev == dev) return &t[dev];
    SideStream n;
    n.dev = dev;
    if (cudaStreamCreateWithFlags(&n.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&n.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&n.join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();  // clear; fall back to the caller's stream
        return nullptr;
    }
    t[dev] = n;
    return &t[dev];
}

ffa_status run_periodogram(const Plan& pl, const void* d_x, int dtype, double* d_periods,
                           int32_t* d_foldbins, float* d_snr, char* ws, cudaStream_t st,
                           bool reset_status = true) {
    unsigned* status = reinterpret_cast<unsigned*>(ws);
    if (reset_status)  // a batch keeps the status of its earlier chunks
        FFA_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st), "cudaMemsetAsync");
    FFA_CUDA(cudaMemcpyAsync(ws + pl.o_tables, pl.pinned, pl.tables_bytes, cudaMemcpyHostToDevice,
                             st),
             "cudaMemcpyAsync(tables)");
    const OctaveDesc* d_oct = reinterpret_cast<const OctaveDesc*>(ws + pl.o_tables + pl.o_oct);
    const TransformDesc* d_trs =
        reinterpret_cast<const TransformDesc*>(ws + pl.o_tables + pl.o_trs);
    const WorkItem* d_items = reinterpret_cast<const WorkItem*>(ws + pl.o_tables + pl.o_items);
    float2* prefix = reinterpret_cast<float2*>(ws + pl.o_prefix);
    float* ds = reinterpret_cast<float*>(ws + pl.o_ds);
    float* s0 = reinterpret_cast<float*>(ws + pl.o_s0);
    float* s1 = reinterpret_cast<float*>(ws + pl.o_s1);

    // ---- parameters of the persistent launch (the item records are made first)
    int* counters = reinterpret_cast<int*>(ws + pl.o_counters);
    PersistentParams pp{};
    BottomParams& bp = pp.bottom;
    bp.src = ds;
    bp.dst = s0;  // sub-trees of a transform with P top passes land in buffer P % 2
    bp.dst_odd = s1;
    bp.trs = d_trs;
    bp.widths = pl.W;
    bp.periods = d_periods;
    bp.foldbins = d_foldbins;
    bp.snr = d_snr;
    bp.status = status;
    bp.nmax = pl.bottom_nmax;
    bp.elems_max = pl.bottom_elems;
    bp.src_cap = pl.ds_floats;
    bp.dst_cap = pl.scratch_floats;
    bp.ntrials = pl.ntrials;
    pp.bottom_snr = bp;
    pp.bottom_snr.nmax = pl.bottom0_nmax;
    pp.bottom_snr.elems_max = pl.bottom0_elems;
    pp.bottom_snr.snr_warps = pl.bottom0_snr_warps;
    pp.bottom_snr.snr_floats = pl.bottom0_snr_floats;
    TopParams& tp = pp.top;
    tp.buf0 = s0;
    tp.buf1 = s1;
    tp.trs = d_trs;
    tp.widths = pl.W;
    tp.periods = d_periods;
    tp.foldbins = d_foldbins;
    tp.snr = d_snr;
    tp.status = status;
    tp.items = d_items;
    tp.buf_cap = pl.scratch_floats;
    tp.ntrials = pl.ntrials;
    ItemHead* heads = reinterpret_cast<ItemHead*>(ws + pl.o_heads);
    int* toptab = reinterpret_cast<int*>(ws + pl.o_toptab);
    pp.heads = heads;
    pp.tables = toptab;
    pp.nitems = pl.nitems;
    pp.queue = counters;
    pp.done = counters + 1;
    pp.smem_floats = pl.smem_floats;
    pp.wait_cycles = (long long)(g_wait_ms.load() * kCyclesPerMs);
    pp.ncounters = (int)(pl.counter_bytes / sizeof(int)) - 1;
    pp.ntables = pl.ntop;
    RecParams rp{};
    rp.top = tp;
    rp.stage_count = reinterpret_cast<const int*>(ws + pl.o_tables + pl.o_stcnt);
    rp.batch_top = reinterpret_cast<const int*>(ws + pl.o_tables + pl.o_btop);
    rp.nitems = pl.nitems;
    rp.ring = pl.ring;
    rp.nbatches = pl.nbatches;
    rp.batch_base = (int)(pl.trs.size() * kMaxStages);
    rp.inject_tr = -1;
    if (fault("stage"))  // the first transform with a top pass
        for (size_t t = 0; t < pl.trs.size() && rp.inject_tr < 0; ++t)
            if (pl.trs[t].depth > 0) rp.inject_tr = (int)t;
    rp.heads = heads;
    rp.tables = toptab;
    rp.ntables = pl.ntop;
    rp.status = status;

    // ---- item records on a side stream, concurrent with prefix sums and
    //      downsampling (they need only the tables); joined before the FFA launch
    SideStream* side = side_stream();
    cudaStream_t sp = st;
    if (side && pl.nitems > 0) {
        FFA_CUDA(cudaEventRecord(side->fork, st), "cudaEventRecord(fork)");
        FFA_CUDA(cudaStreamWaitEvent(side->s, side->fork, 0), "cudaStreamWaitEvent(fork)");
        sp = side->s;
    }
    FFA_CUDA(launch_item_recs(rp, sp), "item record launch");
    if (sp != st) {
        FFA_CUDA(cudaEventRecord(side->join, sp), "cudaEventRecord(join)");
    }

    PrefixParams xp{};
    xp.x = d_x;
    xp.dtype = dtype;
    xp.segs = reinterpret_cast<const PrefixSeg*>(ws + pl.o_tables + pl.o_segs);
    xp.blk_seg = reinterpret_cast<const int*>(ws + pl.o_tables + pl.o_blkseg);
    xp.nsegs = (int)pl.segs.size();
    xp.partial = reinterpret_cast<float2*>(ws + pl.o_partial);
    xp.prefix = prefix;
    xp.nchunks = pl.nchunks;
    xp.total = pl.input_total;
    xp.x_cap = pl.n;
    xp.prefix_cap = pl.prefix_len;
    xp.status = status;
    FFA_CUDA(launch_prefix(xp, st), "prefix launch");
    DownsampleParams dp{};
    dp.x = d_x;
    dp.dtype = dtype;
    dp.n = pl.n;
    dp.prefix = prefix;
    dp.oct = d_oct;
    dp.blocks = reinterpret_cast<const int2*>(ws + pl.o_tables + pl.o_dsblk);
    dp.nblocks = (int)pl.ds_blocks.size();
    dp.total = pl.ds_total;
    dp.out = ds;
    dp.x_cap = pl.n;
    dp.prefix_cap = pl.prefix_len;
    dp.out_cap = pl.ds_floats;
    dp.status = status;
    FFA_CUDA(launch_downsample(dp, st), "downsample launch");

    // ---- all FFA work: one persistent launch over the plan's queue
    FFA_CUDA(cudaMemsetAsync(counters, 0, pl.counter_bytes, st), "cudaMemsetAsync(counters)");
    if (sp != st) FFA_CUDA(cudaStreamWaitEvent(st, side->join, 0), "cudaStreamWaitEvent(join)");
    {
        LaunchScope ls(kFfaPersistent, pl.ffa_bytes, st);
        FFA_CUDA(launch_persistent(pp, pl.smem_floats * 4 + kPersistExtraBytes, st),
                 "ffa_persistent launch");
    }
    return FFA_OK;
}

bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255) == 0; }

}  // namespace

thread_local bool g_no_alloc_call = false;
ffa_status set_error(ffa_status st, const char* msg) { return fail(st, "%s", msg); }

// ---------------------------------------------------------------------------------
LaunchScope::LaunchScope(int k, double b, cudaStream_t s) : kind(k), bytes(b), stream(s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_no_alloc_call) return;  // no event objects are created on the no-allocation path
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    ev0 = pool_get();
    ev1 = pool_get();
    cudaEventRecord(ev0, s);
}
LaunchScope::~LaunchScope() {
    if (!ev0) return;
    cudaEventRecord(ev1, stream);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_pending.push_back(ProfRec{kind, ev0, ev1, bytes});
}

}  // namespace ffa

using namespace ffa;

// =================================================================================
// C ABI
// =================================================================================
extern "C" {

const char* ffa_last_error(void) { return g_err.c_str(); }
const char* ffa_version(void) { return "libffa 0.1 (sm_103a)"; }

int64_t ffa_launch_count(void) { return g_launches.load(); }
ffa_status ffa_set_wait_limit_ms(double ms) {
    if (!(ms > 0.0) || ms > 60000.0) return fail(FFA_ERR_ARG, "wait limit must be in (0, 60000] ms");
    g_wait_ms.store(ms);
    return FFA_OK;
}
int32_t ffa_kernel_kinds(void) { return kAllKinds; }
const char* ffa_kernel_name(int32_t kind) {
    return (kind >= 0 && kind < kAllKinds) ? kKindNames[kind] : "";
}
ffa_status ffa_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return FFA_OK;
}
ffa_status ffa_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_pending();
    for (auto& a : g_acc) a = ProfAcc();
    return FFA_OK;
}
ffa_status ffa_profile_query(int32_t kind, int64_t* launches, double* total_ms, double* alg_bytes) {
    if (kind < 0 || kind >= kAllKinds) return fail(FFA_ERR_ARG, "bad kernel kind");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_pending();
    if (launches) *launches = g_acc[kind].launches;
    if (total_ms) *total_ms = g_acc[kind].ms;
    if (alg_bytes) *alg_bytes = g_acc[kind].bytes;
    return FFA_OK;
}

// ---------------------------------------------------------------------------------
ffa_status ffa_downsample_workspace(int64_t n, size_t* bytes) {
    if (!bytes) return fail(FFA_ERR_ARG, "bytes is null");
    if (n <= 0) return fail(FFA_ERR_ARG, "n must be positive");
    const int64_t nch = (n + prefix_chunk() - 1) / prefix_chunk();
    *bytes = kStatusBytes + align_up((size_t)(n + 1) * sizeof(float2), 256) +
             align_up((size_t)nch * sizeof(float2), 256);
    return FFA_OK;
}

ffa_status ffa_downsample_length(int64_t n, double factor, int64_t* n_out) {
    if (!n_out) return fail(FFA_ERR_ARG, "null pointer");
    if (n <= 0) return fail(FFA_ERR_ARG, "n must be positive");
    if (!(factor >= 1.0) || !std::isfinite(factor) || factor >= 4294967296.0)
        return fail(FFA_ERR_ARG, "factor must be a finite number >= 1");
    *n_out = (int64_t)std::floor((double)n / factor);  // complete windows only
    return FFA_OK;
}

ffa_status ffa_downsample(const float* d_x, int64_t n, double factor, float* d_out,
                          int64_t out_cap, int64_t* n_out, void* d_ws, size_t ws_bytes,
                          void* stream) {
    if (!d_x || !d_out || !n_out || !d_ws) return fail(FFA_ERR_ARG, "null pointer");
    ffa_status st0 = ffa_downsample_length(n, factor, n_out);
    if (st0 != FFA_OK) return st0;
    if (!aligned256(d_ws)) return fail(FFA_ERR_ARG, "workspace must be 256-byte aligned");
    const int64_t nk = *n_out;
    if (out_cap < nk) return fail(FFA_ERR_CAPACITY, "out_cap %lld < %lld", (long long)out_cap,
                                  (long long)nk);
    size_t need = 0;
    ffa_downsample_workspace(n, &need);
    if (ws_bytes < need) return fail(FFA_ERR_CAPACITY, "workspace needs %zu bytes", need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(d_ws);
    const int64_t nch = (n + prefix_chunk() - 1) / prefix_chunk();
    float2* prefix = reinterpret_cast<float2*>(ws + kStatusBytes);
    float2* partial =
        reinterpret_cast<float2*>(ws + kStatusBytes + align_up((size_t)(n + 1) * sizeof(float2), 256));
    FFA_CUDA(cudaMemsetAsync(ws, 0, sizeof(unsigned), st), "cudaMemsetAsync");
    if (nk == 0) return FFA_OK;
    PrefixParams pp{};
    pp.x = d_x;
    pp.dtype = FFA_F32;
    pp.single = PrefixSeg{0, 0, n, 0};
    pp.nsegs = 1;
    pp.partial = partial;
    pp.prefix = prefix;
    pp.nchunks = nch;
    pp.total = n;
    pp.x_cap = n;
    pp.prefix_cap = n + 1;
    pp.status = reinterpret_cast<unsigned*>(ws);
    FFA_CUDA(launch_prefix(pp, st), "prefix launch");
    DownsampleParams dp{};
    dp.x = d_x;
    dp.dtype = FFA_F32;
    dp.n = n;
    dp.prefix = prefix;
    dp.oct = nullptr;
    dp.blocks = nullptr;
    if ((nk + kDownsamplePerBlock - 1) / kDownsamplePerBlock > INT32_MAX)
        return fail(FFA_ERR_UNSUPPORTED, "series too long");
    dp.nblocks = (int)((nk + kDownsamplePerBlock - 1) / kDownsamplePerBlock);
    dp.total = nk;
    dp.out = d_out;
    dp.single.nk = nk;
    dp.single.x_off = 0;
    dp.single.x_n = n;
    dp.single.pre_off = 0;
    dp.x_cap = n;
    dp.prefix_cap = n + 1;
    dp.out_cap = out_cap;
    dp.status = reinterpret_cast<unsigned*>(ws);
    fixed_point(factor, &dp.single.f_int, &dp.single.f_frac);
    FFA_CUDA(launch_downsample(dp, st), "downsample launch");
    return FFA_OK;
}

// ---------------------------------------------------------------------------------
ffa_status ffa_transform_workspace(int32_t rows, int32_t cols, size_t* bytes) {
    if (!bytes) return fail(FFA_ERR_ARG, "bytes is null");
    if (rows < 1 || cols < 1) return fail(FFA_ERR_ARG, "rows and cols must be >= 1");
    if (cols > kMaxCols) return fail(FFA_ERR_UNSUPPORTED, "cols above %d", kMaxCols);
    if ((int64_t)rows * cols >= (int64_t(1) << 31)) return fail(FFA_ERR_UNSUPPORTED, "block too large");
    const int D = depth_for(rows, cols);
    *bytes = kStatusBytes + (D ? align_up((size_t)rows * cols * 4, 256) : 0);
    return FFA_OK;
}

ffa_status ffa_transform(const float* d_in, int32_t rows, int32_t cols, float* d_out,
                         void* d_ws, size_t ws_bytes, void* stream) {
    if (!d_in || !d_out || !d_ws) return fail(FFA_ERR_ARG, "null pointer");
    size_t need = 0;
    ffa_status stt = ffa_transform_workspace(rows, cols, &need);
    if (stt != FFA_OK) return stt;
    if (!aligned256(d_ws)) return fail(FFA_ERR_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < need) return fail(FFA_ERR_CAPACITY, "workspace needs %zu bytes", need);
    const char* a0 = reinterpret_cast<const char*>(d_in);
    const char* b0 = reinterpret_cast<const char*>(d_out);
    const size_t nbytes = (size_t)rows * cols * 4;
    if (a0 < b0 + nbytes && b0 < a0 + nbytes) return fail(FFA_ERR_ARG, "d_in and d_out overlap");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(d_ws);
    unsigned* status = reinterpret_cast<unsigned*>(ws);
    float* scratch = reinterpret_cast<float*>(ws + kStatusBytes);
    FFA_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st), "cudaMemsetAsync");

    const int D = depth_for(rows, cols);
    TransformDesc t{};
    t.p = cols;
    t.m = rows;
    t.kept = rows;
    t.depth = D;
    t.chunk = top_chunk(cols, 0, false);
    if (t.chunk < 1) return fail(FFA_ERR_UNSUPPORTED, "cols too large for the top kernel");
    const int npass = top_passes(D, t.chunk);
    BottomParams bp{};
    bp.src = d_in;
    bp.dst = d_out;     // with P top passes the sub-trees go to buffer P % 2: d_out or scratch
    bp.dst_odd = scratch;
    bp.single = t;
    bp.status = status;
    const int rows_d = (rows + (1 << D) - 1) >> D;
    bp.nmax = rows_d;
    bp.elems_max = rows_d * cols;
    bp.src_cap = (long long)rows * cols;
    bp.dst_cap = (long long)rows * cols;
    const int smem = bottom_layout(bp.nmax, bp.elems_max, 0).total * 4;
    {
        LaunchScope ls(kFfaBottom, 8.0 * rows * cols, st);
        FFA_CUDA(launch_bottom(bp, 1 << D, smem, false, st), "ffa_bottom launch");
    }
    for (int j = 0; j < npass; ++j) {
        const int dout = top_pass_out_depth(D, t.chunk, j);
        const int L = top_pass_in_depth(D, t.chunk, j) - dout;
        const int K = top_rows(cols, L, false, 0);
        if (K < 1) return fail(FFA_ERR_UNSUPPORTED, "cols too large for the top kernel");
        const int nmax = (rows + (1 << dout) - 1) >> dout;
        const int nb = (nmax + K - 1) / K;
        TopParams tp{};
        tp.buf0 = d_out;
        tp.buf1 = scratch;
        tp.single = t;
        tp.status = status;
        tp.single_pass = j;
        tp.single_rows = K;
        tp.buf_cap = (long long)rows * cols;
        LaunchScope ls(kFfaTop, 8.0 * rows * cols, st);
        FFA_CUDA(launch_top(tp, (1 << dout) * nb, top_layout(K, L, cols, 0, false).total * 4, st),
                 "ffa_top launch");
    }
    return FFA_OK;
}

// ---------------------------------------------------------------------------------
ffa_status ffa_boxcar_snr(const float* d_prof, int32_t rows, int32_t cols,
                          const int32_t* h_widths, int32_t nw, double stdnoise, float* d_snr,
                          void* stream) {
    return ffa_boxcar_snr_template(d_prof, rows, cols, h_widths, nw, stdnoise, FFA_BOXCAR_PLAIN,
                                   d_snr, stream);
}

ffa_status ffa_boxcar_snr_template(const float* d_prof, int32_t rows, int32_t cols,
                                   const int32_t* h_widths, int32_t nw, double stdnoise,
                                   int32_t boxcar, float* d_snr, void* stream) {
    if (boxcar != FFA_BOXCAR_PLAIN && boxcar != FFA_BOXCAR_ZERO_MEAN)
        return fail(FFA_ERR_ARG, "boxcar must be FFA_BOXCAR_PLAIN or FFA_BOXCAR_ZERO_MEAN");
    if (!d_prof || !d_snr) return fail(FFA_ERR_ARG, "null pointer");
    if (rows < 0 || cols < 1) return fail(FFA_ERR_ARG, "rows >= 0 and cols >= 1 required");
    if (cols > kMaxCols) return fail(FFA_ERR_UNSUPPORTED, "cols above %d", kMaxCols);
    if (!(stdnoise > 0.0) || !std::isfinite(stdnoise)) return fail(FFA_ERR_ARG, "stdnoise must be > 0");
    SnrParams sp{};
    // the zero-mean template needs off-pulse bins: w < cols
    ffa_status stt = make_widths(h_widths, nw, boxcar ? cols - 1 : cols, &sp.widths, boxcar);
    if (stt != FFA_OK) return stt;
    sp.prof = d_prof;
    sp.rows = rows;
    sp.cols = cols;
    sp.inv_std = (float)(1.0 / stdnoise);
    sp.snr = d_snr;
    sp.warp_floats = snr_warp_floats(cols, sp.widths.wmax);
    if (8 * sp.warp_floats * 4 > kSmemBytes)
        return fail(FFA_ERR_UNSUPPORTED, "cols + max width too large for shared memory");
    FFA_CUDA(launch_snr(sp, static_cast<cudaStream_t>(stream)), "boxcar_snr launch");
    return FFA_OK;
}

// ---------------------------------------------------------------------------------
ffa_status ffa_normalise_workspace(int64_t n, size_t* bytes) {
    if (!bytes) return fail(FFA_ERR_ARG, "bytes is null");
    if (n <= 0) return fail(FFA_ERR_ARG, "n must be positive");
    *bytes = kStatusBytes + align_up((size_t)kNormaliseBlocks * sizeof(double), 256);
    return FFA_OK;
}

ffa_status ffa_normalise(const float* d_x, int64_t n, void* d_out, ffa_dtype out_dtype,
                         double* d_mean_std, void* d_ws, size_t ws_bytes, void* stream) {
    if (!d_x || !d_out || !d_mean_std || !d_ws) return fail(FFA_ERR_ARG, "null pointer");
    if (out_dtype != FFA_F32 && out_dtype != FFA_F16 && out_dtype != FFA_I8)
        return fail(FFA_ERR_ARG, "bad dtype");
    size_t need = 0;
    ffa_status st = ffa_normalise_workspace(n, &need);
    if (st != FFA_OK) return st;
    if (!aligned256(d_ws)) return fail(FFA_ERR_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < need) return fail(FFA_ERR_CAPACITY, "workspace needs %zu bytes", need);
    NormaliseParams P{};
    P.x = d_x;
    P.n = n;
    P.partial = reinterpret_cast<double*>(static_cast<char*>(d_ws) + kStatusBytes);
    P.nblocks = kNormaliseBlocks;
    P.stats = d_mean_std;
    P.out = d_out;
    P.out_dtype = out_dtype;
    FFA_CUDA(launch_normalise(P, static_cast<cudaStream_t>(stream)), "normalise launch");
    return FFA_OK;
}

// ---------------------------------------------------------------------------------
// The tiles a plan's transforms got: plan-wide maxima, and the same per class.
void effective_tiles(const Plan& pl, ffa_plan_opts* o) {
    std::memset(o, 0, sizeof(*o));
    o->boxcar = pl.W.boxcar;
    o->nclasses = (int32_t)pl.tiles.classes.size();
    for (int c = 0; c < o->nclasses; ++c) {
        o->classes[c].m_max = pl.tiles.classes[c].m_max;
        o->classes[c].p_max = pl.tiles.classes[c].p_max;
    }
    auto bump = [](int32_t& v, int x) { v = std::max(v, (int32_t)x); };
    for (size_t t = 0; t < pl.trs.size(); ++t) {
        const TransformDesc& d = pl.trs[t];
        const int rows = (d.m + (1 << d.depth) - 1) >> d.depth;
        const int ci = pl.tr_class[t];
        bump(o->subtree_rows, rows);
        if (d.depth > 0) bump(o->top_levels, d.chunk);
        if (ci >= 0) {
            bump(o->classes[ci].subtree_rows, rows);
            if (d.depth > 0) bump(o->classes[ci].top_levels, d.chunk);
        }
    }
    for (const WorkItem& it : pl.items) {
        if (it.pass < 0) continue;
        bump(o->top_rows, it.rows);
        const int ci = pl.tr_class[it.tr];
        if (ci >= 0) bump(o->classes[ci].top_rows, it.rows);
    }
}

ffa_status ffa_periodogram_plan_opts(int64_t n, double tsamp, double pmin, double pmax,
                                      int32_t bmin, int32_t bmax, const int32_t* h_widths,
                                      int32_t nw, const ffa_plan_opts* opts, ffa_plan_info* out) {
    if (!out) return fail(FFA_ERR_ARG, "out is null");
    Tiles T;
    ffa_status st = read_tiles(opts, &T);
    if (st != FFA_OK) return st;
    Plan* pl = nullptr;
    st = get_plan(n, tsamp, pmin, pmax, bmin, bmax, h_widths, nw, T, &pl);
    if (st != FFA_OK) return st;
    std::memset(out, 0, sizeof(*out));
    out->ntrials = pl->ntrials;
    out->noctaves = (int32_t)pl->oct.size();
    out->ntransforms = (int32_t)pl->trs.size();
    out->nwidths = nw;
    out->max_rows = pl->max_rows;
    out->downsampled_samples = pl->ds_total;
    out->folded_samples = pl->folded;
    out->ffa_adds = pl->ffa_adds;
    out->snr_ops = pl->snr_ops;
    out->workspace_bytes = pl->ws_bytes;
    out->host_workspace_bytes = pl->ws_host_bytes;
    effective_tiles(*pl, &out->opts);
    return FFA_OK;
}

ffa_status ffa_periodogram_plan(int64_t n, double tsamp, double pmin, double pmax, int32_t bmin,
                                int32_t bmax, const int32_t* h_widths, int32_t nw,
                                ffa_plan_info* out) {
    return ffa_periodogram_plan_opts(n, tsamp, pmin, pmax, bmin, bmax, h_widths, nw, nullptr, out);
}

ffa_status ffa_periodogram_opts(const void* d_x, ffa_dtype dtype, int64_t n, double tsamp,
                                 double pmin, double pmax, int32_t bmin, int32_t bmax,
                                 const int32_t* h_widths, int32_t nw, const ffa_plan_opts* opts,
                                 double* d_periods, int32_t* d_foldbins, float* d_snr,
                                 int64_t ntrials_cap, void* d_ws, size_t ws_bytes, void* stream) {
    if (!d_x || !d_periods || !d_foldbins || !d_snr || !d_ws) return fail(FFA_ERR_ARG, "null pointer");
    if (dtype != FFA_F32 && dtype != FFA_F16 && dtype != FFA_I8) return fail(FFA_ERR_ARG, "bad dtype");
    if (!aligned256(d_ws)) return fail(FFA_ERR_ARG, "workspace must be 256-byte aligned");
    Tiles T;
    ffa_status st = read_tiles(opts, &T);
    if (st != FFA_OK) return st;
    Plan* pl = nullptr;
    st = get_plan(n, tsamp, pmin, pmax, bmin, bmax, h_widths, nw, T, &pl);
    if (st != FFA_OK) return st;
    if (ntrials_cap < pl->ntrials)
        return fail(FFA_ERR_CAPACITY, "ntrials_cap %lld < %lld", (long long)ntrials_cap,
                    (long long)pl->ntrials);
    if (ws_bytes < pl->ws_bytes) return fail(FFA_ERR_CAPACITY, "workspace needs %zu bytes", pl->ws_bytes);
    st = ensure_pinned(*pl);
    if (st != FFA_OK) return st;
    return run_periodogram(*pl, d_x, dtype, d_periods, d_foldbins, d_snr, static_cast<char*>(d_ws),
                           static_cast<cudaStream_t>(stream));
}

ffa_status ffa_periodogram_queue(int64_t n, double tsamp, double pmin, double pmax, int32_t bmin,
                                 int32_t bmax, const int32_t* h_widths, int32_t nw,
                                 const ffa_plan_opts* opts, const void* d_ws, size_t ws_bytes,
                                 int32_t* h_out, int64_t cap, int64_t* nitems, void* stream) {
    if (!d_ws || !nitems || (cap > 0 && !h_out) || cap < 0)
        return fail(FFA_ERR_ARG, "null pointer or bad capacity");
    Tiles T;
    ffa_status st = read_tiles(opts, &T);
    if (st != FFA_OK) return st;
    Plan* pl = nullptr;
    st = get_plan(n, tsamp, pmin, pmax, bmin, bmax, h_widths, nw, T, &pl);
    if (st != FFA_OK) return st;
    if (ws_bytes < pl->ws_bytes) return fail(FFA_ERR_CAPACITY, "workspace needs %zu bytes", pl->ws_bytes);
    *nitems = pl->nitems;
    const int64_t k = std::min<int64_t>(cap, pl->nitems);
    if (k <= 0) return FFA_OK;
    std::vector<ItemHead> heads((size_t)k);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FFA_CUDA(cudaMemcpyAsync(heads.data(), static_cast<const char*>(d_ws) + pl->o_heads,
                             (size_t)k * sizeof(ItemHead), cudaMemcpyDeviceToHost, s),
             "cudaMemcpyAsync(heads)");
    FFA_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    for (int64_t q = 0; q < k; ++q) {
        const ItemHead& h = heads[(size_t)q];
        int32_t* o = h_out + 8 * q;
        o[0] = h.item.tr;
        o[1] = h.item.idx;
        o[2] = h.item.pass;
        o[3] = h.tr.batch;
        o[4] = h.wait;
        o[5] = h.need;
        o[6] = h.rel[0];
        o[7] = h.tr.depth;
    }
    return FFA_OK;
}

ffa_status ffa_periodogram(const void* d_x, ffa_dtype dtype, int64_t n, double tsamp, double pmin,
                           double pmax, int32_t bmin, int32_t bmax, const int32_t* h_widths,
                           int32_t nw, double* d_periods, int32_t* d_foldbins, float* d_snr,
                           int64_t ntrials_cap, void* d_ws, size_t ws_bytes, void* stream) {
    return ffa_periodogram_opts(d_x, dtype, n, tsamp, pmin, pmax, bmin, bmax, h_widths, nw,
                                 nullptr, d_periods, d_foldbins, d_snr, ntrials_cap, d_ws,
                                 ws_bytes, stream);
}

ffa_status ffa_plan_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_batches.clear();
    g_plans.clear();
    return FFA_OK;
}

ffa_status ffa_batch_plan_opts(const ffa_series* h_series, int32_t nseries,
                                const int32_t* h_widths, int32_t nw, size_t ws_budget,
                                const ffa_plan_opts* opts, int64_t* h_trial_offsets,
                                ffa_batch_info* out) {
    if (!out) return fail(FFA_ERR_ARG, "out is null");
    Tiles T;
    ffa_status st = read_tiles(opts, &T);
    if (st != FFA_OK) return st;
    Batch* B = nullptr;
    st = get_batch(h_series, nseries, h_widths, nw, ws_budget, T, &B);
    if (st != FFA_OK) return st;
    std::memset(out, 0, sizeof(*out));
    out->ntrials = B->trial0.back();
    out->nchunks = (int32_t)B->chunks.size();
    out->ntransforms = B->ntransforms;
    out->folded_samples = B->folded;
    out->input_samples = B->input;
    out->workspace_bytes = B->ws_bytes;
    if (h_trial_offsets)
        std::memcpy(h_trial_offsets, B->trial0.data(), B->trial0.size() * sizeof(int64_t));
    return FFA_OK;
}

ffa_status ffa_batch_plan(const ffa_series* h_series, int32_t nseries, const int32_t* h_widths,
                          int32_t nw, size_t ws_budget, int64_t* h_trial_offsets,
                          ffa_batch_info* out) {
    return ffa_batch_plan_opts(h_series, nseries, h_widths, nw, ws_budget, nullptr,
                                h_trial_offsets, out);
}

ffa_status ffa_periodogram_batch_opts(const void* d_x, ffa_dtype dtype,
                                       const ffa_series* h_series, int32_t nseries,
                                       const int32_t* h_widths, int32_t nw, size_t ws_budget,
                                       const ffa_plan_opts* opts, double* d_periods,
                                       int32_t* d_foldbins, float* d_snr, int64_t ntrials_cap,
                                       void* d_ws, size_t ws_bytes, void* stream) {
    if (!d_x || !d_periods || !d_foldbins || !d_snr || !d_ws) return fail(FFA_ERR_ARG, "null pointer");
    if (dtype != FFA_F32 && dtype != FFA_F16 && dtype != FFA_I8) return fail(FFA_ERR_ARG, "bad dtype");
    if (!aligned256(d_ws)) return fail(FFA_ERR_ARG, "workspace must be 256-byte aligned");
    Tiles T;
    ffa_status st = read_tiles(opts, &T);
    if (st != FFA_OK) return st;
    Batch* B = nullptr;
    st = get_batch(h_series, nseries, h_widths, nw, ws_budget, T, &B);
    if (st != FFA_OK) return st;
    if (ntrials_cap < B->trial0.back()) return fail(FFA_ERR_CAPACITY, "ntrials_cap too small");
    if (ws_bytes < B->ws_bytes) return fail(FFA_ERR_CAPACITY, "workspace needs %zu bytes", B->ws_bytes);
    const size_t esize = dtype == FFA_F32 ? 4 : (dtype == FFA_F16 ? 2 : 1);
    bool first = true;
    for (const BatchChunk& c : B->chunks) {
        st = ensure_pinned(*c.plan);
        if (st != FFA_OK) return st;
        st = run_periodogram(*c.plan, static_cast<const char*>(d_x) + (size_t)c.x_lo * esize, dtype,
                             d_periods + c.trial0, d_foldbins + c.trial0,
                             d_snr + c.trial0 * c.plan->W.nw, static_cast<char*>(d_ws),
                             static_cast<cudaStream_t>(stream), first);
        first = false;
        if (st != FFA_OK) return st;
    }
    return FFA_OK;
}

ffa_status ffa_periodogram_batch(const void* d_x, ffa_dtype dtype, const ffa_series* h_series,
                                 int32_t nseries, const int32_t* h_widths, int32_t nw,
                                 size_t ws_budget, double* d_periods, int32_t* d_foldbins,
                                 float* d_snr, int64_t ntrials_cap, void* d_ws, size_t ws_bytes,
                                 void* stream) {
    return ffa_periodogram_batch_opts(d_x, dtype, h_series, nseries, h_widths, nw, ws_budget,
                                       nullptr, d_periods, d_foldbins, d_snr, ntrials_cap, d_ws,
                                       ws_bytes, stream);
}

ffa_status ffa_periodogram_host(const float* h_x, int64_t n, double tsamp, double pmin,
                                double pmax, int32_t bmin, int32_t bmax, const int32_t* h_widths,
                                int32_t nw, double* h_periods, int32_t* h_foldbins, float* h_snr,
                                int64_t ntrials_cap, void* d_ws, size_t ws_bytes, void* stream) {
    if (!h_x || !h_periods || !h_foldbins || !h_snr || !d_ws) return fail(FFA_ERR_ARG, "null pointer");
    if (!aligned256(d_ws)) return fail(FFA_ERR_ARG, "workspace must be 256-byte aligned");
    Plan* pl = nullptr;
    ffa_status st = get_plan(n, tsamp, pmin, pmax, bmin, bmax, h_widths, nw, Tiles{}, &pl);
    if (st != FFA_OK) return st;
    if (ntrials_cap < pl->ntrials) return fail(FFA_ERR_CAPACITY, "ntrials_cap too small");
    if (ws_bytes < pl->ws_host_bytes)
        return fail(FFA_ERR_CAPACITY, "workspace needs %zu bytes", pl->ws_host_bytes);
    st = ensure_pinned(*pl);
    if (st != FFA_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(d_ws);
    float* x = reinterpret_cast<float*>(ws + pl->o_hx);
    double* per = reinterpret_cast<double*>(ws + pl->o_hper);
    int32_t* fb = reinterpret_cast<int32_t*>(ws + pl->o_hfb);
    float* snr = reinterpret_cast<float*>(ws + pl->o_hsnr);
    FFA_CUDA(cudaMemcpyAsync(x, h_x, (size_t)n * 4, cudaMemcpyHostToDevice, s), "copy in");
    st = run_periodogram(*pl, x, FFA_F32, per, fb, snr, ws, s);
    if (st != FFA_OK) return st;
    const size_t T = (size_t)pl->ntrials;
    FFA_CUDA(cudaMemcpyAsync(h_periods, per, T * 8, cudaMemcpyDeviceToHost, s), "copy periods");
    FFA_CUDA(cudaMemcpyAsync(h_foldbins, fb, T * 4, cudaMemcpyDeviceToHost, s), "copy foldbins");
    FFA_CUDA(cudaMemcpyAsync(h_snr, snr, T * nw * 4, cudaMemcpyDeviceToHost, s), "copy snr");
    FFA_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return FFA_OK;
}

ffa_status ffa_checked_status(int32_t* checked, uint32_t* bits) {
    if (!checked || !bits) return fail(FFA_ERR_ARG, "null pointer");
    *checked = kChecked ? 1 : 0;
    *bits = 0;
    if (kChecked) {
        FFA_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
        unsigned v[3] = {0, 0, 0};
        FFA_CUDA(bounds_seen_kernels(&v[0]), "read status");
        FFA_CUDA(bounds_seen_median(&v[1]), "read status");
        FFA_CUDA(bounds_seen_peaks(&v[2]), "read status");
        *bits = v[0] | v[1] | v[2];
    }
    return FFA_OK;
}

ffa_status ffa_check(void* d_ws, void* stream) {
    if (!d_ws) return fail(FFA_ERR_ARG, "null workspace");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned v = 0;
    FFA_CUDA(cudaMemcpyAsync(&v, d_ws, sizeof(v), cudaMemcpyDeviceToHost, s), "read status");
    FFA_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    FFA_CUDA(cudaMemsetAsync(d_ws, 0, sizeof(v), s), "clear status");
    if (v & kDevTimeout) return fail(FFA_ERR_TIMEOUT, "a device-side wait ran out of time");
    if (v) {
        // bits 4, 8, 16: the peak finder's input checks (ffa_peaks.cu)
        return fail(FFA_ERR_DEVICE, "device status 0x%x%s%s%s%s%s", v,
                    (v & 2u) ? "; a work item out of range" : "",
                    (v & 4u) ? "; peak finding: more segments than max_segments" : "",
                    (v & 8u) ? "; peak finding: a segment above 16384 trials" : "",
                    (v & 16u) ? "; peak finding: periods not positive and non-decreasing" : "",
                    (v & kDevBounds) ? "; an index out of range (checked build)" : "");
    }
    return FFA_OK;
}

}  // extern "C"
