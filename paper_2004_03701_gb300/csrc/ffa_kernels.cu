// ffa_kernels.cu -- sm_103a kernels of the FFA periodogram (Morello et al. 2020).
//
//   prefix_*      double-float exclusive prefix sums of every raw series (restarting at
//                 each series), so that every real-factor downsampling window (Sec.
//                 5.3, App. A.4) costs two lookups instead of re-reading ~f raw samples.
//   downsample    all pseudo-octaves of all series in one launch; window edges i*f in
//                 exact 64.64 fixed point, partial samples weighted by their overlap.
//   item_rec      the record of every queue position (work item, transform, stage count
//                 and, for top passes, row intervals, shared-memory offsets and bulk-copy
//                 bytes), one thread per item.
//   ffa_persistent  one CTA per SM takes work items from a queue until the periodogram
//                 is done.  Sub-tree items (bottom_item): the rows of a node arrive by
//                 one bulk asynchronous copy (cp.async.bulk + mbarrier), nodes of up to
//                 16 rows are transformed in registers, the remaining levels (Eq.
//                 ffa_merge_rule) in shared memory; the sub-tree is written out or, when
//                 it is the whole transform, scored (fused S/N).  Top-pass items
//                 (top_item): up to three levels above the sub-trees for a block of
//                 output rows, gathering only the row intervals the block depends on;
//                 the last pass scores its rows with the boxcar filters (Sec. 5.4), so
//                 final profiles are never stored.
//   ffa_bottom, ffa_top  the same items as plain grids, for a single ffa_transform.
//   boxcar_snr    standalone S/N of stored profiles.
//   normalise_*   whole-series FP64 mean and standard deviation, FP32/FP16/int8 output.
//
// Every floating-point add of the FFA is the same single float add of H_i[x] and
// T_j[(x + i + b) mod p] that the recursion performs, so transforms are bit-exact.
#include "ffa_internal.h"

#include <cuda_fp16.h>

namespace ffa {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------------
// Small integer helpers shared by the merge kernels.
// ---------------------------------------------------------------------------------

// ceil(log2(n)): the number of merge levels above an n-row block (0 for n = 1).
__device__ __forceinline__ int tree_height(int n) { return n <= 1 ? 0 : 32 - __clz(n - 1); }

// ---------------------------------------------------------------------------------
// Double-float ("float2" = hi + lo) arithmetic: Knuth's two-sum, ~48-bit significand.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s = __fadd_rn(a.x, b.x);
    float bb = __fsub_rn(s, a.x);
    float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    float h = __fadd_rn(s, e);
    float l = __fsub_rn(e, __fsub_rn(h, s));
    return make_float2(h, l);
}
// (a - b) rounded once to float.
__device__ __forceinline__ float df_sub_to_float(float2 a, float2 b) {
    float s = __fsub_rn(a.x, b.x);
    float bb = __fsub_rn(s, a.x);
    float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(-b.x, bb));
    e = __fadd_rn(e, __fsub_rn(a.y, b.y));
    return __fadd_rn(s, e);
}

__device__ __forceinline__ float load_sample(const void* x, int dtype, int64_t i) {
    if (dtype == 0) return static_cast<const float*>(x)[i];
    if (dtype == 1) return __half2float(static_cast<const __half*>(x)[i]);
    return (float)static_cast<const signed char*>(x)[i] * 0.0625f;
}

// ---------------------------------------------------------------------------------
// Prefix sums.  Chunk of 4096 samples per CTA: 256 threads x 16 consecutive samples.
// ---------------------------------------------------------------------------------
constexpr int kPrefixThreads = 256;
constexpr int kPrefixPerThread = 16;
constexpr int kPrefixChunk = kPrefixThreads * kPrefixPerThread;

__device__ __forceinline__ PrefixSeg prefix_seg(const PrefixParams& P, int64_t chunk) {
    if (!P.segs) return P.single;
    return P.segs[P.blk_seg ? P.blk_seg[chunk] : 0];
}

// Loads the chunk [base, base + 4096) of a series ending at `end` into shared memory
// (coalesced), returns this thread's 16 consecutive samples.
__device__ __forceinline__ void prefix_load(const PrefixParams& P, int64_t base, int64_t end,
                                            float* sh, float v[kPrefixPerThread]) {
    for (int q = 0; q < kPrefixPerThread; ++q) {
        int e = q * kPrefixThreads + threadIdx.x;
        int64_t g = base + e;
        float val = g < end ? load_sample(P.x, P.dtype, g) : 0.f;
        sh[(e >> 4) * 17 + (e & 15)] = val;  // padded: conflict-free column reads
    }
    __syncthreads();
    for (int q = 0; q < kPrefixPerThread; ++q) v[q] = sh[threadIdx.x * 17 + q];
}

// Block-wide inclusive scan of one double-float per thread; returns the exclusive
// prefix of this thread, and the block total in *total.
__device__ __forceinline__ float2 block_exclusive_df(float2 a, float2* warp_tot, float2* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 inc = a;
    for (int o = 1; o < 32; o <<= 1) {
        float2 v;
        v.x = __shfl_up_sync(kFull, inc.x, o);
        v.y = __shfl_up_sync(kFull, inc.y, o);
        if (lane >= o) inc = df_add(v, inc);
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    float2 wofs = make_float2(0.f, 0.f), tot = make_float2(0.f, 0.f);
    for (int w = 0; w < kPrefixThreads / 32; ++w) {
        if (w < warp) wofs = df_add(wofs, warp_tot[w]);
        tot = df_add(tot, warp_tot[w]);
    }
    float2 ex;
    ex.x = __shfl_up_sync(kFull, inc.x, 1);
    ex.y = __shfl_up_sync(kFull, inc.y, 1);
    if (lane == 0) ex = make_float2(0.f, 0.f);
    *total = tot;
    return df_add(wofs, ex);
}

__global__ void __launch_bounds__(kPrefixThreads) prefix_partial_kernel(PrefixParams P) {
    __shared__ float sh[kPrefixThreads * 17];
    __shared__ float2 wt[kPrefixThreads / 32];
    const PrefixSeg sg = prefix_seg(P, blockIdx.x);
    if (kChecked && !(in_range(sg.x_off, sg.n, P.x_cap, threadIdx.x ? nullptr : P.status) &&
                      in_range(blockIdx.x, 1, P.nchunks, threadIdx.x ? nullptr : P.status)))
        return;  // uniform
    float v[kPrefixPerThread];
    prefix_load(P, sg.x_off + ((int64_t)blockIdx.x - sg.blk0) * kPrefixChunk, sg.x_off + sg.n, sh,
                v);
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < kPrefixPerThread; ++q) acc = df_add(acc, make_float2(v[q], 0.f));
    float2 tot;
    block_exclusive_df(acc, wt, &tot);
    if (threadIdx.x == 0) P.partial[blockIdx.x] = tot;
}

// One CTA per series: exclusive scan of the series' chunk sums, in place; each thread
// takes kTopPerThread consecutive chunks per round.
constexpr int kTopPerThread = 4;
__global__ void __launch_bounds__(kPrefixThreads) prefix_top_kernel(PrefixParams P) {
    __shared__ float2 wt[kPrefixThreads / 32];
    const PrefixSeg sg = P.segs ? P.segs[blockIdx.x] : P.single;
    const int64_t nb = (sg.n + kPrefixChunk - 1) / kPrefixChunk;
    if (kChecked && !in_range(sg.blk0, nb, P.nchunks, threadIdx.x ? nullptr : P.status)) return;
    float2* part = P.partial + sg.blk0;
    float2 carry = make_float2(0.f, 0.f);
    for (int64_t b0 = 0; b0 < nb; b0 += kPrefixThreads * kTopPerThread) {
        const int64_t i0 = b0 + (int64_t)threadIdx.x * kTopPerThread;
        float2 v[kTopPerThread];
        float2 loc = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < kTopPerThread; ++q) {
            v[q] = i0 + q < nb ? part[i0 + q] : make_float2(0.f, 0.f);
            loc = df_add(loc, v[q]);
        }
        float2 tot;
        float2 run = df_add(carry, block_exclusive_df(loc, wt, &tot));
#pragma unroll
        for (int q = 0; q < kTopPerThread; ++q) {
            if (i0 + q < nb) part[i0 + q] = run;
            run = df_add(run, v[q]);
        }
        carry = df_add(carry, tot);
        __syncthreads();  // wt is reused by the next round
    }
}

__global__ void __launch_bounds__(kPrefixThreads) prefix_final_kernel(PrefixParams P) {
    // the input transpose (first 17 x 256 floats), then the output staging: thread t's 16
    // prefixes at 17 t .. 17 t + 15 (padded: a half-warp's 8-byte stores hit 16 bank pairs)
    __shared__ float2 st2[kPrefixChunk + kPrefixChunk / 16];
    float* sh = reinterpret_cast<float*>(st2);
    __shared__ float2 wt[kPrefixThreads / 32];
    const PrefixSeg sg = prefix_seg(P, blockIdx.x);
    const int64_t local0 = ((int64_t)blockIdx.x - sg.blk0) * kPrefixChunk;  // in the series
    if (kChecked && !(in_range(sg.x_off, sg.n, P.x_cap, threadIdx.x ? nullptr : P.status) &&
                      in_range(sg.pre_off, sg.n + 1, P.prefix_cap, threadIdx.x ? nullptr : P.status) &&
                      in_range(blockIdx.x, 1, P.nchunks, threadIdx.x ? nullptr : P.status)))
        return;  // uniform
    float v[kPrefixPerThread];
    prefix_load(P, sg.x_off + local0, sg.x_off + sg.n, sh, v);
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < kPrefixPerThread; ++q) acc = df_add(acc, make_float2(v[q], 0.f));
    float2 tot;
    float2 run = df_add(P.partial[blockIdx.x], block_exclusive_df(acc, wt, &tot));
    float2* pre = P.prefix + sg.pre_off;
    if (local0 == 0 && threadIdx.x == 0) pre[0] = make_float2(0.f, 0.f);
    // the block's results (the prefix after each sample) staged in shared memory, then
    // stored as whole lines (each thread's 16 consecutive values would be 16 strided
    // stores); st2 was last read before the scan's barriers
    for (int q = 0; q < kPrefixPerThread; ++q) {
        run = df_add(run, make_float2(v[q], 0.f));
        st2[17 * threadIdx.x + q] = run;
    }
    __syncthreads();
    for (int q = 0; q < kPrefixPerThread; ++q) {
        const int e = q * kPrefixThreads + threadIdx.x;
        if (local0 + e < sg.n) pre[local0 + e + 1] = st2[e + (e >> 4)];
    }
}

// ---------------------------------------------------------------------------------
// Downsampling (Sec. 5.3, App. A.4).  Window [A, B) = [i f, (i+1) f):
//   out = (S[floor B] - S[floor A]) - frac(A) x[floor A] + frac(B) x[floor B],
// S the exclusive prefix sum (double-float), x[j] taken as S[j+1] - S[j] rounded to
// float (the sample itself up to the prefix's ~48-bit precision).  A and B are exact in
// 64.64 fixed point.
// ---------------------------------------------------------------------------------
// Each CTA covers up to kDownsamplePerBlock consecutive outputs of one octave (the plan
// assigns CTAs to octaves), four per thread at a stride of the CTA size.
__global__ void __launch_bounds__(kDownsampleThreads) downsample_kernel(DownsampleParams P) {
    const int2 bi = P.blocks ? P.blocks[blockIdx.x]
                             : make_int2(0, (int)blockIdx.x * kDownsamplePerBlock);
    const OctaveDesc od = P.oct ? P.oct[bi.x] : P.single;
    if (kChecked) {  // the octave's ranges (uniform)
        unsigned* st = threadIdx.x ? nullptr : P.status;
        if (!(in_range(od.x_off, od.x_n, P.x_cap, st) && in_range(od.out_off, od.nk, P.out_cap, st) &&
              (od.f_int == 1 && od.f_frac == 0 ? od.nk <= od.x_n
                                               : in_range(od.pre_off, od.x_n + 1, P.prefix_cap, st))))
            return;
    }
#pragma unroll
    for (int q = 0; q < kDownsamplePerBlock / kDownsampleThreads; ++q) {
        const int64_t i64 = (int64_t)bi.y + q * kDownsampleThreads + threadIdx.x;
        if (i64 >= od.nk) break;
        const uint64_t i = (uint64_t)i64;
        float out;
        // window edges local to the series; prefix and samples indexed from its start
        const int64_t xo = od.x_off;
        if (od.f_int == 1 && od.f_frac == 0) {
            out = load_sample(P.x, P.dtype, xo + (int64_t)i);
        } else {
            const uint64_t a_frac = i * od.f_frac;
            const uint64_t a_int = i * od.f_int + __umul64hi(i, od.f_frac);
            uint64_t b_frac = a_frac + od.f_frac;
            uint64_t b_int = a_int + od.f_int + (b_frac < a_frac ? 1 : 0);
            if (b_int >= (uint64_t)od.x_n) {  // the series ends inside the window
                b_int = (uint64_t)od.x_n;
                b_frac = 0;
            }
            const float2* pre = P.prefix + od.pre_off;
            if (kChecked && !(a_int <= b_int && b_int <= (uint64_t)od.x_n &&
                              (a_frac == 0 || a_int < (uint64_t)od.x_n) &&
                              (b_frac == 0 || b_int < (uint64_t)od.x_n))) {
                bounds_violation(P.status);
                continue;
            }
            out = df_sub_to_float(pre[(int64_t)b_int], pre[(int64_t)a_int]);
            // the edge samples as differences of adjacent prefix sums (x[j] = S[j+1] - S[j]):
            // the next entry shares the cache sector of S[j] three times in four, where a
            // load of x[j] would be a sector of its own (outputs f samples apart)
            if (a_frac != 0) {
                float al = __ull2float_rn(a_frac) * 5.42101086242752217e-20f;  // 2^-64
                const float xa = df_sub_to_float(pre[(int64_t)a_int + 1], pre[(int64_t)a_int]);
                out = __fsub_rn(out, __fmul_rn(al, xa));
            }
            if (b_frac != 0) {
                float be = __ull2float_rn(b_frac) * 5.42101086242752217e-20f;
                const float xb = df_sub_to_float(pre[(int64_t)b_int + 1], pre[(int64_t)b_int]);
                out = __fadd_rn(out, __fmul_rn(be, xb));
            }
        }
        P.out[od.out_off + i64] = out;
    }
}

// ---------------------------------------------------------------------------------
// Bulk asynchronous copy global -> shared with an mbarrier, bounded wait.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Shared -> global bulk copy (16-byte aligned ends, bytes a multiple of 16), tracked by
// the issuing thread's bulk async-group.  The shared data must be visible to the async
// proxy first (fence_proxy_async_smem after the barrier that completed it).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// L2 policy of the scratch ring: keep its lines (they are read a few batches later and
// then overwritten, so written back to memory only if evicted).
__device__ __forceinline__ uint64_t policy_keep() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_keep(float* p, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
                 "r"(smem_addr(src)), "r"(bytes), "l"(policy_keep())
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until the issuing thread's bulk stores have completed (their global writes done),
// then orders them before the thread's later generic-proxy accesses.
__device__ __forceinline__ void bulk_store_wait() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ---------------------------------------------------------------------------------
// What a persistent CTA does for its neighbours in the queue while an item's own bulk
// copies are in flight (thread 0): release the completion of the item before (its
// stores have long drained by then, so the device-scope fence costs little), and fetch
// the record of the item it runs next.  A CTA releases before it waits on anyone, so
// a held completion never blocks another CTA's progress.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void release_count(int* cnt) {
    // the item's bulk stores complete and are ordered before the generic-proxy fence that
    // releases them together with every thread's stores (ordered before it by the item's
    // last barrier, which precedes this release in causality order)
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
    asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(cnt) : "memory");
}
// Global -> shared bulk copy of scratch-ring rows (the ring's L2 policy).
__device__ __forceinline__ void bulk_g2s_keep(void* dst, const void* src, unsigned bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy_keep())
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Spins on the mbarrier for at most `limit` SM clock cycles (by default 2^31, about 1 s);
// false if it ran out.
constexpr long long kWaitCycles = 1LL << 31;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  long long limit = kWaitCycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

struct QueueHook {
    static constexpr bool kInitEachItem = false;  // the copy barrier is made once per CTA
    long long wait = kWaitCycles;   // limit of every wait, SM clock cycles (all threads)
    unsigned cpar = 0;              // parity of the copy barrier's next phase (all threads)
    bool failed = false;            // a copy wait of the item ran out (all threads)
    // thread 0 only:
    int* done = nullptr;            // the completion counters
    int pend[2] = {-1, -1};         // counters of the item before, not yet released
    const ItemHead* next = nullptr; // head of the next item (in shared memory), or null
    uint64_t* next_bar = nullptr;   // its barrier, whose phase `next_par` completes it
    unsigned next_par = 0;
    const int* table_src = nullptr; // the top-pass tables in global memory
    int* table_dst = nullptr;       // the next item's table buffer and barrier
    uint64_t* table_bar = nullptr;
    const ItemHead* head_src = nullptr;  // head of the item after the next, or null
    ItemHead* head_dst = nullptr;
    uint64_t* head_bar = nullptr;
    unsigned issued = 0;            // set: the table copy was issued (bit 0), the head copy (bit 1)
    int ntables = 0;                // top-pass tables (checks)
    bool armed = false;
    bool timed_out = false;
    __device__ __forceinline__ void release() {
        for (int j = 0; j < 2; ++j)
            if (pend[j] >= 0) {
                release_count(done + pend[j]);
                pend[j] = -1;
            }
    }
    __device__ __forceinline__ void run() {
        if (threadIdx.x != 0 || !armed) return;
        armed = false;
        release();
        // (the buffers were last read by earlier items, whose reads had all returned
        // before the barrier that ended them, so the copies may overwrite them)
        if (next) {  // the next item's head (fetched one item ago) says whether it has a table
            if (!mbar_wait_bounded(next_bar, next_par, wait)) {
                timed_out = true;
            } else if (next->item.pass >= 0 &&
                       (!kChecked || (next->item.pad >= 0 && next->item.pad < ntables))) {
                mbar_expect_tx(table_bar, (unsigned)kTopRecBytes);
                bulk_g2s(table_dst, table_src + (int64_t)next->item.pad * kTopRecInts,
                         (unsigned)kTopRecBytes, table_bar);
                issued |= 1u;
            }
        }
        if (head_src) {
            mbar_expect_tx(head_bar, (unsigned)sizeof(ItemHead));
            bulk_g2s(head_dst, head_src, (unsigned)sizeof(ItemHead), head_bar);
            issued |= 2u;
        }
    }
    // the shared memory of the item's bulk stores may be reused (their global completion
    // is awaited when the item's completion is released)
    __device__ __forceinline__ void store_wait() {
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    __device__ __forceinline__ unsigned parity() const { return cpar; }
    __device__ __forceinline__ long long limit() const { return wait; }
    __device__ __forceinline__ void copied() { cpar ^= 1u; }
    __device__ __forceinline__ void fail() { failed = true; }
};
// Stand-alone launches: a copy barrier per item, nothing to do for other items, stores
// complete before the CTA exits.
struct NoHook {
    static constexpr bool kInitEachItem = true;
    __device__ __forceinline__ void run() {}
    __device__ __forceinline__ void store_wait() { bulk_store_wait(); }
    __device__ __forceinline__ unsigned parity() const { return 0u; }
    __device__ __forceinline__ long long limit() const { return kWaitCycles; }
    __device__ __forceinline__ void copied() {}
    __device__ __forceinline__ void fail() {}
};

// ---------------------------------------------------------------------------------
// ---------------------------------------------------------------------------------
// Boxcar S/N (Sec. 5.4).  For a profile F of p bins, S is the exclusive prefix sum of F
// over two concatenated repeats; for each width w the score is the largest
// C_k = S[k + w] - S[k] over phases k, times inv_std / sqrt(w).
//
// Half-warp form (p <= kSnrHalfMaxP): a warp scores two profiles, one per half.  Lane h
// of a half owns the Q consecutive phases Q h .. Q h + Q - 1: it forms their F (a merge
// F = A[x] + B[(x + k) mod p] of two shared-memory rows, or a stored row A), sums them
// in registers, and after a 16-lane scan of the lane totals holds S[k] of its phases in
// registers (+inf past p, so that those phases never win) and writes them to the
// half's row in shared memory; the row is extended by the second repeat, and each
// width reads S[k + w] once per phase.  A 16-lane transposed butterfly reduces 16
// widths at a time with 15 shuffles.  `write` false: the half only takes part in the
// shuffles (an odd row count) and stores nothing.
// ---------------------------------------------------------------------------------
// Score of width index iw from the largest boxcar sum cmax of a p-bin profile whose
// bins sum to `total`: plain boxcar cmax / sqrt(w); zero-mean boxcar (value a on the w
// bins, b on the others, zero sum, unit square sum) (a - b) cmax + b total, with
// a - b = sqrt(p / (w (p - w))) and b = -sqrt(w / (p (p - w))).  Times 1 / noise std.
__device__ __forceinline__ float snr_scale(float cmax, float total, const Widths& W, int iw,
                                           int p, float inv_std) {
    if (!W.boxcar) return cmax * inv_std * W.inv_sqrt_w[iw];
    const float w = (float)W.w[iw], fp = (float)p, rest = (float)(p - W.w[iw]);
    const float amb = sqrtf(fp / (w * rest));
    const float b = -sqrtf(w / (fp * rest));
    return __fmaf_rn(amb, cmax, b * total) * inv_std;
}

// max(a, b, c) in one instruction
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
// two float subtractions (round to nearest) in one instruction
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    float2 r;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

template <int Q>
__device__ __forceinline__ void snr_half(const float* A, const float* B, int k, int p, float* S,
                                         const Widths& W, float inv_std, float* out, bool write,
                                         int h) {
    const int x0 = Q * h;
    float sk[Q];
    float run = 0.f;
    if (B) {
        int y = (x0 + k) % p;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            sk[i] = run;
            if (x0 + i < p) run = __fadd_rn(run, __fadd_rn(A[x0 + i], B[y]));
            y = y + 1 == p ? 0 : y + 1;
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            sk[i] = run;
            if (x0 + i < p) run = __fadd_rn(run, A[x0 + i]);
        }
    }
    float inc = run;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const float u = __shfl_up_sync(kFull, inc, o, 16);
        if (h >= o) inc = __fadd_rn(inc, u);
    }
    float ex = __shfl_up_sync(kFull, inc, 1, 16);
    if (h == 0) ex = 0.f;
    const float total = __shfl_sync(kFull, inc, 15, 16);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (x0 + i < p) {
            sk[i] = __fadd_rn(ex, sk[i]);
            S[x0 + i] = sk[i];
        } else {
            sk[i] = INFINITY;
        }
    }
    __syncwarp();
    for (int j = h; j < W.wmax; j += 16) S[p + j] = __fadd_rn(total, S[j]);  // second repeat
    __syncwarp();
    for (int w0 = 0; w0 < W.nw; w0 += 16) {
        float b[16];
#pragma unroll
        for (int iw = 0; iw < 16; ++iw) {
            b[iw] = -INFINITY;
            if (w0 + iw < W.nw) {
                const float* Sw = S + x0 + W.w[w0 + iw];
                // two phases per step (Q is odd): a paired subtraction and a three-input
                // max (max is exact, so the order of the maxima does not matter)
#pragma unroll
                for (int i = 0; i + 1 < Q; i += 2) {
                    const float2 d = fsub2(make_float2(Sw[i], Sw[i + 1]), make_float2(sk[i], sk[i + 1]));
                    b[iw] = fmax3(b[iw], d.x, d.y);
                }
                b[iw] = fmaxf(b[iw], __fsub_rn(Sw[Q - 1], sk[Q - 1]));
            }
        }
        const bool h8 = h & 8, h4 = h & 4, h2 = h & 2, h1 = h & 1;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float keep = h8 ? b[i + 8] : b[i], send = h8 ? b[i] : b[i + 8];
            b[i] = fmaxf(keep, __shfl_xor_sync(kFull, send, 8, 16));
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float keep = h4 ? b[i + 4] : b[i], send = h4 ? b[i] : b[i + 4];
            b[i] = fmaxf(keep, __shfl_xor_sync(kFull, send, 4, 16));
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float keep = h2 ? b[i + 2] : b[i], send = h2 ? b[i] : b[i + 2];
            b[i] = fmaxf(keep, __shfl_xor_sync(kFull, send, 2, 16));
        }
        {
            const float keep = h1 ? b[1] : b[0], send = h1 ? b[0] : b[1];
            b[0] = fmaxf(keep, __shfl_xor_sync(kFull, send, 1, 16));
        }
        // lane h now holds width w0 + h
        if (write && w0 + h < W.nw) out[w0 + h] = snr_scale(b[0], total, W, w0 + h, p, inv_std);
    }
    __syncwarp();
}

#define FFA_SNR_Q(X) X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) \
    X(25) X(27) X(29) X(31) X(33) X(35)

// Two profiles per warp (p <= kSnrHalfMaxP): this lane's half scores F = A + (B << k)
// (B null: F = A) with its prefix-sum row in `S_warp` (snr_warp_floats of the warp).
__device__ __forceinline__ void snr_pair(const float* A, const float* B, int k, int p,
                                         float* S_warp, const Widths& W, float inv_std,
                                         float* out, bool write, int lane) {
    float* S = S_warp + (lane >> 4) * snr_half_stride(p, W.wmax);
    const int h = lane & 15;
    switch (snr_q(p)) {
#define FFA_CASE(Q) case Q: snr_half<Q>(A, B, k, p, S, W, inv_std, out, write, h); return;
        FFA_SNR_Q(FFA_CASE)
#undef FFA_CASE
        default: return;
    }
}

// Boxcar S/N of one long profile (p > kSnrHalfMaxP) by one warp: sequential per-lane
// chunks of the prefix sums, then strided phases per width.  The prefix sums are
// compensated (double-float two-sum accumulation, the lane totals scanned the same way)
// and rounded to float once each, so a long profile's boxcar sums carry one rounding of
// each prefix sum instead of the error of ~p/32 sequential float adds.
__device__ __noinline__ void snr_row_any(const float* prof, int p, float* S, const Widths& W,
                                         float inv_std, float* out, int lane) {
    const int L = p + W.wmax;
    const int c = (L + 31) >> 5;
    const int i0 = lane * c;
    const int i1 = min(i0 + c, L);
    float2 acc = make_float2(0.f, 0.f);
    for (int i = i0; i < i1; ++i) acc = df_add(acc, make_float2(prof[i < p ? i : i - p], 0.f));
    float2 inc = acc;
    for (int o = 1; o < 32; o <<= 1) {
        float2 u;
        u.x = __shfl_up_sync(kFull, inc.x, o);
        u.y = __shfl_up_sync(kFull, inc.y, o);
        if (lane >= o) inc = df_add(u, inc);
    }
    float2 run;
    run.x = __shfl_up_sync(kFull, inc.x, 1);
    run.y = __shfl_up_sync(kFull, inc.y, 1);
    if (lane == 0) {
        run = make_float2(0.f, 0.f);
        S[0] = 0.f;
    }
    for (int i = i0; i < i1; ++i) {
        run = df_add(run, make_float2(prof[i < p ? i : i - p], 0.f));
        S[i + 1] = __fadd_rn(run.x, run.y);
    }
    __syncwarp();
    for (int iw = 0; iw < W.nw; ++iw) {
        const int w = W.w[iw];
        float best = -INFINITY;
        for (int k = lane; k < p; k += 32) best = fmaxf(best, S[k + w] - S[k]);
        for (int o = 16; o; o >>= 1) best = fmaxf(best, __shfl_xor_sync(kFull, best, o));
        if (lane == 0) out[iw] = snr_scale(best, S[p], W, iw, p, inv_std);
    }
    __syncwarp();
}

__device__ __forceinline__ double trial_period(double tau, int p, int m, int s) {
    // P_s = tau p^2 / (p - s / (m - 1))  (Sec. 2.3), same operation order as the oracle
    return tau * (double)p * (double)p / ((double)p - (double)s / (double)(m - 1));
}

// One merge (Eq. ffa_merge_rule) of shared-memory rows by one warp:
//   sm[o + x] = sm[a + x] + sm[b + (x + k) mod p],   0 <= k < p.
// Offsets are in floats from the shared-memory base; lanes take consecutive columns.
// Columns x0 + lane + 32 t, t < NS: the body is fully unrolled and every load of the
// lane is issued before its first add (a runtime-bounded slot loop runs at two thirds of
// this rate).  A slot past the end of the row neither loads nor stores.
template <int NS>
__device__ __forceinline__ void merge_cols(float* sm, int o, int a, int b, int k, int p, int x0,
                                           int lane) {
    int kb = x0 + k;  // (x0 + k) mod p, for x0, k < p
    if (kb >= p) kb -= p;
    const float* pa = sm + a + x0 + lane;
    const float* pb = sm + b + kb + lane;  // T[(x + k) mod p] = pb[32 t], or pb[32 t - p] once wrapped
    float* po = sm + o + x0 + lane;
    const int wrap = p - kb - lane;        // slot t has wrapped once 32 t >= wrap
    const int lim = p - x0 - lane;         // slot t lies in the row while 32 t < lim
    float hv[NS], tv[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
        if (32 * t < lim) {
            hv[t] = pa[32 * t];
            tv[t] = pb[32 * t - (32 * t >= wrap ? p : 0)];
        } else {
            hv[t] = 0.f;
            tv[t] = 0.f;
        }
    }
#pragma unroll
    for (int t = 0; t < NS; ++t)
        if (32 * t < lim) po[32 * t] = __fadd_rn(hv[t], tv[t]);
}
template <int NS>
__device__ __forceinline__ void copy_cols(float* sm, int o, int a, int p, int x0, int lane) {
    const float* pa = sm + a + x0 + lane;
    float* po = sm + o + x0 + lane;
    const int lim = p - x0 - lane;
    float v[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) v[t] = 32 * t < lim ? pa[32 * t] : 0.f;
#pragma unroll
    for (int t = 0; t < NS; ++t)
        if (32 * t < lim) po[32 * t] = v[t];
}
// A whole row: one unrolled body for rows of up to 512 columns, 256-column pieces beyond.
__device__ __forceinline__ void merge_row(float* sm, int o, int a, int b, int k, int p, int lane) {
    switch ((p + 31) >> 5) {
#define FFA_MR(N) case N: merge_cols<N>(sm, o, a, b, k, p, 0, lane); return;
        FFA_MR(1) FFA_MR(2) FFA_MR(3) FFA_MR(4) FFA_MR(5) FFA_MR(6) FFA_MR(7) FFA_MR(8)
        FFA_MR(9) FFA_MR(10) FFA_MR(11) FFA_MR(12) FFA_MR(13) FFA_MR(14) FFA_MR(15) FFA_MR(16)
#undef FFA_MR
        default:
            for (int x0 = 0; x0 < p; x0 += 256) merge_cols<8>(sm, o, a, b, k, p, x0, lane);
    }
}
__device__ __forceinline__ void copy_row(float* sm, int o, int a, int p, int lane) {
    switch ((p + 31) >> 5) {
#define FFA_CR(N) case N: copy_cols<N>(sm, o, a, p, 0, lane); return;
        FFA_CR(1) FFA_CR(2) FFA_CR(3) FFA_CR(4) FFA_CR(5) FFA_CR(6) FFA_CR(7) FFA_CR(8)
        FFA_CR(9) FFA_CR(10) FFA_CR(11) FFA_CR(12) FFA_CR(13) FFA_CR(14) FFA_CR(15) FFA_CR(16)
#undef FFA_CR
        default:
            for (int x0 = 0; x0 < p; x0 += 256) copy_cols<8>(sm, o, a, p, x0, lane);
    }
}

// Rows [0, total) of `src` (global) into shared memory at sm + dst (a float offset whose
// alignment mod 4 matches src's): one bulk copy of the 16-byte-aligned interior, plain
// loads for up to 3 floats at either end.  bulk_bytes() is what the copy moves; every
// thread can evaluate it, so all agree on whether to wait.
__device__ __forceinline__ int bulk_lead(const float* src) {
    const int h = (int)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);
    return h ? 4 - h : 0;
}
__device__ __forceinline__ unsigned bulk_bytes(const float* src, int total) {
    const int lead = bulk_lead(src);
    return total > lead ? (unsigned)(((total - lead) & ~3) * 4) : 0u;
}
__device__ __forceinline__ void issue_rows_copy(float* sm, int dst, const float* src, int total,
                                                uint64_t* bar, bool keep = false) {
    const int lead = bulk_lead(src);
    const unsigned bytes = bulk_bytes(src, total);
    if (!bytes) return;
    if (keep) bulk_g2s_keep(sm + dst + lead, src + lead, bytes, bar);
    else bulk_g2s(sm + dst + lead, src + lead, bytes, bar);
}
__device__ __forceinline__ void load_row_ends(float* sm, int dst, const float* src, int total,
                                              int tid, int nthreads) {
    const int lead = bulk_lead(src);
    const int body = (int)(bulk_bytes(src, total) / 4);
    const int tail0 = lead + body;
    const int nends = lead + (total - tail0);
    for (int e = tid; e < nends; e += nthreads) {
        const int q = e < lead ? e : tail0 + (e - lead);
        sm[dst + q] = src[q];
    }
}

// ---------------------------------------------------------------------------------
// Shared-memory FFA of one sub-tree (all of its levels, breadth-first by height).
// ---------------------------------------------------------------------------------

// Descriptor of row r of an n-row sub-tree at merge level `lev`: the row belongs to one
// node of height <= lev whose parent is higher; nodes of height lev merge (Eq.
// ffa_merge_rule), lower ones are carried unchanged.  Packed: x = head row | tail row
// << 16 (tail 0xffff = copy), y = shift.
__device__ __forceinline__ int2 bottom_desc(int n, int lev, int r, int p) {
    int st = 0, sz = n;
    while (tree_height(sz) > lev) {
        const int nh = sz >> 1;
        if (r - st >= nh) { st += nh; sz -= nh; } else { sz = nh; }
    }
    if (tree_height(sz) != lev) return make_int2(r | (0xffff << 16), 0);
    const Split sp = merge_split(sz, r - st);
    return make_int2((st + sp.i) | ((st + (sz >> 1) + sp.j) << 16), sp.shift % p);
}

// ---------------------------------------------------------------------------------
// Register stage: the transform of a node of S <= 16 rows (its whole sub-tree, up to
// four merge levels) on a strip of 64 consecutive columns, two per lane: lane L holds
// strip columns L and L + 32 of every row.  The rotation T[(x + k) mod p] reads strip
// column u + k: for u = L that is lane L + k's first column, or once L + k passes 31,
// lane L + k - 32's second one, so one shuffle (each lane sending the column its
// receiver needs) serves the first column and one the second.  An output column depends
// on input columns x .. x + S - 1 only, so strip columns 0 .. 64 - S are exact and the
// strips advance by 65 - S columns (a single column per lane would keep 33 - S of 32).
// The merge schedule of each S is a compile-time table, so every operand is a fixed
// register.
// ---------------------------------------------------------------------------------
template <int S>
struct RegSched {
    int i[S], j[S], sh[S];
    constexpr RegSched() : i(), j(), sh() {
        constexpr int nh = S / 2, nt = S - S / 2;
        for (int s = 0; s < S; ++s) {
            i[s] = S > 1 ? (2 * (nh - 1) * s + (S - 1)) / (2 * (S - 1)) : 0;
            j[s] = S > 1 ? (2 * (nt - 1) * s + (S - 1)) / (2 * (S - 1)) : 0;
            sh[s] = s - j[s];
        }
    }
};

template <int OFF, int S, int N>
__device__ __forceinline__ void reg_ffa(float (&v0)[N], float (&v1)[N], int lane) {
    if constexpr (S > 1) {
        constexpr int nh = S / 2;
        reg_ffa<OFF, nh, N>(v0, v1, lane);
        reg_ffa<OFF + nh, S - nh, N>(v0, v1, lane);
        constexpr RegSched<S> sc{};
        float o0[S], o1[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int h = OFF + sc.i[s], t = OFF + nh + sc.j[s], k = sc.sh[s];
            if (k == 0) {
                o0[s] = __fadd_rn(v0[h], v0[t]);
                o1[s] = __fadd_rn(v1[h], v1[t]);
            } else {
                const float send = lane >= k ? v0[t] : v1[t];  // for receiver lane - k (mod 32)
                o0[s] = __fadd_rn(v0[h], __shfl_sync(kFull, send, lane + k));
                o1[s] = __fadd_rn(v1[h], __shfl_sync(kFull, v1[t], lane + k));
            }
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            v0[OFF + s] = o0[s];
            v1[OFF + s] = o1[s];
        }
    }
}

// One strip of one node: rows [st, st + S) of `in`, strip columns from c0, into `out`;
// vstep <= 65 - S (the exact columns).
template <int S>
__device__ __forceinline__ void reg_strip(float* sm, int in, int out, int st, int p, int c0,
                                          int vstep, int lane) {
    int x0 = c0 + lane, x1 = c0 + lane + 32;
    if (x0 >= p) x0 %= p;
    if (x1 >= p) x1 %= p;
    float v0[S], v1[S];
#pragma unroll
    for (int r = 0; r < S; ++r) {
        v0[r] = sm[in + (st + r) * p + x0];
        v1[r] = sm[in + (st + r) * p + x1];
    }
    reg_ffa<0, S, S>(v0, v1, lane);
    if (lane < vstep && c0 + lane < p) {
#pragma unroll
        for (int r = 0; r < S; ++r) sm[out + (st + r) * p + x0] = v0[r];
    }
    if (lane + 32 < vstep && c0 + lane + 32 < p) {
#pragma unroll
        for (int r = 0; r < S; ++r) sm[out + (st + r) * p + x1] = v1[r];
    }
}

__device__ __forceinline__ void reg_strip_any(float* sm, int in, int out, int st, int sz, int p,
                                              int c0, int vstep, int lane) {
    switch (sz) {
#define FFA_REG(S) case S: reg_strip<S>(sm, in, out, st, p, c0, vstep, lane); break;
        FFA_REG(1) FFA_REG(2) FFA_REG(3) FFA_REG(4) FFA_REG(5) FFA_REG(6) FFA_REG(7) FFA_REG(8)
        FFA_REG(9) FFA_REG(10) FFA_REG(11) FFA_REG(12) FFA_REG(13) FFA_REG(14) FFA_REG(15)
        FFA_REG(16)
#undef FFA_REG
        default: break;
    }
}


template <bool kSnr, class Hook>
__device__ __forceinline__ void bottom_item(const BottomParams& P, const WorkItem item,
                                            const TransformDesc& tr, float* smem, Hook& hook) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kBottomThreads / 32;
    const BottomLayout lay = bottom_layout(P.nmax, P.elems_max, P.snr_floats);
    int2* desc = reinterpret_cast<int2*>(smem + lay.desc);  // nmax per shared-memory level

    const int p = tr.p;

    // Node `idx` at depth `depth`: descend by the bits of idx (head = 0, tail = 1).
    int start = 0, n = tr.m;
    for (int b = tr.depth - 1; b >= 0; --b) {
        const int nh = n >> 1;
        if ((item.idx >> b) & 1) { start += nh; n -= nh; } else { n = nh; }
    }

    // ---- rows [start, start + n) -> buffer A (row 0 at float offset a0)
    const float* src = P.src + tr.src_off + (int64_t)start * p;
    const int total = n * p;
    const int a0 = lay.buf_a + (int)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);
    int* rnodes = reinterpret_cast<int*>(smem + lay.nodes);
    int& nreg = reinterpret_cast<int*>(smem)[2];           // header: barrier, then 2 ints
    int& regmax = reinterpret_cast<int*>(smem)[3];
    if constexpr (Hook::kInitEachItem) {
        if (tid == 0) {
            mbar_init(bar, 1);
            nreg = 0;
            regmax = 1;
        }
        __syncthreads();
    }
    const unsigned bytes = bulk_bytes(src, total);
    const int H = tree_height(n);
    bool skip = false;  // checked builds: a bad item is skipped (the queue hook still runs)
    if constexpr (kChecked) {  // the item's ranges, alike in every thread
        unsigned* st = tid == 0 ? P.status : nullptr;
        const long long dyn = dyn_smem_floats();
        const int nw = P.widths.nw;
        const long long sw = (long long)P.snr_warps * snr_warp_floats(p, P.widths.wmax);
        bool ok = n >= 1 && n <= P.nmax && total + 4 <= lay.buf_floats &&
                  in_range(tr.src_off + (long long)start * p, total, P.src_cap, st) &&
                  in_range(lay.buf_b, lay.buf_floats, dyn, st) &&
                  in_range(lay.desc, 2LL * (H > kRegLevels ? H - kRegLevels : 0) * P.nmax,
                           lay.nodes, st) &&
                  in_range(lay.nodes, P.nmax, lay.buf_a, st);
        if (kSnr)
            ok = ok && tr.kept <= n && in_range(tr.trial0, tr.kept, P.ntrials, st) &&
                 in_range(lay.buf_a, sw, dyn, st) && in_range(lay.buf_b, sw, dyn, st) && nw >= 1;
        else
            ok = ok && in_range(tr.scratch_off + (long long)start * p, total, P.dst_cap, st);
        skip = !ok;
    }
    // Warp 0 runs the hook (thread 0: release the item before, fetch the next records)
    // while warps 1.. issue the copy and make the item's tables (the persistent loop has
    // reset nreg and regmax before its claim barrier).
    if (warp == 0) {
        hook.run();
    } else if (!skip) {
        const int t = tid - 32, nt = kBottomThreads - 32;
        if (t == 0 && bytes) {
            mbar_expect_tx(bar, bytes);  // the single arrival of this barrier phase
            issue_rows_copy(smem, a0, src, total, bar);
        }
        load_row_ends(smem, a0, src, total, t, nt);
        // nodes of the register stage: height <= kRegLevels, parent higher (one per start row)
        for (int r = t; r < n; r += nt) {
            int st = 0, sz = n;
            while (tree_height(sz) > kRegLevels) {
                const int nh = sz >> 1;
                if (r - st >= nh) { st += nh; sz -= nh; } else { sz = nh; }
            }
            if (r == st) {
                const int q = atomicAdd(&nreg, 1);
                if (in_range(q, 1, P.nmax, P.status)) rnodes[q] = st | (sz << 16);
                atomicMax(&regmax, sz);
            }
        }
        // row descriptors of every shared-memory level, made while the rows are in flight
        const int nlev = H - kRegLevels;
        for (int e = t; e < nlev * n; e += nt) {
            const int l = e / n, r = e - l * n;
            desc[l * P.nmax + r] = bottom_desc(n, kRegLevels + 1 + l, r, p);
        }
    }
    const bool landed = skip || bytes == 0 || mbar_wait_bounded(bar, hook.parity(), hook.limit());
    if (__syncthreads_or(!landed)) {
        if (tid == 0) {
            atomicOr(P.status, kDevTimeout);
            mbar_wait_bounded(bar, hook.parity(), hook.limit());  // a late copy lands before the CTA exits
        }
        hook.fail();
        return;
    }
    if (skip) {
        if (Hook::kInitEachItem && tid == 0) mbar_inval(bar);
        return;
    }
    if (bytes) hook.copied();

    // ---- register stage: complete transforms of the nodes of <= 16 rows, A -> B
    // Rows after the register stage sit at the 16-byte phase of their destination in
    // global memory (hd floats past a 16-byte boundary), so that the finished sub-tree
    // leaves by one bulk copy.  The buffers have 4 floats of slack for it.
    float* const dst_g = kSnr ? nullptr
                              : ((top_passes(tr.depth, tr.chunk) & 1) ? P.dst_odd : P.dst) +
                                    tr.scratch_off + (int64_t)start * p;
    const int hd = kSnr ? 0 : (int)((reinterpret_cast<uintptr_t>(dst_g) >> 2) & 3);
    int in = lay.buf_b + hd, out = lay.buf_a + hd;
    {
        const int vstep = 65 - regmax;
        const int nstrip = (p + vstep - 1) / vstep;
        const int nwork = nreg * nstrip;
        for (int w = warp; w < nwork; w += nwarps) {
            const int q = w / nstrip, c = w - q * nstrip;
            const int nd = rnodes[q];
            if (kChecked && !((nd >> 16) >= 1 && (nd >> 16) <= 16 &&
                              in_range(nd & 0xffff, nd >> 16, n, lane == 0 ? P.status : nullptr)))
                continue;
            reg_strip_any(smem, a0, in, nd & 0xffff, nd >> 16, p, c * vstep, vstep, lane);
        }
        __syncthreads();
    }

    // ---- merge levels kRegLevels+1 .. H in shared memory
    for (int lev = kRegLevels + 1; lev <= H; ++lev) {
        const int2* dc = desc + (lev - kRegLevels - 1) * P.nmax;
        for (int r = warp; r < n; r += nwarps) {
            const int2 d = dc[r];
            const int ha = d.x & 0xffff, tb = (d.x >> 16) & 0xffff;
            if (kChecked && !(in_range(ha, 1, n, lane == 0 ? P.status : nullptr) &&
                              (tb == 0xffff || in_range(tb, 1, n, lane == 0 ? P.status : nullptr)) &&
                              d.y >= 0 && d.y < p))
                continue;
            if (tb != 0xffff) merge_row(smem, out + r * p, in + ha * p, in + tb * p, d.y, p, lane);
            else copy_row(smem, out + r * p, in + r * p, p, lane);
        }
        __syncthreads();
        const int t = in;
        in = out;
        out = t;
    }

    if constexpr (!kSnr) {
        // the 16-byte-aligned interior by one bulk copy, up to 3 floats at either end by
        // plain stores; the copy has read the buffer before the item ends (it is reused)
        const int lead = bulk_lead(dst_g);
        const unsigned bytes = bulk_bytes(dst_g, total);
        if (tid == 0 && bytes) {
            fence_proxy_async_smem();
            bulk_s2g(dst_g + lead, smem + in + lead, bytes);
        }
        const int tail0 = lead + (int)(bytes / 4);
        for (int e = tid; e < lead + (total - tail0); e += kBottomThreads) {
            const int q = e < lead ? e : tail0 + (e - lead);
            dst_g[q] = smem[in + q];
        }
        if (tid == 0 && bytes) hook.store_wait();
    } else {
        // The sub-tree is the whole transform: score rows s < kept (Sec. 2.3).
        float* S = smem + out + warp * snr_warp_floats(p, P.widths.wmax);
        const int nw = P.widths.nw;
        if (p <= kSnrHalfMaxP) {
            for (int s0 = 2 * warp; warp < P.snr_warps && s0 < tr.kept; s0 += 2 * P.snr_warps) {
                const int s = min(s0 + (lane >> 4), (int)tr.kept - 1);
                snr_pair(smem + in + s * p, nullptr, 0, p, S, P.widths, tr.inv_std,
                         P.snr + (tr.trial0 + s) * nw, s0 + (lane >> 4) < tr.kept, lane);
            }
        } else {
            for (int s = warp; warp < P.snr_warps && s < tr.kept; s += P.snr_warps)
                snr_row_any(smem + in + s * p, p, S, P.widths, tr.inv_std,
                            P.snr + (tr.trial0 + s) * nw, lane);
        }
        for (int s = tid; s < tr.kept; s += kBottomThreads) {
            P.periods[tr.trial0 + s] = trial_period(tr.tau, p, tr.m, s);
            P.foldbins[tr.trial0 + s] = p;
        }
    }
    __syncthreads();
    if (Hook::kInitEachItem && tid == 0) mbar_inval(bar);
}

template <bool kSnr>
__global__ void __launch_bounds__(kBottomThreads, kBottomMinBlocks) ffa_bottom_kernel(BottomParams P) {
    extern __shared__ __align__(16) float smem[];
    const WorkItem item = P.items ? P.items[blockIdx.x] : WorkItem{0, (int)blockIdx.x, 0, 0, 0};
    const TransformDesc tr = P.trs ? P.trs[item.tr] : P.single;
    NoHook hook;
    bottom_item<kSnr>(P, item, tr, smem, hook);
}

// ---------------------------------------------------------------------------------
// Top of the tree: up to three merge levels per pass, gathered.  A CTA computes rows
// [lo, hi] of one node at depth d_out from the complete transforms of its descendants
// at depth d_in = d_out + L.  Because the merge indices i(s), j(s) grow with s, the rows
// needed from each descendant form one interval; only those are loaded (one bulk copy
// per interval) and merged in shared memory.  The last pass of a periodogram scores
// its rows with the boxcar filters instead of storing them.
// ---------------------------------------------------------------------------------
// Fills the record of top-pass item `item` (see kTopRecInts) in one thread.
__device__ void top_record(const TopParams& P, const TransformDesc& tr, const WorkItem item,
                           int* r) {
    const int p = tr.p, m = tr.m;
    const int npass = top_passes(tr.depth, tr.chunk);
    const int pass = item.pass;
    const int d_in = top_pass_in_depth(tr.depth, tr.chunk, pass);
    const int d_out = top_pass_out_depth(tr.depth, tr.chunk, pass);
    const int L = d_in - d_out;
    const int K = item.rows;
    const bool score = pass == npass - 1 && P.snr != nullptr;
    const float* in = ((npass - pass) & 1 ? P.buf1 : P.buf0) + tr.scratch_off;
    const TopLayout lay = top_layout(K, L, p, P.widths.wmax, score);
    // target node (depth d_out) and its row block
    const int nmax = (m + (1 << d_out) - 1) >> d_out;
    const int nb = ((score ? tr.kept : nmax) + K - 1) / K;
    const int node = item.idx / nb, blk = item.idx - node * nb;
    int st0 = 0, n0 = m;
    for (int b = d_out - 1; b >= 0; --b) {
        const int nh = n0 >> 1;
        if ((node >> b) & 1) { st0 += nh; n0 -= nh; } else { n0 = nh; }
    }
    const int lo0 = blk * K;
    const int hi0 = min(lo0 + K, score ? tr.kept : n0) - 1;
    r[0] = st0; r[1] = n0; r[2] = lo0; r[3] = hi0;
    r[kRecBytes] = 0;
    if (lo0 > hi0) return;  // block past the end of a smaller node: nothing to do
    top_intervals(st0, n0, lo0, hi0, L, r);
    // level L: each interval in a 16-byte-aligned region, data at +h so that the bulk
    // copy of its aligned interior lands aligned
    int acc = 0;
    unsigned bytes = 0;
    for (int j = 0; j < (1 << L); ++j) {
        const int e = (1 << L) - 1 + j;
        const float* g = in + (int64_t)(r[8 * e] + r[8 * e + 2]) * p;
        const int total = (r[8 * e + 3] - r[8 * e + 2] + 1) * p;
        const int h = (int)((reinterpret_cast<uintptr_t>(g) >> 2) & 3);
        r[8 * e + 4] = lay.buf_a + acc + h;
        acc += round4(h + total);
        bytes += bulk_bytes(g, total);
    }
    // levels L-1 .. 0: compact, one row after another, alternating buffers
    int nd = 0;
    for (int l = L - 1; l >= 0; --l) {
        const int base = (((L - l) & 1) == 0) ? lay.buf_a : lay.buf_b;
        r[kRecLvl + L - 1 - l] = nd;
        int rows = 0;
        for (int j = 0; j < (1 << l); ++j) {
            const int e = (1 << l) - 1 + j;
            r[8 * e + 4] = base + rows * p;
            rows += r[8 * e + 3] - r[8 * e + 2] + 1;
        }
        nd += rows;
    }
    r[kRecLvl + L] = nd;
    r[kRecBytes] = (int)bytes;
}

// The records of all queue positions, one thread each: the head (work item, transform,
// the counter it waits for and the counters it releases) and, for a top-pass item, its
// interval table and layout (top_record).
constexpr int kPrepThreads = 64;  // small CTAs: the work is one latency-bound chain per item
__global__ void __launch_bounds__(kPrepThreads) item_rec_kernel(RecParams R) {
    const int q = blockIdx.x * kPrepThreads + threadIdx.x;
    if (q >= R.nitems) return;
    const WorkItem item = R.top.items[q];
    const TransformDesc tr = R.top.trs[item.tr];
    ItemHead h;
    h.item = item;
    h.tr = tr;
    h.wait = -1;
    h.need = 0;
    h.rel[0] = -1;
    h.rel[1] = -1;
    const int stage = item.pass < 0 ? 0 : item.pass + 1;
    if (stage > 0) {  // every item of the stage before, in this transform
        h.wait = item.tr * kMaxStages + stage - 1;
        h.need = R.stage_count[h.wait];
        if (item.tr == R.inject_tr && stage == 1) h.need += 1;  // fault injection (tests)
    } else if (item.pass == -1 && tr.batch >= R.ring) {
        // a sub-tree writes its batch's ring slot once the batch that used it before has
        // finished reading it: all of that batch's last-pass items
        h.wait = R.batch_base + tr.batch - R.ring;
        h.need = R.batch_top[tr.batch - R.ring];
    }
    if (item.pass != -2) {
        const int npass = top_passes(tr.depth, tr.chunk);
        if (item.pass < npass - 1) {
            h.rel[0] = item.tr * kMaxStages + stage;  // a later stage of the transform waits
        } else if (tr.batch + R.ring < R.nbatches) {
            // the last pass: the batch's slot is free once all of these are done (the earlier
            // passes of a transform end before its last one starts)
            h.rel[0] = R.batch_base + tr.batch;
        }
    }
    R.heads[q] = h;
    if (item.pass >= 0 && in_range(item.pad, 1, R.ntables, R.status))
        top_record(R.top, tr, item, R.tables + (int64_t)item.pad * kTopRecInts);
}

// Returns whether a later stage of the transform waits for this item (not the last pass).
// `rec`: the item's interval table and layout (top_record), or null to build it here.
template <class Hook>
__device__ __forceinline__ bool top_item(const TopParams& P, const WorkItem item,
                                         const TransformDesc& tr, const int* rec, float* smem,
                                         Hook& hook) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kTopThreads / 32;

    const int p = tr.p, m = tr.m;
    const int npass = top_passes(tr.depth, tr.chunk);
    const int pass = item.pass;
    const int d_in = top_pass_in_depth(tr.depth, tr.chunk, pass);
    const int d_out = top_pass_out_depth(tr.depth, tr.chunk, pass);
    const int L = d_in - d_out;
    const int K = item.rows;
    const bool last = pass == npass - 1;
    const bool score = last && P.snr != nullptr;
    const float* in = ((npass - pass) & 1 ? P.buf1 : P.buf0) + tr.scratch_off;
    float* out = ((npass - pass - 1) & 1 ? P.buf1 : P.buf0) + tr.scratch_off;
    const TopLayout lay = top_layout(K, L, p, P.widths.wmax, score);

    // ---- the item's record: intervals, shared-memory layout, descriptor counts
    const int* tab = rec;
    if (!rec) {
        int* t = reinterpret_cast<int*>(smem + lay.table);
        if (tid == 0) top_record(P, tr, item, t);
        tab = t;
    }
    const int* lvl_desc = tab + kRecLvl;  // first descriptor of each level, levels L-1..0, + end
    if constexpr (Hook::kInitEachItem) {
        if (tid == 0) mbar_init(bar, 1);
        __syncthreads();
    }
    const int st0 = tab[0], lo0 = tab[2], hi0 = tab[3];
    if (lo0 > hi0) {  // uniform: block past the end of a smaller node
        if (Hook::kInitEachItem && tid == 0) mbar_inval(bar);
        return !last;
    }
    bool skip = false;  // checked builds: a bad item is skipped (the queue hook still runs)
    if constexpr (kChecked) {  // the item's table, alike in every thread
        unsigned* st = tid == 0 ? P.status : nullptr;
        const long long dyn = dyn_smem_floats();
        bool ok = L >= 1 && L <= kTopMaxLevels;
        // every node: its rows inside the transform, the needed interval inside the node,
        // its rows in shared memory inside the launch's; the gathered ones in the scratch
        for (int e = 0; ok && e < (2 << L) - 1; ++e) {
            const int* t = tab + 8 * e;
            const int rows = t[3] - t[2] + 1;
            ok = rows >= 1 && in_range(t[0], t[1], m, st) && in_range(t[2], rows, t[1], st) &&
                 in_range(t[4], (long long)rows * p, dyn, st);
            if (ok && e >= (1 << L) - 1)
                ok = in_range(tr.scratch_off + (long long)(t[0] + t[2]) * p, (long long)rows * p,
                              P.buf_cap, st);
        }
        ok = ok && lvl_desc[L] <= lay.desc_cap && in_range(lay.desc, 4LL * lvl_desc[L], dyn, st);
        if (score)
            ok = ok && hi0 < tr.kept && in_range(tr.trial0 + lo0, hi0 - lo0 + 1, P.ntrials, st) &&
                 in_range(lay.sbuf, (long long)nwarps * lay.sbuf_warp, dyn, st);
        else
            ok = ok && in_range(tr.scratch_off + (long long)(st0 + lo0) * p,
                                (long long)(hi0 - lo0 + 1) * p, P.buf_cap, st);
        skip = !ok;
    }

    // ---- gather the needed rows of the depth-d_in transforms: one bulk copy per interval,
    //      all counted by a single arrival on the barrier; the unaligned ends of all
    //      intervals by plain loads, one element per thread.  Warp 0 runs the hook
    //      (thread 0: release the item before, fetch the next records) meanwhile.
    const unsigned bytes = (unsigned)tab[kRecBytes];
    int4* desc = reinterpret_cast<int4*>(smem + lay.desc);
    if (warp == 0) {
        hook.run();
    } else if (!skip) {
        const int t = tid - 32, nt = kTopThreads - 32;
        if (t == 0 && bytes) {
            mbar_expect_tx(bar, bytes);
            for (int j = 0; j < (1 << L); ++j) {
                const int e = (1 << L) - 1 + j;
                const float* g = in + (int64_t)(tab[8 * e] + tab[8 * e + 2]) * p;
                issue_rows_copy(smem, tab[8 * e + 4], g, (tab[8 * e + 3] - tab[8 * e + 2] + 1) * p,
                                bar, true);
            }
        }
        for (int u = t; u < (8 << L); u += nt) {
            const int e = (1 << L) - 1 + (u >> 3), c = u & 7;
            const float* g = in + (int64_t)(tab[8 * e] + tab[8 * e + 2]) * p;
            const int total = (tab[8 * e + 3] - tab[8 * e + 2] + 1) * p;
            const int lead = bulk_lead(g);
            const int tail0 = lead + (int)(bulk_bytes(g, total) / 4);
            if (c < lead + (total - tail0)) {  // at most 3 + 3 ends per interval
                const int q = c < lead ? c : tail0 + (c - lead);
                smem[tab[8 * e + 4] + q] = g[q];
            }
        }
        // ---- row descriptors {out, head row, tail row, shift} for levels L-1 .. 0, made
        //      while the bulk copies are in flight
        const int ndesc = lvl_desc[L];
        for (int q = t; q < ndesc; q += nt) {
            int l = L - 1;
            while (q >= lvl_desc[L - l]) --l;  // level of descriptor q
            int r = q - lvl_desc[L - 1 - l];
            int e = (1 << l) - 1;
            while (r > tab[8 * e + 3] - tab[8 * e + 2]) {
                r -= tab[8 * e + 3] - tab[8 * e + 2] + 1;
                ++e;
            }
            const int s = tab[8 * e + 2] + r;
            const Split sp = merge_split(tab[8 * e + 1], s);
            const int eh = 2 * e + 1, et = 2 * e + 2;
            int4 d;
            d.x = tab[8 * e + 4] + r * p;
            d.y = tab[8 * eh + 4] + (sp.i - tab[8 * eh + 2]) * p;
            d.z = tab[8 * et + 4] + (sp.j - tab[8 * et + 2]) * p;
            d.w = sp.shift % p;
            if (kChecked && !(in_range(sp.i - tab[8 * eh + 2], 1, tab[8 * eh + 3] - tab[8 * eh + 2] + 1,
                                       P.status) &&
                              in_range(sp.j - tab[8 * et + 2], 1, tab[8 * et + 3] - tab[8 * et + 2] + 1,
                                       P.status)))
                d = make_int4(d.x, d.x, d.x, 0);  // inside the item's rows; the status tells
            desc[q] = d;
        }
    }

    const bool landed = skip || bytes == 0 || mbar_wait_bounded(bar, hook.parity(), hook.limit());
    if (__syncthreads_or(!landed)) {
        if (tid == 0) {
            atomicOr(P.status, kDevTimeout);
            mbar_wait_bounded(bar, hook.parity(), hook.limit());
        }
        hook.fail();
        return !last;
    }
    if (skip) {
        if (Hook::kInitEachItem && tid == 0) mbar_inval(bar);
        return !last;
    }
    if (bytes) hook.copied();

    // ---- merge levels L-1 .. 1, and level 0 unless it is scored straight from level 1
    const bool fused = score && p <= kSnrHalfMaxP;
    for (int l = L - 1; l >= (fused ? 1 : 0); --l) {
        const int q1 = lvl_desc[L - l];
        for (int q = lvl_desc[L - 1 - l] + warp; q < q1; q += nwarps) {
            const int4 d = desc[q];
            merge_row(smem, d.x, d.y, d.z, d.w, p, lane);
        }
        __syncthreads();
    }

    // ---- level 0: score (last pass of a periodogram) or store
    const int o0 = tab[4];
    const int rows0 = hi0 - lo0 + 1;
    if (score) {
        float* S = smem + lay.sbuf + warp * lay.sbuf_warp;
        const int nw = P.widths.nw;
        if (fused) {  // two rows per warp, the last merge level formed on the fly
            const int q0 = lvl_desc[L - 1];
            for (int r0 = 2 * warp; r0 < rows0; r0 += 2 * nwarps) {
                const int r = min(r0 + (lane >> 4), rows0 - 1);
                const int4 d = desc[q0 + r];
                snr_pair(smem + d.y, smem + d.z, d.w, p, S, P.widths, tr.inv_std,
                         P.snr + (tr.trial0 + lo0 + r) * nw, r0 + (lane >> 4) < rows0, lane);
            }
        } else {
            for (int r = warp; r < rows0; r += nwarps)
                snr_row_any(smem + o0 + r * p, p, S, P.widths, tr.inv_std,
                            P.snr + (tr.trial0 + lo0 + r) * nw, lane);
        }
        for (int r = tid; r < rows0; r += kTopThreads) {
            P.periods[tr.trial0 + lo0 + r] = trial_period(tr.tau, p, m, lo0 + r);
            P.foldbins[tr.trial0 + lo0 + r] = p;
        }
    } else {
        float* dst = out + (int64_t)(st0 + lo0) * p;
        const uint64_t pol = policy_keep();
        for (int e = tid; e < rows0 * p; e += kTopThreads) st_keep(dst + e, smem[o0 + e], pol);
    }
    __syncthreads();
    if (Hook::kInitEachItem && tid == 0) mbar_inval(bar);
    return !last;
}

__global__ void __launch_bounds__(kTopThreads, kTopMinBlocks) ffa_top_kernel(TopParams P) {
    extern __shared__ __align__(16) float smem[];
    const WorkItem item = P.items ? P.items[blockIdx.x]
                                  : WorkItem{0, (int)blockIdx.x, (int16_t)P.single_pass,
                                             (int16_t)P.single_rows, 0};
    const TransformDesc tr = P.trs ? P.trs[item.tr] : P.single;
    NoHook hook;
    top_item(P, item, tr, nullptr, smem, hook);
}

// ---------------------------------------------------------------------------------
// Persistent FFA kernel of a periodogram: one CTA per SM takes work items from a
// queue (one atomic counter) until the list is exhausted.  Items are sub-trees
// (stage 0) or top passes (stage pass + 1) of the transforms; an item of stage s > 0
// first waits until every item of stage s - 1 of its transform has completed.  The
// queue lists all items of a stage before any item of the next stage of the same
// transform, and a CTA never waits on an item listed after its own, so every wait
// ends: the items it waits on were taken earlier by CTAs that are running (a CTA may
// hold two claimed items ahead of the one it runs; claims are in queue order, so the
// smallest unfinished item is always running).  Completions are released one item
// late, at the next item's copy wait or before any wait of the CTA, so a held
// completion never blocks anyone.  Waits are bounded (about 1 s); on expiry the
// status word gets kDevTimeout and all CTAs stop at their next claim.
// Each item starts from its head (ItemHead), fetched by one bulk copy two items ahead,
// and, for a top pass, its interval table, fetched one item ahead.  Completion: the CTA synchronises, then one thread waits for its bulk
// stores, fences at device scope and adds to the stage counter.  The waiting thread
// acquires the counter, then orders the async (bulk-copy) proxy after it before the
// item's rows are copied in.
// ---------------------------------------------------------------------------------
static_assert(kBottomThreads == kTopThreads, "persistent CTAs run both item kinds");
__global__ void __launch_bounds__(kTopThreads, kTopMinBlocks) ffa_persistent_kernel(PersistentParams P) {
    extern __shared__ __align__(16) float smem[];
    int* slot = reinterpret_cast<int*>(smem + P.smem_floats);    // [0]: the item to run
    uint64_t* hbar = reinterpret_cast<uint64_t*>(slot + 4);      // barriers of the three heads
    uint64_t* tbar = hbar + 3;                                   // ... and of the two tables
    ItemHead* hbuf = reinterpret_cast<ItemHead*>(slot + 16);     // three head buffers
    int* tbuf = reinterpret_cast<int*>(hbuf + 3);                // two table buffers
    const int tid = threadIdx.x;
    const int N = P.nitems;
    // thread 0: queue positions claimed in order (a runs now, then b, then c; d is being
    // claimed), the barrier parities (bits 0-2 heads, 3-4 tables) and the copies in flight;
    // the status word is read one item ahead (a relaxed load whose latency the item's work
    // hides).  All threads: head buffer `ha` and table buffer `ta` of the running item.
    int a = N, b = N, c = N, d = N;
    unsigned stat = 0, par = 0, inflight = 0;
    int ha = 0, ta = 0;
    QueueHook hook;
    hook.wait = P.wait_cycles;
    if (tid == 0) {
        hook.done = P.done;
        hook.ntables = P.ntables;
        for (int j = 0; j < 5; ++j) mbar_init(&hbar[j], 1);
        mbar_init(reinterpret_cast<uint64_t*>(smem), 1);  // the items' copy barrier
        a = atomicAdd(P.queue, 1);
        b = atomicAdd(P.queue, 1);
        c = atomicAdd(P.queue, 1);
        for (int j = 0; j < 2; ++j) {
            const int q = j == 0 ? a : b;
            if (q < N) {
                mbar_expect_tx(&hbar[j], (unsigned)sizeof(ItemHead));
                bulk_g2s(&hbuf[j], P.heads + q, (unsigned)sizeof(ItemHead), &hbar[j]);
                inflight |= 1u << j;
            }
        }
        // the first item's table, once its head has landed
        if (a < N && mbar_wait_bounded(&hbar[0], 0, P.wait_cycles)) {
            par ^= 1u;
            inflight &= ~1u;
            if (hbuf[0].item.pass >= 0 &&
                in_range(hbuf[0].item.pad, 1, P.ntables, P.bottom.status)) {
                mbar_expect_tx(&tbar[0], (unsigned)kTopRecBytes);
                bulk_g2s(tbuf, P.tables + (int64_t)hbuf[0].item.pad * kTopRecInts,
                         (unsigned)kTopRecBytes, &tbar[0]);
                inflight |= 1u << 3;
            }
        } else if (a < N) {
            atomicOr(P.bottom.status, kDevTimeout);
            a = N;
        }
    }
    for (;;) {
        // thread 0 alone waits for the item's table (a top pass) and for the counter it
        // depends on; the barrier then hands both to the CTA.  slot[0] is rewritten only
        // after the barrier at the end of the item, when every thread has read it.
        if (tid == 0) {
            int q = (stat & kDevTimeout) ? N : a;
            if (q < N) {
                const ItemHead& H = hbuf[ha];
                bool ok = true;
                if (kChecked)
                    ok = (H.wait < 0 || in_range(H.wait, 1, P.ncounters, P.bottom.status)) &&
                         (H.rel[0] < 0 || in_range(H.rel[0], 1, P.ncounters, P.bottom.status)) &&
                         (H.rel[1] < 0 || in_range(H.rel[1], 1, P.ncounters, P.bottom.status)) &&
                         (H.item.pass < 0 || in_range(H.item.pad, 1, P.ntables, P.bottom.status));
                if (ok && H.item.pass >= 0) {
                    ok = mbar_wait_bounded(&tbar[ta], (par >> (3 + ta)) & 1u, P.wait_cycles);
                    par ^= 1u << (3 + ta);
                    inflight &= ~(1u << (3 + ta));
                }
                if (ok && H.wait >= 0) {
                    const int* cnt = P.done + H.wait;
                    int seen;
                    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(seen) : "l"(cnt) : "memory");
                    if (seen < H.need) {
                        hook.release();  // before waiting on anyone
                        const long long t0 = clock64();
                        for (;;) {
                            __nanosleep(256);
                            asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(seen) : "l"(cnt) : "memory");
                            if (seen >= H.need) break;
                            if (clock64() - t0 > P.wait_cycles) {
                                ok = false;
                                break;
                            }
                        }
                    }
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                }
                if (!ok) {
                    atomicOr(P.bottom.status, kDevTimeout);
                    q = N;
                }
            }
            slot[0] = q;
            reinterpret_cast<int*>(smem)[2] = 0;  // a sub-tree's register-stage node count
            reinterpret_cast<int*>(smem)[3] = 1;  // and largest node
        }
        __syncthreads();
        const int q = slot[0];
        if (q >= N) break;
        const ItemHead& H = hbuf[ha];
        const WorkItem item = H.item;
        const TransformDesc tr = H.tr;
        if (tid == 0) {
            d = atomicAdd(P.queue, 1);
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(stat) : "l"(P.bottom.status) : "memory");
            // during the item: release the item before, fetch the next item's table and
            // the head of the one after it
            const int hb = ha == 2 ? 0 : ha + 1, hc = hb == 2 ? 0 : hb + 1;
            hook.armed = true;
            hook.issued = 0;
            hook.timed_out = false;
            hook.next = b < N ? &hbuf[hb] : nullptr;
            hook.next_bar = &hbar[hb];
            hook.next_par = (par >> hb) & 1u;
            hook.table_src = P.tables;
            hook.table_dst = tbuf + (ta ^ 1) * kTopRecInts;
            hook.table_bar = &tbar[ta ^ 1];
            hook.head_src = c < N ? P.heads + c : nullptr;
            hook.head_dst = &hbuf[hc];
            hook.head_bar = &hbar[hc];
        }
        if (item.pass == -2) bottom_item<true>(P.bottom_snr, item, tr, smem, hook);
        else if (item.pass == -1) bottom_item<false>(P.bottom, item, tr, smem, hook);
        else top_item(P.top, item, tr, tbuf + ta * kTopRecInts, smem, hook);
        __syncthreads();
        if (hook.failed) break;  // a copy wait ran out (uniform)
        if (tid == 0) {
            hook.run();  // an item that returned before its copy wait
            const int hb = ha == 2 ? 0 : ha + 1, hc = hb == 2 ? 0 : hb + 1;
            if (hook.next && !hook.timed_out) {  // the next item's head was consumed by the hook
                par ^= 1u << hb;
                inflight &= ~(1u << hb);
            }
            if (hook.issued & 1u) inflight |= 1u << (3 + (ta ^ 1));
            if (hook.issued & 2u) inflight |= 1u << hc;
            if (hook.timed_out) {
                atomicOr(P.bottom.status, kDevTimeout);
                stat |= kDevTimeout;
            }
            hook.pend[0] = H.rel[0];
            hook.pend[1] = H.rel[1];
        }
        ha = ha == 2 ? 0 : ha + 1;
        ta ^= 1;
        a = b;
        b = c;
        c = d;
    }
    if (tid == 0) {
        hook.release();
        // copies still in flight land before the CTA exits
        for (int j = 0; j < 5; ++j)
            if ((inflight >> j) & 1u) mbar_wait_bounded(&hbar[j], (par >> j) & 1u, P.wait_cycles);
    }
}

// Standalone boxcar S/N of stored profiles: two rows per warp (one per half-warp), or
// one per warp for long profiles.
__global__ void __launch_bounds__(256) boxcar_snr_kernel(SnrParams P) {
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* S = smem + warp * P.warp_floats;
    const int64_t nwarps = (int64_t)gridDim.x * 8, gw = (int64_t)blockIdx.x * 8 + warp;
    const int nw = P.widths.nw;
    if constexpr (kChecked) {  // the warps' prefix-sum rows and the widths (uniform)
        unsigned* st = threadIdx.x ? nullptr : P.status;
        bool ok = P.widths.wmax <= P.cols &&
                  in_range(snr_warp_floats(P.cols, P.widths.wmax), 0, P.warp_floats, st) &&
                  in_range(0, 8LL * P.warp_floats, dyn_smem_floats(), st);
        for (int i = 0; ok && i < nw; ++i) ok = P.widths.w[i] >= 1 && P.widths.w[i] <= P.widths.wmax;
        if (!ok) {
            if (threadIdx.x == 0) bounds_violation(P.status);
            return;
        }
    }
    if (P.cols <= kSnrHalfMaxP) {
        for (int64_t r0 = 2 * gw; r0 < P.rows; r0 += 2 * nwarps) {
            const int64_t r = min(r0 + (lane >> 4), P.rows - 1);
            snr_pair(P.prof + r * P.cols, nullptr, 0, P.cols, S, P.widths, P.inv_std,
                     P.snr + r * nw, r0 + (lane >> 4) < P.rows, lane);
        }
    } else {
        for (int64_t r = gw; r < P.rows; r += nwarps)
            snr_row_any(P.prof + r * P.cols, P.cols, S, P.widths, P.inv_std, P.snr + r * nw, lane);
    }
}

// ---------------------------------------------------------------------------------
// Normalisation (Sec. 3.1, Sec. 5.2): mean and standard deviation of the whole series
// in FP64 (two passes: sum, then sum of squared deviations), then every sample becomes
// (x - mean) / std, rounded to the storage type: float, half, or int8 q with value q/16
// (q = rint(16 x'), clipped to [-128, 127]).  Reduction order is fixed (grid size and
// block shape constant), so results are deterministic.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double block_sum_f64(double v, double* sh) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;
}

// mode 0: partial sums of x; mode 1: partial sums of (x - mean)^2
__global__ void __launch_bounds__(256) normalise_partial_kernel(NormaliseParams P, int mode) {
    __shared__ double sh[8];
    const double mean = mode ? P.stats[0] : 0.0;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)P.x[i] - mean;
        acc += mode ? d * d : d;
    }
    const double t = block_sum_f64(acc, sh);
    if (threadIdx.x == 0) P.partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) normalise_final_kernel(NormaliseParams P, int mode) {
    __shared__ double sh[8];
    double acc = 0.0;
    for (int b = threadIdx.x; b < P.nblocks; b += blockDim.x) acc += P.partial[b];
    const double t = block_sum_f64(acc, sh);
    if (threadIdx.x == 0) {
        if (mode == 0) P.stats[0] = t / (double)P.n;
        else P.stats[1] = sqrt(t / (double)P.n);
    }
}

__global__ void __launch_bounds__(256) normalise_write_kernel(NormaliseParams P) {
    const double mean = P.stats[0];
    const double sd = P.stats[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = sd > 0.0 ? ((double)P.x[i] - mean) / sd : 0.0;
        if (P.out_dtype == 0) {
            static_cast<float*>(P.out)[i] = (float)v;
        } else if (P.out_dtype == 1) {
            static_cast<__half*>(P.out)[i] = __double2half(v);
        } else {
            double q = rint(16.0 * v);
            q = q < -128.0 ? -128.0 : (q > 127.0 ? 127.0 : q);
            static_cast<signed char*>(P.out)[i] = (signed char)q;
        }
    }
}

// Raises a kernel's dynamic shared memory limit once per device (to the CTA maximum
// minus the kernel's static shared memory).  A failure is left for the launch check.
void allow_max_smem(const void* func, int slot) {
    static unsigned char done[8][64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[slot][dev]) return;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) return;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBytes - (int)fa.sharedSizeBytes) != cudaSuccess)
        return;
    done[slot][dev] = 1;
}

}  // namespace

int prefix_chunk() { return kPrefixChunk; }

// ---------------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------------
cudaError_t launch_prefix(const PrefixParams& P, cudaStream_t s) {
    if (P.nchunks <= 0 || P.nsegs <= 0) return cudaSuccess;
    const double n = (double)P.total;
    const double es = P.dtype == 0 ? 4.0 : (P.dtype == 1 ? 2.0 : 1.0);
    {
        LaunchScope ls(kPrefixPartial, es * n + 8.0 * P.nchunks, s);
        prefix_partial_kernel<<<(unsigned)P.nchunks, kPrefixThreads, 0, s>>>(P);
    }
    {
        LaunchScope ls(kPrefixTop, 16.0 * P.nchunks, s);
        prefix_top_kernel<<<(unsigned)P.nsegs, kPrefixThreads, 0, s>>>(P);
    }
    {
        LaunchScope ls(kPrefixFinal, es * n + 8.0 * (n + P.nsegs) + 8.0 * P.nchunks, s);
        prefix_final_kernel<<<(unsigned)P.nchunks, kPrefixThreads, 0, s>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_downsample(const DownsampleParams& P, cudaStream_t s) {
    if (P.total <= 0 || P.nblocks <= 0) return cudaSuccess;
    // per output: two prefix lookups (8 B each), up to two samples, one store
    LaunchScope ls(kDownsample, 28.0 * (double)P.total, s);
    downsample_kernel<<<(unsigned)P.nblocks, kDownsampleThreads, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_bottom(const BottomParams& P, int nblocks, int smem_bytes, bool snr_mode,
                          cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    if (snr_mode) {
        allow_max_smem((const void*)ffa_bottom_kernel<true>, 0);
        ffa_bottom_kernel<true><<<nblocks, kBottomThreads, smem_bytes, s>>>(P);
    } else {
        allow_max_smem((const void*)ffa_bottom_kernel<false>, 1);
        ffa_bottom_kernel<false><<<nblocks, kBottomThreads, smem_bytes, s>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_top(const TopParams& P, int nblocks, int smem_bytes, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    allow_max_smem((const void*)ffa_top_kernel, 2);
    ffa_top_kernel<<<nblocks, kTopThreads, smem_bytes, s>>>(P);
    return cudaGetLastError();
}

cudaError_t bounds_seen_kernels(unsigned* bits) {
    unsigned v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_bounds_seen, sizeof(v));
    if (e != cudaSuccess) return e;
    *bits = v;
    v = 0;
    return cudaMemcpyToSymbol(g_bounds_seen, &v, sizeof(v));
}

cudaError_t launch_snr(const SnrParams& P, cudaStream_t s) {
    if (P.rows <= 0) return cudaSuccess;
    int64_t blocks = (P.rows + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const int smem = 8 * P.warp_floats * 4;
    allow_max_smem((const void*)boxcar_snr_kernel, 3);
    LaunchScope ls(kBoxcarSnr, 4.0 * (double)P.rows * (P.cols + P.widths.nw), s);
    boxcar_snr_kernel<<<(unsigned)blocks, 256, smem, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_normalise(const NormaliseParams& P, cudaStream_t s) {
    // algorithmic bytes: three reads of x (sum, deviations, write pass) and the output
    const double out_bytes = P.out_dtype == 0 ? 4.0 : (P.out_dtype == 1 ? 2.0 : 1.0);
    {
        LaunchScope ls(kNormalise, 4.0 * P.n, s);
        normalise_partial_kernel<<<P.nblocks, 256, 0, s>>>(P, 0);
    }
    {
        LaunchScope ls(kNormalise, 8.0 * P.nblocks, s);
        normalise_final_kernel<<<1, 256, 0, s>>>(P, 0);
    }
    {
        LaunchScope ls(kNormalise, 4.0 * P.n, s);
        normalise_partial_kernel<<<P.nblocks, 256, 0, s>>>(P, 1);
    }
    {
        LaunchScope ls(kNormalise, 8.0 * P.nblocks, s);
        normalise_final_kernel<<<1, 256, 0, s>>>(P, 1);
    }
    {
        LaunchScope ls(kNormalise, (4.0 + out_bytes) * P.n, s);
        normalise_write_kernel<<<P.nblocks, 256, 0, s>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_item_recs(const RecParams& R, cudaStream_t s) {
    if (R.nitems <= 0) return cudaSuccess;
    LaunchScope ls(kItemRecs, (16.0 + sizeof(TransformDesc) + sizeof(ItemHead)) * R.nitems, s);
    item_rec_kernel<<<(unsigned)((R.nitems + kPrepThreads - 1) / kPrepThreads), kPrepThreads, 0, s>>>(R);
    return cudaGetLastError();
}

cudaError_t launch_persistent(const PersistentParams& P, int smem_bytes, cudaStream_t s) {
    if (P.nitems <= 0) return cudaSuccess;
    allow_max_smem((const void*)ffa_persistent_kernel, 4);
    // as many CTAs as can be resident at once (the queue needs no more)
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ffa_persistent_kernel, kTopThreads,
                                                      smem_bytes) != cudaSuccess ||
        per_sm <= 0)
        per_sm = 1;
    ffa_persistent_kernel<<<sms * per_sm, kTopThreads, smem_bytes, s>>>(P);
    return cudaGetLastError();
}

}  // namespace ffa
