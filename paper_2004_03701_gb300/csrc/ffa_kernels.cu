// ffa_kernels.cu -- sm_103a kernels of the FFA periodogram (Morello et al. 2020).
//
//   prefix_*      double-float exclusive prefix sums of the raw series, so that every
//                 real-factor downsampling window (Sec. 5.3, App. A.4) costs two
//                 lookups instead of re-reading ~f raw samples per output sample.
//   downsample    all pseudo-octaves in one launch; window edges i*f in exact 64.64
//                 fixed point, partial samples weighted by their overlap.
//   ffa_bottom    one CTA per depth-D sub-tree of an FFA transform: the rows arrive by
//                 one bulk asynchronous copy (cp.async.bulk + mbarrier), then every
//                 merge level of the sub-tree (Eq. ffa_merge_rule) runs in shared
//                 memory; either writes the sub-tree's transform or, when the sub-tree
//                 is the whole transform, scores its rows directly (fused S/N).
//   ffa_level     one merge level of the top of the tree, through L2.
//   ffa_final_snr the last merge level fused with the boxcar S/N (Sec. 5.4): the final
//                 folded profiles are built in shared memory and never stored.
//   boxcar_snr    standalone S/N of stored profiles.
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

// nint(a / d), ties up, for a >= 0, d > 0 (Sec. 2.2: i and j of the merge rule).
__device__ __forceinline__ int nint_div(long long a, long long d) {
    long long num = 2 * a + d, den = 2 * d;
    if (num < 4294967296LL) return (int)((unsigned)num / (unsigned)den);
    return (int)(num / den);
}

// Merge rule for output row s of an n-row node: head row i, tail row j, shift i + b.
struct Split {
    int i, j, shift;
};
__device__ __forceinline__ Split merge_split(int n, int s) {
    int nh = n >> 1, nt = n - nh;
    Split r;
    r.i = nint_div((long long)(nh - 1) * s, n - 1);
    r.j = nint_div((long long)(nt - 1) * s, n - 1);
    r.shift = s - r.j;  // i + b = s - j
    return r;
}

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

// Loads a chunk into shared memory (coalesced), returns this thread's 16 samples.
__device__ __forceinline__ void prefix_load(const PrefixParams& P, int64_t base, float* sh,
                                            float v[kPrefixPerThread]) {
    for (int q = 0; q < kPrefixPerThread; ++q) {
        int e = q * kPrefixThreads + threadIdx.x;
        int64_t g = base + e;
        float val = g < P.n ? load_sample(P.x, P.dtype, g) : 0.f;
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
    float v[kPrefixPerThread];
    prefix_load(P, (int64_t)blockIdx.x * kPrefixChunk, sh, v);
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < kPrefixPerThread; ++q) acc = df_add(acc, make_float2(v[q], 0.f));
    float2 tot;
    block_exclusive_df(acc, wt, &tot);
    if (threadIdx.x == 0) P.partial[blockIdx.x] = tot;
}

// One CTA: exclusive scan of the chunk sums, in place.
__global__ void __launch_bounds__(kPrefixThreads) prefix_top_kernel(PrefixParams P) {
    __shared__ float2 wt[kPrefixThreads / 32];
    float2 carry = make_float2(0.f, 0.f);
    for (int64_t b0 = 0; b0 < P.nchunks; b0 += kPrefixThreads) {
        int64_t b = b0 + threadIdx.x;
        float2 a = b < P.nchunks ? P.partial[b] : make_float2(0.f, 0.f);
        float2 tot;
        float2 ex = block_exclusive_df(a, wt, &tot);
        if (b < P.nchunks) P.partial[b] = df_add(carry, ex);
        carry = df_add(carry, tot);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kPrefixThreads) prefix_final_kernel(PrefixParams P) {
    __shared__ float sh[kPrefixThreads * 17];
    __shared__ float2 wt[kPrefixThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kPrefixChunk;
    float v[kPrefixPerThread];
    prefix_load(P, base, sh, v);
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < kPrefixPerThread; ++q) acc = df_add(acc, make_float2(v[q], 0.f));
    float2 tot;
    float2 run = df_add(P.partial[blockIdx.x], block_exclusive_df(acc, wt, &tot));
    if (blockIdx.x == 0 && threadIdx.x == 0) P.prefix[0] = make_float2(0.f, 0.f);
    const int64_t g0 = base + (int64_t)threadIdx.x * kPrefixPerThread;
    for (int q = 0; q < kPrefixPerThread; ++q) {
        run = df_add(run, make_float2(v[q], 0.f));
        if (g0 + q < P.n) P.prefix[g0 + q + 1] = run;
    }
}

// ---------------------------------------------------------------------------------
// Downsampling (Sec. 5.3, App. A.4).  Window [A, B) = [i f, (i+1) f):
//   out = (S[floor B] - S[floor A]) - frac(A) x[floor A] + frac(B) x[floor B],
// S the exclusive prefix sum.  A and B are exact in 64.64 fixed point.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) downsample_kernel(DownsampleParams P) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < P.total; g += stride) {
        int lo = 0, hi = P.oct ? P.noct - 1 : 0;  // last octave with first <= g
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (P.oct[mid].first <= g) lo = mid; else hi = mid - 1;
        }
        const OctaveDesc od = P.oct ? P.oct[lo] : P.single;
        const uint64_t i = (uint64_t)(g - od.first);
        float out;
        if (od.f_int == 1 && od.f_frac == 0) {
            out = load_sample(P.x, P.dtype, (int64_t)i);
        } else {
            const uint64_t a_frac = i * od.f_frac;
            const uint64_t a_int = i * od.f_int + __umul64hi(i, od.f_frac);
            uint64_t b_frac = a_frac + od.f_frac;
            uint64_t b_int = a_int + od.f_int + (b_frac < a_frac ? 1 : 0);
            if (b_int >= (uint64_t)P.n) {  // the series ends inside the window
                b_int = (uint64_t)P.n;
                b_frac = 0;
            }
            out = df_sub_to_float(P.prefix[b_int], P.prefix[a_int]);
            if (a_frac != 0) {
                float al = __ull2float_rn(a_frac) * 5.42101086242752217e-20f;  // 2^-64
                out = __fsub_rn(out, __fmul_rn(al, load_sample(P.x, P.dtype, (int64_t)a_int)));
            }
            if (b_frac != 0) {
                float be = __ull2float_rn(b_frac) * 5.42101086242752217e-20f;
                out = __fadd_rn(out, __fmul_rn(be, load_sample(P.x, P.dtype, (int64_t)b_int)));
            }
        }
        P.out[od.out_off + (int64_t)i] = out;
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
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Spins on the mbarrier for at most ~1 s of SM clock; false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 31)) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------------
// Boxcar S/N of one profile by one warp (Sec. 5.4).  S = exclusive prefix sum over
// two concatenated repeats (length p + wmax + 1, in shared memory), then for each
// width w the largest S[k + w] - S[k], scaled by 1 / (stdnoise sqrt(w)).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void warp_snr(const float* prof, int p, float* S, const Widths& W,
                                         float inv_std, float* out, int lane) {
    const int L = p + W.wmax;
    const int c = (L + 31) >> 5;
    const int i0 = lane * c;
    const int i1 = min(i0 + c, L);
    float acc = 0.f;
    for (int i = i0; i < i1; ++i) acc += prof[i < p ? i : i - p];
    float inc = acc;
    for (int o = 1; o < 32; o <<= 1) {
        float v = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += v;
    }
    float run = __shfl_up_sync(kFull, inc, 1);
    if (lane == 0) {
        run = 0.f;
        S[0] = 0.f;
    }
    for (int i = i0; i < i1; ++i) {
        run += prof[i < p ? i : i - p];
        S[i + 1] = run;
    }
    __syncwarp();
    for (int iw = 0; iw < W.nw; ++iw) {
        const int w = W.w[iw];
        float best = -INFINITY;
        for (int k = lane; k < p; k += 32) best = fmaxf(best, S[k + w] - S[k]);
        for (int o = 16; o; o >>= 1) best = fmaxf(best, __shfl_xor_sync(kFull, best, o));
        if (lane == 0) out[iw] = best * inv_std * W.inv_sqrt_w[iw];
    }
    __syncwarp();
}

__device__ __forceinline__ double trial_period(double tau, int p, int m, int s) {
    // P_s = tau p^2 / (p - s / (m - 1))  (Sec. 2.3), same operation order as the oracle
    return tau * (double)p * (double)p / ((double)p - (double)s / (double)(m - 1));
}

// ---------------------------------------------------------------------------------
// Shared-memory FFA of one sub-tree.
// ---------------------------------------------------------------------------------
template <bool kSnr>
__global__ void __launch_bounds__(kBottomThreads) ffa_bottom_kernel(BottomParams P) {
    extern __shared__ __align__(16) float smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    float* bufA = smem + 4;
    float* bufB = bufA + P.buf_floats;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kBottomThreads / 32;

    const WorkItem item = P.items ? P.items[blockIdx.x] : WorkItem{0, (int)blockIdx.x};
    const TransformDesc tr = P.trs ? P.trs[item.tr] : P.single;
    const int p = tr.p;

    // Node `idx` at depth `depth`: descend by the bits of idx (head = 0, tail = 1).
    int start = 0, n = tr.m;
    for (int b = tr.depth - 1; b >= 0; --b) {
        const int nh = n >> 1;
        if ((item.idx >> b) & 1) { start += nh; n -= nh; } else { n = nh; }
    }

    // ---- load rows [start, start + n): bulk copy of the 16-byte-aligned interior,
    //      plain loads for up to 3 floats at either end.
    const float* src = P.src + tr.src_off + (int64_t)start * p;
    const int64_t total = (int64_t)n * p;
    const int h = (int)((reinterpret_cast<uintptr_t>(src) >> 2) & 3);  // row 0 at bufA + h
    float* in = bufA + h;
    const int lead = h ? 4 - h : 0;                // floats before the aligned interior
    const int64_t body = total > lead ? ((total - lead) & ~(int64_t)3) : 0;
    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();
    if (body > 0 && tid == 0) {
        mbar_expect_tx(bar, (unsigned)(body * 4));
        bulk_g2s(in + lead, src + lead, (unsigned)(body * 4), bar);
    }
    for (int64_t e = tid; e < total; e += kBottomThreads) {
        if (e < lead || e >= lead + body) in[e] = src[e];
    }
    const bool landed = body == 0 || mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!landed)) {
        if (tid == 0) {
            atomicOr(P.status, kDevTimeout);
            mbar_wait_bounded(bar, 0);  // let a late copy land before the CTA exits
        }
        return;
    }

    // ---- merge levels 1..H of the sub-tree, breadth-first by node height.  At level
    //      `lev` every row belongs to one node of height <= lev whose parent is higher:
    //      nodes of height lev merge (Eq. ffa_merge_rule), lower ones are carried.
    float* out = bufB;
    const int H = tree_height(n);
    for (int lev = 1; lev <= H; ++lev) {
        for (int r = warp; r < n; r += nwarps) {
            int st = 0, sz = n;
            while (tree_height(sz) > lev) {
                const int nh = sz >> 1;
                if (r - st >= nh) { st += nh; sz -= nh; } else { sz = nh; }
            }
            float* o = out + (int64_t)r * p;
            if (tree_height(sz) == lev) {
                const Split sp = merge_split(sz, r - st);
                const float* ra = in + (int64_t)(st + sp.i) * p;
                const float* rb = in + (int64_t)(st + (sz >> 1) + sp.j) * p;
                const int k = sp.shift % p;
                for (int x = lane; x < p; x += 32) {
                    int y = x + k;
                    if (y >= p) y -= p;
                    o[x] = __fadd_rn(ra[x], rb[y]);
                }
            } else {
                const float* ra = in + (int64_t)r * p;
                for (int x = lane; x < p; x += 32) o[x] = ra[x];
            }
        }
        __syncthreads();
        float* t = in;
        in = out;
        out = (t == bufA + h) ? bufA : t;
    }

    if constexpr (!kSnr) {
        float* dst = ((tr.depth & 1) ? P.dst_odd : P.dst) + tr.scratch_off + (int64_t)start * p;
        for (int64_t e = tid; e < total; e += kBottomThreads) dst[e] = in[e];
    } else {
        // The sub-tree is the whole transform: score rows s < kept (Sec. 2.3).
        float* S = out + warp * (p + P.widths.wmax + 1);
        for (int s = warp; warp < P.snr_warps && s < tr.kept; s += P.snr_warps) {
            const int64_t t = tr.trial0 + s;
            warp_snr(in + (int64_t)s * p, p, S, P.widths, tr.inv_std, P.snr + t * P.widths.nw,
                     lane);
            if (lane == 0) {
                P.periods[t] = trial_period(tr.tau, p, tr.m, s);
                P.foldbins[t] = p;
            }
        }
    }
    __syncthreads();
    if (tid == 0) mbar_inval(bar);
}

// ---------------------------------------------------------------------------------
// One merge level of the top of the tree: rows of the depth-d nodes from the complete
// transforms of their depth-(d+1) children, through L2.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(kLevelThreads) ffa_level_kernel(LevelParams P) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WorkItem item = P.items ? P.items[blockIdx.x] : WorkItem{0, (int)blockIdx.x};
    const TransformDesc tr = P.trs ? P.trs[item.tr] : P.single;
    const int p = tr.p, m = tr.m;
    const float* in = P.in + tr.scratch_off;
    float* out = P.out + tr.scratch_off;
    const int r1 = min(m, (item.idx + 1) * kLevelRows);
    for (int r = item.idx * kLevelRows + warp; r < r1; r += kLevelThreads / 32) {
        int st = 0, sz = m;
        for (int b = 0; b < P.depth; ++b) {
            const int nh = sz >> 1;
            if (r - st >= nh) { st += nh; sz -= nh; } else { sz = nh; }
        }
        const Split sp = merge_split(sz, r - st);
        const float* ra = in + (int64_t)(st + sp.i) * p;
        const float* rb = in + (int64_t)(st + (sz >> 1) + sp.j) * p;
        const int k = sp.shift % p;
        float* o = out + (int64_t)r * p;
        for (int x = lane; x < p; x += 32) {
            int y = x + k;
            if (y >= p) y -= p;
            o[x] = __fadd_rn(ra[x], rb[y]);
        }
    }
}

// ---------------------------------------------------------------------------------
// Root merge level fused with the boxcar S/N: each warp builds F_s in shared memory
// from the two depth-1 transforms and scores it.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(kFinalThreads) ffa_final_snr_kernel(FinalParams P) {
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WorkItem item = P.items ? P.items[blockIdx.x] : WorkItem{0, (int)blockIdx.x};
    const TransformDesc tr = P.trs ? P.trs[item.tr] : P.single;
    const int p = tr.p, m = tr.m;
    const float* in = P.in + tr.scratch_off;
    float* prof = smem + warp * P.warp_floats;
    float* S = prof + p;
    const int s1 = min(tr.kept, (item.idx + 1) * kFinalRows);
    for (int s = item.idx * kFinalRows + warp; s < s1; s += kFinalThreads / 32) {
        const Split sp = merge_split(m, s);
        const float* ra = in + (int64_t)sp.i * p;
        const float* rb = in + (int64_t)((m >> 1) + sp.j) * p;
        const int k = sp.shift % p;
        for (int x = lane; x < p; x += 32) {
            int y = x + k;
            if (y >= p) y -= p;
            prof[x] = __fadd_rn(ra[x], rb[y]);
        }
        __syncwarp();
        const int64_t t = tr.trial0 + s;
        warp_snr(prof, p, S, P.widths, tr.inv_std, P.snr + t * P.widths.nw, lane);
        if (lane == 0) {
            P.periods[t] = trial_period(tr.tau, p, m, s);
            P.foldbins[t] = p;
        }
    }
}

// Standalone boxcar S/N of stored profiles: one warp per row.
__global__ void __launch_bounds__(256) boxcar_snr_kernel(SnrParams P) {
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* S = smem + warp * P.warp_floats;
    const int64_t stride = (int64_t)gridDim.x * 8;
    for (int64_t r = (int64_t)blockIdx.x * 8 + warp; r < P.rows; r += stride) {
        warp_snr(P.prof + r * P.cols, P.cols, S, P.widths, P.inv_std, P.snr + r * P.widths.nw,
                 lane);
    }
}

// Raises a kernel's dynamic shared memory limit once per device.
void allow_max_smem(const void* func, int slot) {
    static unsigned char done[8][64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[slot][dev]) return;
    cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    done[slot][dev] = 1;
}

}  // namespace

int prefix_chunk() { return kPrefixChunk; }

// ---------------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------------
cudaError_t launch_prefix(const PrefixParams& P, cudaStream_t s) {
    const double n = (double)P.n;
    {
        LaunchScope ls(kPrefixPartial, 4.0 * n + 8.0 * P.nchunks, s);
        prefix_partial_kernel<<<(unsigned)P.nchunks, kPrefixThreads, 0, s>>>(P);
    }
    {
        LaunchScope ls(kPrefixTop, 16.0 * P.nchunks, s);
        prefix_top_kernel<<<1, kPrefixThreads, 0, s>>>(P);
    }
    {
        LaunchScope ls(kPrefixFinal, 4.0 * n + 8.0 * (n + 1) + 8.0 * P.nchunks, s);
        prefix_final_kernel<<<(unsigned)P.nchunks, kPrefixThreads, 0, s>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_downsample(const DownsampleParams& P, cudaStream_t s) {
    if (P.total <= 0) return cudaSuccess;
    int64_t blocks = (P.total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    // per output: two prefix lookups (8 B each), up to two samples, one store
    LaunchScope ls(kDownsample, 28.0 * (double)P.total, s);
    downsample_kernel<<<(unsigned)blocks, 256, 0, s>>>(P);
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

cudaError_t launch_level(const LevelParams& P, int nblocks, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    ffa_level_kernel<<<nblocks, kLevelThreads, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_final(const FinalParams& P, int nblocks, int smem_bytes, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    allow_max_smem((const void*)ffa_final_snr_kernel, 2);
    ffa_final_snr_kernel<<<nblocks, kFinalThreads, smem_bytes, s>>>(P);
    return cudaGetLastError();
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

}  // namespace ffa
