// ffa_median.cu -- running-median de-reddening (paper Sec. 5.2) for sm_103a.
//
// The paper removes the low-frequency noise of a series by subtracting a running median
// before normalising it.  Here med[i] is the median of the w = 2h + 1 samples
// x[i-h .. i+h], the series being extended at both ends by its end samples.
//
// A sliding median has no streaming form: each output is an order statistic of its
// window.  Two structures were weighed for the GPU:
//   - a sorted window kept per CTA and updated by merges (fast for small w, but w = 1 s
//     of 64 us samples is 15625 floats and the double buffer does not fit one SM);
//   - a wavelet matrix over the whole series (Claude, Navarro and Ordonez, "The wavelet
//     matrix", SPIRE 2012 / Inf. Syst. 2015), which answers "k-th smallest of x[l, r)"
//     for any range with one rank lookup per key bit and both ends of the range.
// The second is used: it is exact, independent of w, and both its build and its
// queries are coalesced passes over L2-resident arrays.
//
// Keys.  A float maps to a uint32 whose unsigned order is the float order (negative
// values have all bits flipped, others their sign bit set); the k-th smallest key maps
// back to the k-th smallest sample.  NaNs have no order and must not occur.
//
// Build (one stable partition per key bit, most significant first).  Level L holds
// the keys in an order A_L (A_0 is the series); bit b = 31 - L of A_L[i] is stored as
// a bit vector B_L with a rank directory, and A_{L+1} lists the keys of A_L whose bit b
// is 0, in order, then those whose bit is 1.  Z_L is the number of zeros of level L.
// Each level is one launch over tiles of 4096 keys: every CTA sums the per-tile zero
// counts before its tile (a one-CTA scan launch does it for series of more than 4096
// tiles), writes B_L's words (warp ballots) with their rank directory and A_{L+1}, and
// counts next level's zeros per destination tile (three count buffers rotate).
//
// Query.  For a range [l, r) of A_L and a rank k inside it, the zeros of B_L in the
// range map to [rank0(l), rank0(r)) of A_{L+1} and the ones to Z_L + the same for the
// ones; the k-th smallest lies in the zeros iff k < their count, which fixes bit b of
// its key.  32 levels give the key.  rank0 is one 8-byte load: {zeros before the word,
// the word's bits}.  Each thread follows four windows at once to overlap the loads.
// Windows that reach past an end hold c copies of an end sample besides a clamped
// range; a count of the range's keys below each end key places the copies.  Both kinds
// of output run in one launch.
#include "ffa.h"
#include "ffa_internal.h"
#include "ffa_kinds.h"

#include <cstdint>
#include <cstdio>

namespace ffa {
ffa_status set_error(ffa_status st, const char* msg);
}

namespace {

using ffa::LaunchScope;

constexpr int kLevels = 32;         // key bits
constexpr int kThreads = 256;       // build CTA
constexpr int kRounds = 16;         // keys per build thread
constexpr int kTile = kThreads * kRounds;  // keys per build CTA (128 words of B_L)
constexpr int kScanThreads = 1024;  // the one-CTA scan
constexpr int kFusedPrefixMaxTiles = 4096;  // up to here each scatter CTA sums the counts
constexpr int kQueryThreads = 256;
constexpr int kQueryILP = 4;        // windows per query thread
constexpr int64_t kMaxN = 2147483647;

__device__ __forceinline__ uint32_t float_key(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// zeros of B_L before position i (0 <= i <= n)
__device__ __forceinline__ uint32_t rank0(const uint2* __restrict__ D, uint32_t i) {
    const uint2 e = __ldg(D + (i >> 5));
    return e.x + __popc(~e.y & ((1u << (i & 31)) - 1u));
}

// Checked builds: false (and the status bit set) when `ok` fails.
__device__ __forceinline__ bool ck(bool ok, unsigned* status) {
    if (!ffa::kChecked || ok) return true;
    ffa::bounds_violation(status);
    return false;
}

// Level 0: zero count of the top key bit per tile, the two end keys, and a cleared count
// buffer for level 1.
__global__ void __launch_bounds__(kThreads)
wm_count_kernel(const float* __restrict__ x, int64_t n, uint32_t* __restrict__ tz,
                uint32_t* __restrict__ tz_clear, uint32_t* __restrict__ ends) {
    const int64_t t0 = (int64_t)blockIdx.x * kTile;
    uint32_t z = 0;
#pragma unroll
    for (int j = 0; j < kRounds; ++j) {
        const int64_t idx = t0 + j * kThreads + threadIdx.x;
        if (idx < n) z += (float_key(x[idx]) >> 31) ^ 1u;
    }
    for (int o = 16; o; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    __shared__ uint32_t s[kThreads / 32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = z;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += s[w];
        tz[blockIdx.x] = t;
        tz_clear[blockIdx.x] = 0;
        if (blockIdx.x == 0) {
            ends[0] = float_key(x[0]);
            ends[1] = float_key(x[n - 1]);
        }
    }
}

// One CTA: exclusive prefix of the per-tile zero counts and Z_L, for series with more
// tiles than the scatter CTAs sum themselves.
__global__ void __launch_bounds__(kScanThreads)
wm_scan_kernel(const uint32_t* __restrict__ tz, int ntiles, uint32_t* __restrict__ pre,
               uint32_t* __restrict__ Zl) {
    const int tid = threadIdx.x;
    const int per = (ntiles + kScanThreads - 1) / kScanThreads;
    const int b = tid * per, e = min(b + per, ntiles);
    uint32_t sum = 0;
    for (int i = b; i < e; ++i) sum += tz[i];
    uint32_t inc = sum;
    const int lane = tid & 31, warp = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    __shared__ uint32_t s[kScanThreads / 32];
    if (lane == 31) s[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = s[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        s[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    uint32_t run = inc - sum + (warp ? s[warp - 1] : 0u);
    for (int i = b; i < e; ++i) {
        pre[i] = run;
        run += tz[i];
    }
    if (tid == kScanThreads - 1) *Zl = s[kScanThreads / 32 - 1];
}

// Level L: bit vector and rank directory of A_L, stable partition into A_{L+1}, and the
// zero counts of the next bit per destination tile.  xsrc (level 0) or src holds A_L;
// dst and tz_next are null at the last level.  The zeros before this tile and Z_L come
// from `pre` and `Zl` when a scan ran (large series); otherwise every CTA sums the tile
// counts `tz` itself and CTA 0 stores Z_L.  The count buffer of level L + 2 is cleared
// here (level L + 1 adds into tz_next, and level L - 1 read tz_clear).
__global__ void __launch_bounds__(kThreads, 4)
wm_scatter_kernel(const uint32_t* __restrict__ src, const float* __restrict__ xsrc,
                  uint32_t* __restrict__ dst, int64_t n, int bit, int ntiles,
                  const uint32_t* __restrict__ tz, const uint32_t* __restrict__ pre,
                  uint32_t* __restrict__ Zl, uint2* __restrict__ dir,
                  uint32_t* __restrict__ tz_next, uint32_t* __restrict__ tz_clear,
                  unsigned* status) {
    __shared__ uint32_t s_z[kRounds * (kThreads / 32)];  // zeros per (round, warp)
    __shared__ uint32_t s_base[2 * (kThreads / 32)];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * kTile;
    uint32_t key[kRounds], ones[kRounds], valid[kRounds];
    // all loads first: the ballots below would otherwise wait on each in turn
#pragma unroll
    for (int j = 0; j < kRounds; ++j) {
        const int64_t idx = t0 + j * kThreads + tid;
        key[j] = idx < n ? (xsrc ? float_key(__ldg(xsrc + idx)) : __ldg(src + idx)) : 0u;
    }
    uint32_t before = 0, total = 0;  // zeros of the tiles before this one, and of all
    if (!pre) {
#pragma unroll 4
        for (int i = tid; i < ntiles; i += kThreads) {
            const uint32_t c = __ldg(tz + i);
            total += c;
            before += i < (int)blockIdx.x ? c : 0u;
        }
    }
#pragma unroll
    for (int j = 0; j < kRounds; ++j) {
        const bool v = t0 + j * kThreads + tid < n;
        valid[j] = __ballot_sync(0xffffffffu, v);
        ones[j] = __ballot_sync(0xffffffffu, v && ((key[j] >> bit) & 1u));
        if (lane == 0) s_z[j * (kThreads / 32) + warp] = __popc(valid[j] & ~ones[j]);
    }
    if (!pre) {
        for (int o = 16; o; o >>= 1) {
            before += __shfl_xor_sync(0xffffffffu, before, o);
            total += __shfl_xor_sync(0xffffffffu, total, o);
        }
        if (lane == 0) {
            s_base[warp] = before;
            s_base[kThreads / 32 + warp] = total;
        }
    }
    if (tid == 0 && tz_clear) tz_clear[blockIdx.x] = 0;
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 128 (round, warp) counts, in position order
        uint32_t a[4], sum = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a[q] = s_z[lane * 4 + q];
            sum += a[q];
        }
        uint32_t inc = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            s_z[lane * 4 + q] = run;
            run += a[q];
        }
    }
    __syncthreads();
    uint32_t base0, Z;
    if (pre) {
        base0 = __ldg(pre + blockIdx.x);
        Z = *Zl;
    } else {
        base0 = 0;
        Z = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            base0 += s_base[w];
            Z += s_base[kThreads / 32 + w];
        }
        if (blockIdx.x == 0 && tid == 0) *Zl = Z;
    }
    const uint32_t lt = (1u << lane) - 1u;
    // This tile's zeros land in one run of A_{L+1} starting at base0, its ones in one run
    // starting at Z + t0 - base0; each run (<= 4096 keys) meets at most two destination
    // tiles.  cnt[c] counts the keys whose next bit is 0, c = 2 * side + (second tile).
    const uint32_t tz_first = base0 / kTile, to_first = (Z + (uint32_t)t0 - base0) / kTile;
    uint32_t cnt[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < kRounds; ++j) {
        const uint32_t zw = base0 + s_z[j * (kThreads / 32) + warp];  // zeros before the word
        const int64_t w0 = t0 + j * kThreads + warp * 32;             // the word's first position
        if (lane == 0 && w0 < n) dir[w0 >> 5] = make_uint2(zw, ones[j]);
        if (!dst) continue;
        const bool v = (valid[j] >> lane) & 1u;
        const bool one = (ones[j] >> lane) & 1u;
        uint32_t d = 0;
        if (v) {
            const uint32_t z = zw + __popc(valid[j] & ~ones[j] & lt);  // zeros before me
            d = one ? Z + (uint32_t)(w0 + lane) - z : z;
            if (ck((int64_t)d < n, status)) dst[d] = key[j];
        }
        const bool nz = v && !((key[j] >> (bit - 1)) & 1u);
        const bool second = d / kTile != (one ? to_first : tz_first);
        cnt[0] += __popc(__ballot_sync(0xffffffffu, nz && !one && !second));
        cnt[1] += __popc(__ballot_sync(0xffffffffu, nz && !one && second));
        cnt[2] += __popc(__ballot_sync(0xffffffffu, nz && one && !second));
        cnt[3] += __popc(__ballot_sync(0xffffffffu, nz && one && second));
    }
    if ((n & 31) == 0 && blockIdx.x == gridDim.x - 1 && tid == 0)
        dir[n >> 5] = make_uint2(Z, 0u);  // rank0(n) when n ends a word
    if (!dst) return;
    __shared__ uint32_t s_cnt[4];
    if (tid < 4) s_cnt[tid] = 0;
    __syncthreads();
    if (lane < 4)  // the counts are warp-uniform: lane c adds count c
        atomicAdd(s_cnt + lane, lane == 0 ? cnt[0] : lane == 1 ? cnt[1] : lane == 2 ? cnt[2] : cnt[3]);
    __syncthreads();
    if (tid < 4 && s_cnt[tid]) {
        const uint32_t tile = ((tid >> 1) ? to_first : tz_first) + (tid & 1);
        if (ck(tile < (uint32_t)ntiles, status)) atomicAdd(tz_next + tile, s_cnt[tid]);
    }
}

struct Matrix {
    const uint2* dir;  // level L's directory at dir + L * nwords
    int64_t nwords;
    const uint32_t* Z;
    uint32_t n;        // keys per level (checks)
    unsigned* status;  // (checks)
};

// Checked builds: a range [l, r) of a level inside [0, n); otherwise set to [0, 0)
// with the status bit set.
__device__ __forceinline__ void ck_range(const Matrix& M, uint32_t& l, uint32_t& r) {
    if (!ck(l <= r && r <= M.n, M.status)) l = r = 0;
}

// key of the k-th smallest (from 0) of A_0[l, r)
__device__ __forceinline__ uint32_t wm_select(const Matrix& M, const uint32_t* sZ, uint32_t l,
                                              uint32_t r, uint32_t k) {
    uint32_t key = 0;
#pragma unroll 4
    for (int L = 0; L < kLevels; ++L) {
        const uint2* D = M.dir + L * M.nwords;
        if (ffa::kChecked) ck_range(M, l, r);
        const uint32_t zl = rank0(D, l), zr = rank0(D, r), zeros = zr - zl;
        key <<= 1;
        if (k < zeros) {
            l = zl;
            r = zr;
        } else {
            k -= zeros;
            key |= 1u;
            l = sZ[L] + l - zl;
            r = sZ[L] + r - zr;
        }
    }
    return key;
}

// number of keys of A_0[l, r) below v
__device__ __forceinline__ uint32_t wm_count_less(const Matrix& M, const uint32_t* sZ,
                                                  uint32_t l, uint32_t r, uint32_t v) {
    uint32_t cnt = 0;
    for (int L = 0; L < kLevels; ++L) {
        const uint2* D = M.dir + L * M.nwords;
        if (ffa::kChecked) ck_range(M, l, r);
        const uint32_t zl = rank0(D, l), zr = rank0(D, r);
        if ((v >> (31 - L)) & 1u) {
            cnt += zr - zl;
            l = sZ[L] + l - zl;
            r = sZ[L] + r - zr;
        } else {
            l = zl;
            r = zr;
        }
    }
    return cnt;
}

__device__ __forceinline__ void emit(const float* x, float* med, float* y, int64_t i, float m) {
    if (y) y[i] = x[i] - m;
    if (med) med[i] = m;
}

// Windows inside the series, outputs [e0, e1) with e0 >= h and e1 <= n - h: four per
// thread, their 32 levels interleaved.
__device__ __forceinline__ void median_inner(const float* x, int64_t base, int64_t e1, int64_t h,
                                             const Matrix& M, const uint32_t* sZ, float* med,
                                             float* y) {
    uint32_t l[kQueryILP], r[kQueryILP], k[kQueryILP], key[kQueryILP];
#pragma unroll
    for (int u = 0; u < kQueryILP; ++u) {
        const int64_t i = base + u * kQueryThreads;
        const bool act = i < e1;
        l[u] = act ? (uint32_t)(i - h) : 0u;
        r[u] = act ? (uint32_t)(i + h + 1) : 0u;
        k[u] = (uint32_t)h;
        key[u] = 0;
    }
#pragma unroll 4
    for (int L = 0; L < kLevels; ++L) {
        const uint2* D = M.dir + L * M.nwords;
        const uint32_t zL = sZ[L];
#pragma unroll
        for (int u = 0; u < kQueryILP; ++u) {
            if (ffa::kChecked) ck_range(M, l[u], r[u]);
            const uint32_t zl = rank0(D, l[u]), zr = rank0(D, r[u]), zeros = zr - zl;
            key[u] <<= 1;
            if (k[u] < zeros) {
                l[u] = zl;
                r[u] = zr;
            } else {
                k[u] -= zeros;
                key[u] |= 1u;
                l[u] = zL + l[u] - zl;
                r[u] = zL + r[u] - zr;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < kQueryILP; ++u) {
        const int64_t i = base + u * kQueryThreads;
        if (i < e1 && ck(i >= 0 && i < (int64_t)M.n, M.status)) emit(x, med, y, i, key_float(key[u]));
    }
}

// A window that reaches past an end: the clamped range [max(i - h, 0), min(i + h + 1, n))
// plus c0 copies of x[0] and c1 of x[n-1]; its k-th smallest is placed among the copies
// by counts of the range's keys below each end key.
__device__ __forceinline__ void median_edge(const float* x, int64_t n, int64_t h, int64_t i,
                                            const Matrix& M, const uint32_t* sZ,
                                            const uint32_t* ends, float* med, float* y) {
    const int64_t lo = i - h, hi = i + h + 1;
    const uint32_t l = (uint32_t)(lo < 0 ? 0 : lo), r = (uint32_t)(hi > n ? n : hi);
    uint32_t c0 = (uint32_t)(lo < 0 ? -lo : 0), c1 = (uint32_t)(hi > n ? hi - n : 0);
    uint32_t v0 = ends[0], v1 = ends[1];
    if (v1 < v0) {  // the copies in key order
        const uint32_t tv = v0, tc = c0;
        v0 = v1, c0 = c1, v1 = tv, c1 = tc;
    }
    uint32_t k = (uint32_t)h, key;
    const uint32_t b0 = wm_count_less(M, sZ, l, r, v0);
    if (k < b0) {
        key = wm_select(M, sZ, l, r, k);
    } else if (k < b0 + c0) {
        key = v0;
    } else {
        k -= c0;  // now the k-th of the range plus the c1 copies of v1, k >= b0
        const uint32_t b1 = wm_count_less(M, sZ, l, r, v1);
        if (k < b1)
            key = wm_select(M, sZ, l, r, k);
        else if (k < b1 + c1)
            key = v1;
        else
            key = wm_select(M, sZ, l, r, k - c1);
    }
    if (ck(i >= 0 && i < n, M.status)) emit(x, med, y, i, key_float(key));
}

// One launch for all outputs: the first `edge_blocks` CTAs take the outputs whose window
// reaches past an end, [0, e0) and [e1, n), one per thread (their three traversals run
// beside the inner CTAs); the others take [e0, e1).
__global__ void __launch_bounds__(kQueryThreads)
wm_median_kernel(const float* x, int64_t n, int64_t h, int64_t e0, int64_t e1,
                 int64_t edge_blocks, Matrix M, const uint32_t* ends, float* med, float* y) {
    __shared__ uint32_t sZ[kLevels];
    if (threadIdx.x < kLevels) sZ[threadIdx.x] = M.Z[threadIdx.x];
    __syncthreads();
    if ((int64_t)blockIdx.x < edge_blocks) {
        const int64_t t = (int64_t)blockIdx.x * kQueryThreads + threadIdx.x;
        if (t < e0 + (n - e1)) median_edge(x, n, h, t < e0 ? t : e1 + (t - e0), M, sZ, ends, med, y);
        return;
    }
    const int64_t base =
        e0 + ((int64_t)blockIdx.x - edge_blocks) * (kQueryThreads * kQueryILP) + threadIdx.x;
    median_inner(x, base, e1, h, M, sZ, med, y);
}

struct Workspace {
    unsigned* status;  // device status word (ffa_check)
    uint32_t* keys[2];
    uint2* dir;
    uint32_t* tz[3];
    uint32_t* pre;
    uint32_t* Z;
    uint32_t* ends;
    int64_t nwords;
    int ntiles;
    size_t bytes;
};

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

Workspace layout(int64_t n, char* base) {
    Workspace w{};
    w.ntiles = (int)((n + kTile - 1) / kTile);
    w.nwords = (n >> 5) + 1;
    size_t off = 0;
    auto take = [&](size_t b) {
        char* p = base ? base + off : nullptr;
        off += up256(b);
        return p;
    };
    w.status = reinterpret_cast<unsigned*>(take(4));
    w.keys[0] = reinterpret_cast<uint32_t*>(take(4 * (size_t)n));
    w.keys[1] = reinterpret_cast<uint32_t*>(take(4 * (size_t)n));
    w.dir = reinterpret_cast<uint2*>(take(8 * (size_t)w.nwords * kLevels));
    w.tz[0] = reinterpret_cast<uint32_t*>(take(4 * (size_t)w.ntiles));
    w.tz[1] = reinterpret_cast<uint32_t*>(take(4 * (size_t)w.ntiles));
    w.tz[2] = reinterpret_cast<uint32_t*>(take(4 * (size_t)w.ntiles));
    w.pre = reinterpret_cast<uint32_t*>(take(4 * (size_t)w.ntiles));
    w.Z = reinterpret_cast<uint32_t*>(take(4 * kLevels));
    w.ends = reinterpret_cast<uint32_t*>(take(8));
    w.bytes = off;
    return w;
}

ffa_status cuda_err(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "ffa_running_median: %s: %s", what, cudaGetErrorString(e));
    return ffa::set_error(FFA_ERR_CUDA, buf);
}

}  // namespace

extern "C" ffa_status ffa_running_median_workspace(int64_t n, size_t* bytes) {
    if (!bytes) return ffa::set_error(FFA_ERR_ARG, "ffa_running_median_workspace: bytes is null");
    if (n <= 0 || n > kMaxN)
        return ffa::set_error(FFA_ERR_ARG, "ffa_running_median_workspace: n must be in [1, 2^31 - 1]");
    *bytes = layout(n, nullptr).bytes;
    return FFA_OK;
}

extern "C" ffa_status ffa_running_median(const float* d_x, int64_t n, int64_t width,
                                         float* d_med, float* d_y, void* d_ws, size_t ws_bytes,
                                         void* stream) {
    if (!d_x || !d_ws || (!d_med && !d_y))
        return ffa::set_error(FFA_ERR_ARG, "ffa_running_median: null pointer (x, workspace, or "
                                           "both outputs)");
    if (n <= 0 || n > kMaxN)
        return ffa::set_error(FFA_ERR_ARG, "ffa_running_median: n must be in [1, 2^31 - 1]");
    if (width < 1 || (width & 1) == 0 || width > kMaxN)
        return ffa::set_error(FFA_ERR_ARG, "ffa_running_median: width must be odd, in [1, 2^31 - 1]");
    if (d_med && d_med == d_y)
        return ffa::set_error(FFA_ERR_ARG, "ffa_running_median: med and y must differ");
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return ffa::set_error(FFA_ERR_ARG, "ffa_running_median: workspace must be 256-byte aligned");
    const Workspace W = layout(n, static_cast<char*>(d_ws));
    if (ws_bytes < W.bytes)
        return ffa::set_error(FFA_ERR_CAPACITY, "ffa_running_median: workspace too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t h = width / 2;
    {
        const cudaError_t e = cudaMemsetAsync(W.status, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) return cuda_err(e, "cudaMemsetAsync");
    }
    {
        // 32 levels: per level, reads and writes of the keys and the directory words
        LaunchScope ls(ffa::kMedianBuild, (double)kLevels * (8.0 * n + 8.0 * W.nwords), st);
        wm_count_kernel<<<W.ntiles, kThreads, 0, st>>>(d_x, n, W.tz[0], W.tz[1], W.ends);
        const bool scan = W.ntiles > kFusedPrefixMaxTiles;
        for (int L = 0; L < kLevels; ++L) {
            const bool last = L == kLevels - 1;
            uint32_t* tz = W.tz[L % 3];
            if (scan) wm_scan_kernel<<<1, kScanThreads, 0, st>>>(tz, W.ntiles, W.pre, W.Z + L);
            wm_scatter_kernel<<<W.ntiles, kThreads, 0, st>>>(
                L ? W.keys[(L - 1) & 1] : nullptr, L ? nullptr : d_x,
                last ? nullptr : W.keys[L & 1], n, kLevels - 1 - L, W.ntiles, tz,
                scan ? W.pre : nullptr, W.Z + L, W.dir + (size_t)L * W.nwords,
                last ? nullptr : W.tz[(L + 1) % 3], last ? nullptr : W.tz[(L + 2) % 3], W.status);
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(e, "build launch");
    }
    const Matrix M{W.dir, W.nwords, W.Z, (uint32_t)n, W.status};
    // outputs whose window lies inside the series: [e0, e1) = [h, n - h)
    const int64_t e0 = h < n ? h : n;
    const int64_t e1 = n - h > e0 ? n - h : e0;
    {
        LaunchScope ls(ffa::kMedianQuery, 4.0 * n * ((d_med ? 1 : 0) + (d_y ? 2 : 0)), st);
        const int64_t nedge = e0 + (n - e1);
        const int64_t eb = (nedge + kQueryThreads - 1) / kQueryThreads;
        const int64_t per = (int64_t)kQueryThreads * kQueryILP;
        const int64_t ib = (e1 - e0 + per - 1) / per;
        wm_median_kernel<<<(unsigned)(eb + ib), kQueryThreads, 0, st>>>(d_x, n, h, e0, e1, eb, M,
                                                                      W.ends, d_med, d_y);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(e, "query launch");
    }
    return FFA_OK;
}

cudaError_t ffa::bounds_seen_median(unsigned* bits) {
    unsigned v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, ffa::g_bounds_seen, sizeof(v));
    if (e != cudaSuccess) return e;
    *bits = v;
    v = 0;
    return cudaMemcpyToSymbol(ffa::g_bounds_seen, &v, sizeof(v));
}
