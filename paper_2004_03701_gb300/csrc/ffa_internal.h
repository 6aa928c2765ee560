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
constexpr int kBottomThreads = 512;  // CTA of the shared-memory FFA kernel
constexpr int kLevelThreads = 256;   // CTA of the global merge-level kernel
constexpr int kLevelRows = 32;       // output rows per CTA of a merge level
constexpr int kFinalThreads = 256;   // CTA of the last-level + S/N kernel
constexpr int kFinalRows = 32;       // output rows per CTA of that kernel

// Device status word bits (first word of every workspace).
constexpr unsigned kDevTimeout = 1u;
constexpr unsigned kDevBadItem = 2u;

// One FFA transform of a search: base period p (bins), m rows of the octave series.
struct TransformDesc {
    int64_t src_off;      // float offset of row 0 in the source buffer
    int64_t scratch_off;  // float offset of row 0 in the scratch buffers
    int64_t trial0;       // index of its first trial in the periodogram
    double tau;           // sampling time of its octave (s)
    int32_t p;            // bins per row
    int32_t m;            // rows
    int32_t kept;         // rows s with P_s < (p + 1) tau  (Sec. 2.3)
    int32_t depth;        // depth of the shared-memory sub-trees (0 = whole tree)
    float inv_std;        // 1 / sqrt(m V_f): noise std of one folded bin, inverted
    int32_t pad;
};
static_assert(sizeof(TransformDesc) == 56, "TransformDesc layout");

// A CTA's share of a launch: transform index and node / row-block index.
struct WorkItem {
    int32_t tr;
    int32_t idx;
};

// Downsampling of one octave: factor f in 64.64 fixed point (exact for a double).
struct OctaveDesc {
    int64_t out_off;   // float offset of the octave's series in the series buffer
    int64_t nk;        // samples: floor(n / f)
    int64_t first;     // index of its first output in the flat launch
    uint64_t f_int;    // floor(f)
    uint64_t f_frac;   // (f - floor(f)) * 2^64, exact
};

struct Widths {
    int32_t nw;
    int32_t wmax;
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
    kFfaLevel,
    kFfaFinalSnr,
    kBoxcarSnr,
    kNumKinds
};

// ------------------------------------------------------------------------------
// Launch parameter blocks.
// ------------------------------------------------------------------------------
struct PrefixParams {
    const void* x;
    int dtype;            // ffa_dtype
    int64_t n;
    float2* partial;      // per-chunk double-float sums
    float2* prefix;       // n + 1 double-float exclusive prefix sums
    int64_t nchunks;
};

struct DownsampleParams {
    const void* x;
    int dtype;
    int64_t n;
    const float2* prefix;
    const OctaveDesc* oct;          // null: one octave, `single`
    OctaveDesc single;
    int noct;
    int64_t total;        // sum of nk
    float* out;           // series buffer
};

struct BottomParams {
    const float* src;               // octave series buffer or the caller's block
    float* dst;                     // where sub-trees of even depth are written
    float* dst_odd;                 // where sub-trees of odd depth are written
    const TransformDesc* trs;       // null: use `single`
    const WorkItem* items;          // null: item = {0, blockIdx.x}
    TransformDesc single;
    Widths widths;
    double* periods;
    int32_t* foldbins;
    float* snr;
    unsigned* status;
    int buf_floats;                 // floats per shared-memory buffer
    int snr_warps;                  // warps that score rows (fused S/N mode)
};

struct LevelParams {
    const float* in;
    float* out;
    const TransformDesc* trs;
    const WorkItem* items;
    TransformDesc single;
    int depth;                      // depth of the nodes this launch computes
};

struct FinalParams {
    const float* in;                // depth-1 transforms
    const TransformDesc* trs;
    const WorkItem* items;
    TransformDesc single;
    Widths widths;
    double* periods;
    int32_t* foldbins;
    float* snr;
    int warp_floats;                // shared floats per warp
};

struct SnrParams {
    const float* prof;
    int64_t rows;
    int cols;
    Widths widths;
    float inv_std;
    float* snr;
    int warp_floats;
};

// Launchers (ffa_kernels.cu).  Each returns the cudaError_t of the launch.
cudaError_t launch_prefix(const PrefixParams& P, cudaStream_t s);
cudaError_t launch_downsample(const DownsampleParams& P, cudaStream_t s);
cudaError_t launch_bottom(const BottomParams& P, int nblocks, int smem_bytes, bool snr_mode,
                          cudaStream_t s);
cudaError_t launch_level(const LevelParams& P, int nblocks, cudaStream_t s);
cudaError_t launch_final(const FinalParams& P, int nblocks, int smem_bytes, cudaStream_t s);
cudaError_t launch_snr(const SnrParams& P, cudaStream_t s);

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
