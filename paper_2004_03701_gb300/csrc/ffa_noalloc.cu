// ffa_noalloc.cu -- ffa_transform for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or size and own a workspace: plugins whose host
// application manages every device allocation, pipelines that forbid allocation once
// they are running, or code whose device memory is all reserved by another runtime's
// pool.  ffa_transform_noalloc serves them: it runs the same kernels as ffa_transform,
// but its scratch (the status word and one m x p intermediate buffer) lives in a
// file-scope __device__ array of fixed size that every GPU loading this library holds
// until the process exits.  The caller still provides the input and output buffers.
#include "ffa.h"
#include "ffa_internal.h"

#include <mutex>

namespace ffa {
// Thread-local flag read by LaunchScope: no profiling events are created while set.
extern thread_local bool g_no_alloc_call;
ffa_status set_error(ffa_status st, const char* msg);  // ffa_last_error() text
}  // namespace ffa

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;  // 4 MiB per device

// The shared scratch.  Its host-side name is only a stand-in: the device address is
// obtained with cudaGetSymbolAddress, once per device, below.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_addr[256] = {};  // device address of the scratch, per device (set up once)

}  // namespace

extern "C" ffa_status ffa_transform_noalloc(const float* d_in, int32_t rows, int32_t cols,
                                            float* d_out, void* stream) {
    size_t need = 0;
    ffa_status st = ffa_transform_workspace(rows, cols, &need);
    if (st != FFA_OK) return st;
    if (need > kNoAllocScratchBytes)
        return ffa::set_error(FFA_ERR_CAPACITY,
                              "ffa_transform_noalloc: this block needs more scratch than the "
                              "fixed 4 MiB (rows * cols above 1048512 when sub-trees are "
                              "needed); use ffa_transform with a workspace");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
        return ffa::set_error(FFA_ERR_CUDA, "ffa_transform_noalloc: no current device");
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            // set-up, once per device, with that device current
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return ffa::set_error(FFA_ERR_CUDA, "ffa_transform_noalloc: "
                                                    "cudaGetSymbolAddress of the scratch failed");
            }
            g_addr[dev] = p;
        }
        scratch = g_addr[dev];
    }
    ffa::g_no_alloc_call = true;
    st = ffa_transform(d_in, rows, cols, d_out, scratch, kNoAllocScratchBytes, stream);
    ffa::g_no_alloc_call = false;
    return st;
}
