// lx_eri_batch_static: the batch evaluation for callers that cannot allocate device memory.
//
// Some host programs cannot hand this library a workspace: their device memory is owned by
// an allocator the integral code cannot reach (a plugin inside another framework's memory
// pool), or the process runs where cudaMalloc is not permitted.  For them this entry point
// runs the same kernels with a fixed scratch array that lives in the library's own device
// image, so the call needs nothing but the inputs and the output buffer.
//
// The array is a file-scope __device__ object: every GPU on which the library's device code
// is loaded holds LX_STATIC_SCRATCH_BYTES for it until the process exits.  In host code its
// name is only a host-side stand-in, so its device address is looked up with
// cudaGetSymbolAddress, once per device with that device current (on the first call made
// on that device), and only that address is handed to the kernels.
#include <mutex>

#include "lx_internal.cuh"

namespace {

__device__ __align__(256) unsigned char lx_static_scratch[LX_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void* g_scratch_ptr[MAX_DEVICES];

}  // namespace

extern "C" int lx_eri_batch_static(const lx_shell* shells, int32_t nshell, const double* exps, const double* coefs,
                                   int32_t nprim_total, const lx_quartet* quartets, int64_t nquartet, int32_t flags,
                                   double* out, void* cuda_stream) {
    // Routing needs scratch this entry does not have; stage timing would create CUDA events.
    if (flags & (LX_PATH_ROUTED | LX_TIME_STAGES)) return LX_ERR_FLAGS;
    // The smallest workspace this batch can run in (it is processed in chunks that fit).
    const int64_t need = lx_eri_workspace_min(shells, nshell, quartets, nquartet, flags);
    if (need < 0) return (int)need;
    if (need > (int64_t)LX_STATIC_SCRATCH_BYTES) return LX_ERR_STATIC_SCRATCH;
    // A capturing stream is refused (the descriptor uploads below read host vectors that are
    // released when the call returns); then the device is set up and its architecture checked.
    unsigned* status = nullptr;
    int v = lx::entry_prepare(cuda_stream, "lx_eri_batch_static", &status);
    if (v != LX_OK) return v;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lx::report_cuda_error(e);
    if (dev < 0 || dev >= MAX_DEVICES) return LX_ERR_ARCH;
    void* ptr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if ((e = cudaGetSymbolAddress(&p, lx_static_scratch)) != cudaSuccess) return lx::report_cuda_error(e);
            if (!p) return LX_ERR_CUDA;
            g_scratch_ptr[dev] = p;
        }
        ptr = g_scratch_ptr[dev];
    }
    // Nothing in the pipeline reads scratch it has not written in the same call, so the
    // array's leftover contents from an earlier call need no clearing.  The descriptors are
    // uploaded from pageable memory: no pinned staging buffer is allocated for this call.
    return lx::eri_batch_unstaged(shells, nshell, exps, coefs, nprim_total, quartets, nquartet, flags, out, ptr,
                                  (size_t)LX_STATIC_SCRATCH_BYTES, cuda_stream);
}
