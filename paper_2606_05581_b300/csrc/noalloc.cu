// noalloc.cu -- an allocation-free variant of mcs_estimate_dtn.
//
// Some callers cannot allocate device memory at the point where they need an
// estimate: code running inside a memory pool or arena they do not own, a
// custom allocator that forbids cudaMalloc during a critical section, or a
// host process whose allocator state must not change (for example while other
// work holds the device's memory close to full).  For them this entry point
// runs the same estimator with its scratch taken from one fixed array that
// the library reserves in device memory when it is loaded, so the call itself
// allocates nothing.
#include <mutex>

#include "mcs_internal.h"

namespace {

// scratch of the allocation-free estimate; every GPU that loads the library
// holds these bytes until the process exits
constexpr size_t kNoAllocBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices] = {};

// device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol's name as a device address)
mcs_status scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mcs::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        mcs::set_error("mcs_estimate_dtn_noalloc: device index out of range");
        return MCS_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return mcs::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return MCS_OK;
}

}  // namespace

extern "C" {

size_t mcs_estimate_dtn_noalloc_capacity(void) { return kNoAllocBytes; }

mcs_status mcs_estimate_dtn_noalloc(mcs_mesh m, const mcs_rows *rows, const mcs_params *p, const mcs_outputs *out,
                                    mcs_stats *stats, void *stream) {
    MCS_ARG(m && rows && p && out, "mcs_estimate_dtn_noalloc: NULL mesh, rows, params or outputs");
    MCS_ARG(rows->n_rows > 0 && p->walks_per_row > 0, "mcs_estimate_dtn_noalloc: n_rows and walks_per_row must be positive");
    const size_t need = mcs_estimate_workspace_size(m, rows->n_rows, p->walks_per_row, p->killing_walks);
    if (need > kNoAllocBytes) {
        mcs::set_error("mcs_estimate_dtn_noalloc: the estimate needs " + std::to_string(need) +
                       " bytes of scratch, more than the fixed " + std::to_string(kNoAllocBytes) +
                       " (use mcs_estimate_dtn with a caller workspace)");
        return MCS_ERR_ARG;
    }
    void *scratch = nullptr;
    const mcs_status s = scratch_address(&scratch);
    if (s != MCS_OK) return s;
    // phase timing would create CUDA events; keep this call free of them
    mcs_params q = *p;
    q.timing = 0;
    return mcs_estimate_dtn(m, rows, &q, out, scratch, kNoAllocBytes, stats, stream);
}

}  // extern "C"
