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
#include "mcs_internal.h"

namespace {

// scratch of the allocation-free estimate; every GPU that loads the library
// holds these bytes until the process exits
constexpr size_t kNoAllocBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// device address of the scratch array in the current CUDA context (host
// code cannot use the symbol's name as a device address).  Looked up on
// every call, so that a new context (after cudaDeviceReset) never sees a
// stale address; once the module is loaded the lookup allocates nothing.
mcs_status scratch_address(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return mcs::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = p;
    return MCS_OK;
}

}  // namespace

// called by mesh creation (which allocates anyway) on the current device:
// loading noalloc.cu's module reserves the scratch array, and the estimate's
// kernels are loaded too, so that the entry point below loads nothing
mcs_status mcs::noalloc_prepare() {
    // at every mesh creation (once per batched build): after a device reset
    // the modules load again, so no memo of an earlier load is kept; once
    // loaded, these queries are cheap
    void *p = nullptr;
    const mcs_status s = scratch_address(&p);
    if (s != MCS_OK) return s;
    return mcs::preload_estimate_kernels();
}

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
    // phase timing would create CUDA events; keep this call free of them.
    // The walks run in the caller's row order: the Z-order schedule needs a
    // library sort whose kernels depend on the size; the results do not
    // depend on the schedule (counter-based walks, exact argmin)
    mcs_params q = *p;
    q.timing = 0;
    q.queue_order |= 1;
    return mcs_estimate_dtn(m, rows, &q, out, scratch, kNoAllocBytes, stats, stream);
}

}  // extern "C"
