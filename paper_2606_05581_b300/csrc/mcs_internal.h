// mcs_internal.h -- host-side internals shared by the library's .cu files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mcsteklov.h"
#include "mcs_device.cuh"

struct mcs_mesh_s {
    int device = 0;
    int nv = 0, nf = 0;
    // device memory owned by the mesh: one block (`block`) holding the arrays
    // below, except the 4-wide copy (`nodes4`, its own allocation)
    void *block = nullptr;
    double *V = nullptr;           // nv x 3
    int32_t *F = nullptr;          // nf x 3
    mcs::Node *nodes = nullptr;    // nf - 1
    mcs::Node4 *nodes4 = nullptr;  // n4: the same tree, 4-wide (mcs_mesh_build_wide)
    int n4 = 0;
    int *child = nullptr;          // binary links, parents and child boxes, kept for the 4-wide copy
    int *parent = nullptr;
    float *nodebox = nullptr;
    mcs::Tri32 *t32 = nullptr;     // nf
    mcs::Tri64 *t64 = nullptr;     // nf
    int32_t *inc_f = nullptr;      // 3 nf: faces of each vertex, ascending
    int32_t *vstart = nullptr;     // nv + 1
    int *err = nullptr;            // device status word of the test hooks
    // host copies of mesh constants
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    double rmax = 0.0;             // interior tangent-ball clamp: half the shortest AABB side
    float scale = 0.f;             // max |coordinate|
    mcs::DevMesh dev() const {
        mcs::DevMesh d;
        d.V = V; d.F = F; d.nodes = nodes; d.nodes4 = nodes4; d.t32 = t32; d.t64 = t64;
        d.nv = nv; d.nf = nf; d.scale = scale;
        return d;
    }
};

namespace mcs {
void set_error(const std::string &msg);
std::string get_error();
mcs_status cuda_fail(cudaError_t e, const char *what);
inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
int num_sms();
// kernels of this library enqueued since it was loaded (mcs_launch_count)
extern std::atomic<unsigned long long> g_launches;
inline void note_launch(unsigned long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }
// an NVTX range over a scope (entry points and their phases: profilers
// attribute the kernels launched inside it; no cost without a tool attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
// load (CUDA loads code lazily) every kernel of a one-mesh estimate
mcs_status preload_estimate_kernels();
// load the allocation-free estimate's scratch array and the estimate's
// kernels on the current device; called by mesh creation, which allocates anyway
mcs_status noalloc_prepare();
}  // namespace mcs

#define MCS_CUDA(call)                                                      \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return mcs::cuda_fail(e_, #call);            \
    } while (0)

#define MCS_ARG(cond, msg)                                                  \
    do {                                                                    \
        if (!(cond)) {                                                      \
            mcs::set_error(msg);                                            \
            return MCS_ERR_ARG;                                             \
        }                                                                   \
    } while (0)
