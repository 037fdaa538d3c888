// mesh.cu -- mesh upload, linear BVH build, vertex rows, closest-point and
// Philox test hooks.
//
// BVH: Morton codes of triangle centroids (30 bits) with the triangle id in
// the low 32 bits (unique keys), CUB radix sort, the parallel hierarchy of
// Karras (HPG 2012, "Maximizing parallelism in the construction of BVHs,
// octrees, and k-d trees"), bottom-up refit with per-node arrival counters.
// Child boxes live in the parent node and are rounded outward to float, so
// one node array serves both FP32 and FP64 traversals conservatively.
#include <cub/cub.cuh>

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mcs_internal.h"

namespace mcs {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
std::string get_error() { return g_err; }
mcs_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MCS_ERR_OOM : MCS_ERR_CUDA;
}
std::atomic<unsigned long long> g_launches{0};

int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ---------------------------------------------------------------- kernels
__global__ void k_validate(const double *V, int nv, const int32_t *F, int nf, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nv; i += gridDim.x * blockDim.x)
        if (!isfinite(V[i])) atomicOr(bad, 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * nf; i += gridDim.x * blockDim.x)
        if (F[i] < 0 || F[i] >= nv) atomicOr(bad, 2);
}

// per-block min / max of the vertex coordinates, then one block folds them
__global__ void k_bounds_partial(const double *V, int nv, double *part) {
    __shared__ double smin[3][256], smax[3][256];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
        for (int k = 0; k < 3; k++) {
            const double x = V[3 * v + k];
            mn[k] = fmin(mn[k], x);
            mx[k] = fmax(mx[k], x);
        }
    for (int k = 0; k < 3; k++) { smin[k][threadIdx.x] = mn[k]; smax[k][threadIdx.x] = mx[k]; }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 3; k++) {
                smin[k][threadIdx.x] = fmin(smin[k][threadIdx.x], smin[k][threadIdx.x + s]);
                smax[k][threadIdx.x] = fmax(smax[k][threadIdx.x], smax[k][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) { part[6 * blockIdx.x + k] = smin[k][0]; part[6 * blockIdx.x + 3 + k] = smax[k][0]; }
}
struct BoxFrame { double lo[3], inv[3]; };

// one warp folds the partial boxes (min and max are exact in any order)
__global__ void k_bounds_final(const double *part, int nb, double *out, BoxFrame *fr) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = lane; b < nb; b += 32)
        for (int k = 0; k < 3; k++) { mn[k] = fmin(mn[k], part[6 * b + k]); mx[k] = fmax(mx[k], part[6 * b + 3 + k]); }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 3; k++) {
            mn[k] = fmin(mn[k], __shfl_xor_sync(0xFFFFFFFFu, mn[k], o));
            mx[k] = fmax(mx[k], __shfl_xor_sync(0xFFFFFFFFu, mx[k], o));
        }
    if (lane != 0) return;
    for (int k = 0; k < 3; k++) {
        out[k] = mn[k];
        out[3 + k] = mx[k];
        fr->lo[k] = mn[k];
        fr->inv[k] = 1.0 / (mx[k] - mn[k]);
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}
__device__ __forceinline__ uint32_t morton30(double x, double y, double z, const double *lo, const double *inv) {
    const double fx = fmin(fmax((x - lo[0]) * inv[0], 0.0), 1.0);
    const double fy = fmin(fmax((y - lo[1]) * inv[1], 0.0), 1.0);
    const double fz = fmin(fmax((z - lo[2]) * inv[2], 0.0), 1.0);
    const uint32_t ix = min((uint32_t)(fx * 1024.0), 1023u);
    const uint32_t iy = min((uint32_t)(fy * 1024.0), 1023u);
    const uint32_t iz = min((uint32_t)(fz * 1024.0), 1023u);
    return (spread10(ix) << 2) | (spread10(iy) << 1) | spread10(iz);
}

// the keys' frame, formed on the device from the bounds (no host round trip);
// the kernels that index V through F return at once when validation flagged
// the input (*bad != 0), which the build reports after its single sync
__global__ void k_tri_keys(const double *V, const int32_t *F, int nf, const BoxFrame *frp, const int *bad,
                           uint32_t *mort, int32_t *fidx) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || *bad) return;
    const BoxFrame fr = *frp;
    const double *a = V + 3 * F[3 * f], *b = V + 3 * F[3 * f + 1], *c = V + 3 * F[3 * f + 2];
    const double cx = ((a[0] + b[0]) + c[0]) / 3.0, cy = ((a[1] + b[1]) + c[1]) / 3.0, cz = ((a[2] + b[2]) + c[2]) / 3.0;
    // sorted stably by the code with the face as value: the order of the
    // unique keys (code << 32 | f) in half the radix passes
    mort[f] = morton30(cx, cy, cz, fr.lo, fr.inv);
    fidx[f] = f;
}

// triangle slots in BVH order: (a, ab, ac) in FP64 and, from float-rounded
// vertices, in FP32; box of each slot rounded outward to float
__global__ void k_tri_slots(const double *V, const int32_t *F, int nf, const uint32_t *mort_s, const int32_t *fidx_s,
                            const int *bad, unsigned long long *keys, Tri32 *t32, Tri64 *t64, float *slotbox) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nf || *bad) return;
    const int f = fidx_s[s];
    keys[s] = ((unsigned long long)mort_s[s] << 32) | (unsigned)f;
    const double *A = V + 3 * F[3 * f], *B = V + 3 * F[3 * f + 1], *C = V + 3 * F[3 * f + 2];
    Tri64 t;
    Tri32 u;
    float fa[3], fab[3], fac[3];
    for (int k = 0; k < 3; k++) {
        t.a[k] = A[k];
        t.ab[k] = B[k] - A[k];
        t.ac[k] = C[k] - A[k];
        const float a = (float)A[k], b = (float)B[k], c = (float)C[k];
        fa[k] = a;
        fab[k] = b - a;
        fac[k] = c - a;
        slotbox[6 * s + k] = __double2float_rd(fmin(fmin(A[k], B[k]), C[k]));
        slotbox[6 * s + 3 + k] = __double2float_ru(fmax(fmax(A[k], B[k]), C[k]));
    }
    t.id = f;
    t.pad = 0;
    u.a = make_float4(fa[0], fa[1], fa[2], __int_as_float(f));
    u.ab = make_float4(fab[0], fab[1], fab[2],
                       __int_as_float(tri_zero_normal<float>(fab[0], fab[1], fab[2], fac[0], fac[1], fac[2]) ? 1 : 0));
    u.ac = make_float4(fac[0], fac[1], fac[2], 0.f);
    t64[s] = t;
    t32[s] = u;
}

__device__ __forceinline__ int kdelta(const unsigned long long *k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    return __clzll(k[i] ^ k[j]);
}

// Karras 2012: internal node i covers a key range [min(i,j), max(i,j)] split
// at gamma; children >= 0 internal, < 0 leaf (~slot)
__global__ void k_karras(const unsigned long long *k, int n, const int *bad, int *child, int *parent_int,
                         int *parent_leaf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1 || *bad) return;
    const int d = (kdelta(k, n, i, i + 1) - kdelta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = kdelta(k, n, i, i - d);
    int lmax = 2;
    while (kdelta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (kdelta(k, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = kdelta(k, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (kdelta(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int gamma = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    int left, right;
    if (lo == gamma) { left = ~gamma; parent_leaf[gamma] = i; }
    else { left = gamma; parent_int[gamma] = i; }
    if (hi == gamma + 1) { right = ~(gamma + 1); parent_leaf[gamma + 1] = i; }
    else { right = gamma + 1; parent_int[gamma + 1] = i; }
    child[2 * i] = left;
    child[2 * i + 1] = right;
}

// bottom-up refit: one thread per leaf climbs; the second arrival at a node
// unites its two child boxes and continues
__global__ void k_refit(int n, const int *child, const int *parent_int, const int *parent_leaf, const float *slotbox,
                        float *nodebox, int *arrive, int *err, const int *bad) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n || *bad) return;
    float box[6];
    for (int k = 0; k < 6; k++) box[k] = slotbox[6 * s + k];
    int me = ~s;
    int p = parent_leaf[s];
    // 64-bit keys bound the depth of the hierarchy by 64
    for (int level = 0;; level++) {
        if (level > 70 || p < 0 || p >= n - 1) { atomicOr(err, kErrTree); return; }
        const int side = (child[2 * p] == me) ? 0 : 1;
        volatile float *nb = nodebox + 12 * p;
        for (int k = 0; k < 6; k++) nb[6 * side + k] = box[k];
        __threadfence();
        if (atomicAdd(&arrive[p], 1) == 0) return;
        __threadfence();
        for (int k = 0; k < 3; k++) {
            box[k] = fminf(nb[k], nb[6 + k]);
            box[3 + k] = fmaxf(nb[3 + k], nb[9 + k]);
        }
        if (p == 0) return;
        me = p;
        p = parent_int[p];
    }
}

__global__ void k_pack_nodes(int n, const int *child, const float *nodebox, const int *bad, Node *nodes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1 || *bad) return;
    const float *b = nodebox + 12 * i;
    Node nd;
    nd.a = make_float4(b[0], b[1], b[2], b[3]);
    nd.b = make_float4(b[4], b[5], b[6], b[7]);
    nd.c = make_float4(b[8], b[9], b[10], b[11]);
    nd.d = make_int4(child[2 * i], child[2 * i + 1], 0, 0);
    nodes[i] = nd;
}

// depth parity of every internal node (the root has depth 0)
__global__ void k_even_depth(int n, const int *parent_int, int *even, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = 0, p = i;
    while (p != 0) {
        p = parent_int[p];
        if (++d > 130 || p < 0 || p >= n - 1) { atomicOr(err, kErrTree); even[i] = 0; return; }
    }
    even[i] = (d & 1) == 0;
}

// 4-wide nodes: every binary node at even depth keeps its children, with an
// internal child (odd depth) replaced by that child's two children; boxes
// are copied, so the 4-wide tree bounds exactly what the binary one does
__global__ void k_collapse4(int n, const int *child, const float *nodebox, const int *even, const int *idx4,
                            Node4 *nodes4) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1 || !even[i]) return;
    float lo[3][4], hi[3][4];
    int ch[4];
    int k = 0;
    auto add = [&](const float *b, int c) {
        for (int a = 0; a < 3; a++) { lo[a][k] = b[a]; hi[a][k] = b[3 + a]; }
        ch[k] = c < 0 ? c : idx4[c];
        k++;
    };
    for (int side = 0; side < 2; side++) {
        const int c = child[2 * i + side];
        if (c < 0) {
            add(nodebox + 12 * i + 6 * side, c);
        } else {
            for (int g = 0; g < 2; g++) add(nodebox + 12 * c + 6 * g, child[2 * c + g]);
        }
    }
    for (; k < 4; k++) {
        for (int a = 0; a < 3; a++) { lo[a][k] = INFINITY; hi[a][k] = -INFINITY; }
        ch[k] = kNoChild;
    }
    Node4 nd;
    nd.lox = make_float4(lo[0][0], lo[0][1], lo[0][2], lo[0][3]);
    nd.loy = make_float4(lo[1][0], lo[1][1], lo[1][2], lo[1][3]);
    nd.loz = make_float4(lo[2][0], lo[2][1], lo[2][2], lo[2][3]);
    nd.hix = make_float4(hi[0][0], hi[0][1], hi[0][2], hi[0][3]);
    nd.hiy = make_float4(hi[1][0], hi[1][1], hi[1][2], hi[1][3]);
    nd.hiz = make_float4(hi[2][0], hi[2][1], hi[2][2], hi[2][3]);
    nd.child = make_int4(ch[0], ch[1], ch[2], ch[3]);
    nd.pad = make_int4(0, 0, 0, 0);
    nodes4[idx4[i]] = nd;
}

// (vertex, face) incidences, sorted stably by vertex: faces ascend within a
// vertex because they enter in face order
__global__ void k_incidence(const int32_t *F, int nf, uint32_t *vkey, int32_t *fval) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    for (int k = 0; k < 3; k++) {
        vkey[3 * f + k] = (uint32_t)F[3 * f + k];
        fval[3 * f + k] = f;
    }
}
__global__ void k_incidence_csr(const uint32_t *vkey, const int32_t *fval, int m, int nv, const int *bad,
                                int32_t *inc_f, int32_t *vstart) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || *bad) return;
    const int v = (int)vkey[i];
    inc_f[i] = fval[i];
    const int vprev = i == 0 ? -1 : (int)vkey[i - 1];
    for (int w = vprev + 1; w <= v; w++) vstart[w] = i;
    if (i == m - 1)
        for (int w = v + 1; w <= nv; w++) vstart[w] = m;
}

// vertex rows: normal = normalised sum of (b-a)x(c-a) over incident faces in
// ascending face order; area = (sum of incident face areas) / 3
__global__ void k_vertex_rows(const double *V, const int32_t *F, const int32_t *inc_f, const int32_t *vstart, int nv,
                              double *pos, double *nrm, double *area) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double S0 = 0.0, S1 = 0.0, S2 = 0.0, A = 0.0;
    for (int e = vstart[v]; e < vstart[v + 1]; e++) {
        const int f = inc_f[e];
        const double *a = V + 3 * F[3 * f], *b = V + 3 * F[3 * f + 1], *c = V + 3 * F[3 * f + 2];
        const double ab0 = b[0] - a[0], ab1 = b[1] - a[1], ab2 = b[2] - a[2];
        const double ac0 = c[0] - a[0], ac1 = c[1] - a[1], ac2 = c[2] - a[2];
        const double N0 = ab1 * ac2 - ab2 * ac1;
        const double N1 = ab2 * ac0 - ab0 * ac2;
        const double N2 = ab0 * ac1 - ab1 * ac0;
        const double ar = 0.5 * sqrt(N0 * N0 + N1 * N1 + N2 * N2);
        S0 += N0; S1 += N1; S2 += N2;
        A += ar;
    }
    const double l = sqrt(S0 * S0 + S1 * S1 + S2 * S2);
    pos[3 * v] = V[3 * v]; pos[3 * v + 1] = V[3 * v + 1]; pos[3 * v + 2] = V[3 * v + 2];
    nrm[3 * v] = l > 0.0 ? S0 / l : 0.0;
    nrm[3 * v + 1] = l > 0.0 ? S1 / l : 0.0;
    nrm[3 * v + 2] = l > 0.0 ? S2 / l : 0.0;
    area[v] = A / 3.0;
}

template <typename T, bool WIDE>
__global__ void k_closest_points(DevMesh m, const double *P, int n, double *d2, int32_t *tri, double *bary,
                                 int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Hit<T> h;
    int e = 0;
    if (WIDE) closest4<T>(m, (T)P[3 * i], (T)P[3 * i + 1], (T)P[3 * i + 2], -1, h, &e);
    else closest<T>(m, (T)P[3 * i], (T)P[3 * i + 1], (T)P[3 * i + 2], -1, h, &e);
    if (e) atomicOr(err, e);
    d2[i] = (double)h.d2;
    tri[i] = h.id;
    bary[3 * i] = (double)h.b0;
    bary[3 * i + 1] = (double)h.b1;
    bary[3 * i + 2] = (double)h.b2;
}

__global__ void k_philox(unsigned long long start, unsigned long long n, uint32_t c2, uint32_t c3, uint32_t k0,
                         uint32_t k1, uint32_t *out) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long g = start + i;
        const uint4 w = philox(make_uint4((uint32_t)g, (uint32_t)(g >> 32), c2, c3), k0, k1);
        reinterpret_cast<uint4 *>(out)[i] = w;
    }
}

}  // namespace mcs

using namespace mcs;

// ---------------------------------------------------------------- host API
static bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static void mesh_free(mcs_mesh_s *m) {
    if (!m) return;
    cudaFree(m->block);  // every array of the mesh but the 4-wide copy
    cudaFree(m->nodes4);
    delete m;
}

// the pool of the BVH build's temporaries, one per device: stream-ordered
// allocation, so that freeing them does not synchronise the device (as
// cudaFree does) and consecutive builds reuse the memory (up to 1 GiB stays
// reserved between builds)
static cudaError_t temp_pool(int dev, cudaMemPool_t *out) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> g(mu);
    const auto it = pools.find(dev);
    if (it != pools.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    cudaMemPool_t p;
    cudaError_t e = cudaMemPoolCreate(&p, &pp);
    if (e != cudaSuccess) return e;
    uint64_t keep = 1ull << 30;
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return e;
    pools[dev] = p;
    *out = p;
    return cudaSuccess;
}

extern "C" {

const char *mcs_last_error(void) { return g_err.c_str(); }
const char *mcs_version(void) { return "mcsteklov 0.1 (sm_103a)"; }

unsigned long long mcs_launch_count(void) { return mcs::g_launches.load(std::memory_order_relaxed); }

void mcs_mesh_destroy(mcs_mesh m) { mesh_free(m); }
int mcs_mesh_nv(mcs_mesh m) { return m ? m->nv : 0; }
int mcs_mesh_nf(mcs_mesh m) { return m ? m->nf : 0; }

}  // extern "C"

static mcs_status build_args(const double *V, int nv, const int32_t *F, int nf, const char *who) {
    MCS_ARG(V != nullptr && F != nullptr, std::string(who) + ": V or F is NULL");
    MCS_ARG(nv >= 3 && nf >= 1, std::string(who) + ": need nv >= 3 and nf >= 1");
    MCS_ARG((long long)nf * 3 < (1LL << 31) && (long long)nv * 3 < (1LL << 31), std::string(who) + ": mesh too large");
    return MCS_OK;
}

// a BVH build enqueued on st without a host round trip: the mesh's arrays
// (one block it owns) and the build's temporaries (pool memory freed in
// stream order); the validation flags (2 ints) and the bounds (6 doubles)
// are copied to flags_dev / box_dev for build_finish.  *out is the mesh
// (its host fields lo, hi, rmax, scale set by build_finish)
static mcs_status build_enqueue(const double *V, int nv, const int32_t *F, int nf, cudaStream_t st, int *flags_dev,
                                double *box_dev, mcs_mesh_s **out) {
    const bool vdev = is_device_ptr(V), fdev = is_device_ptr(F);
    mcs_mesh_s *m = new mcs_mesh_s();
    m->nv = nv;
    m->nf = nf;
    cudaGetDevice(&m->device);
    // two device allocations: the mesh's arrays (one block it owns) and the
    // build's temporaries (one block, freed before returning); parts 256-byte aligned
    void *tbuf = nullptr;
    auto fail = [&](mcs_status s) {
        if (tbuf) cudaFreeAsync(tbuf, st);
        mesh_free(m);
        return s;
    };
#define MB_CUDA(call)                                            \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return fail(cuda_fail(e_, #call)); \
    } while (0)
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ni = nf > 1 ? (size_t)(nf - 1) : 0;
    const size_t msz[11] = {sizeof(double) * 3 * nv, sizeof(int32_t) * 3 * nf, sizeof(int),
                            sizeof(Tri32) * nf,      sizeof(Tri64) * nf,       sizeof(Node) * ni,
                            sizeof(int) * 2 * ni,    sizeof(int) * ni,         sizeof(float) * 12 * ni,
                            sizeof(int32_t) * 3 * nf, sizeof(int32_t) * (nv + 1)};
    size_t mtot = 0;
    for (size_t x : msz) mtot += al(x);
    MB_CUDA(cudaMalloc(&m->block, mtot));
    char *mp = (char *)m->block;
    auto mtake = [&](size_t bytes) -> void * {
        if (!bytes) return nullptr;
        void *r = mp;
        mp += al(bytes);
        return r;
    };
    m->V = (double *)mtake(msz[0]);
    m->F = (int32_t *)mtake(msz[1]);
    m->err = (int *)mtake(msz[2]);
    m->t32 = (Tri32 *)mtake(msz[3]);
    m->t64 = (Tri64 *)mtake(msz[4]);
    m->nodes = (Node *)mtake(msz[5]);
    m->child = (int *)mtake(msz[6]);
    m->parent = (int *)mtake(msz[7]);
    m->nodebox = (float *)mtake(msz[8]);
    m->inc_f = (int32_t *)mtake(msz[9]);
    m->vstart = (int32_t *)mtake(msz[10]);

    // radix passes over the bits that vary: 30 for the Morton codes, those of
    // the largest vertex id for the incidences
    const int vbits = nv > 1 ? 32 - __builtin_clz((unsigned)(nv - 1)) : 1;
    size_t sort_bytes = 0, sort_bytes2 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, (uint32_t *)nullptr, (uint32_t *)nullptr, (int32_t *)nullptr,
                                    (int32_t *)nullptr, nf, 0, 30, st);
    cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes2, (uint32_t *)nullptr, (uint32_t *)nullptr, (int32_t *)nullptr,
                                    (int32_t *)nullptr, 3 * nf, 0, vbits, st);
    const int nbp = 256;
    const size_t tsz[12] = {sizeof(int) * 2,  sizeof(double) * 6 * nbp, sizeof(double) * 6,
                            sizeof(unsigned long long) * nf, sizeof(unsigned long long) * nf,
                            sizeof(unsigned long long) * 3 * nf, sizeof(unsigned long long) * 3 * nf,
                            std::max(sort_bytes, sort_bytes2), sizeof(float) * 6 * nf, sizeof(int) * nf,
                            sizeof(int) * ni, sizeof(BoxFrame)};
    size_t ttot = 0;
    for (size_t x : tsz) ttot += al(x);
    cudaMemPool_t pool;
    MB_CUDA(temp_pool(m->device, &pool));
    MB_CUDA(cudaMallocFromPoolAsync(&tbuf, ttot, pool, st));
    char *tp = (char *)tbuf;
    auto ttake = [&](size_t bytes) -> void * {
        void *r = tp;
        tp += al(bytes);
        return r;
    };
    int *d_bad = (int *)ttake(tsz[0]);
    double *d_part = (double *)ttake(tsz[1]);
    double *d_box = (double *)ttake(tsz[2]);
    unsigned long long *keys = (unsigned long long *)ttake(tsz[3]);
    unsigned long long *keys_s = (unsigned long long *)ttake(tsz[4]);
    unsigned long long *pairs = (unsigned long long *)ttake(tsz[5]);
    unsigned long long *pairs_s = (unsigned long long *)ttake(tsz[6]);
    void *d_sort = ttake(tsz[7]);
    float *slotbox = (float *)ttake(tsz[8]);
    int *par_l = (int *)ttake(tsz[9]);
    int *arrive = (int *)ttake(tsz[10]);
    BoxFrame *d_frame = (BoxFrame *)ttake(tsz[11]);

    MB_CUDA(cudaMemsetAsync(m->err, 0, sizeof(int), st));
    MB_CUDA(cudaMemcpyAsync(m->V, V, sizeof(double) * 3 * nv, vdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    MB_CUDA(cudaMemcpyAsync(m->F, F, sizeof(int32_t) * 3 * nf, fdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    MB_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int) * 2, st));
    note_launch();
    k_validate<<<num_sms() * 4, 256, 0, st>>>(m->V, nv, m->F, nf, d_bad);
    note_launch();
    k_bounds_partial<<<nbp, 256, 0, st>>>(m->V, nv, d_part);
    note_launch();
    k_bounds_final<<<1, 32, 0, st>>>(d_part, nbp, d_box, d_frame);
    const int tb = 256;
    note_launch();
    // Morton codes and faces in the keys' space, sorted into the incidences'
    // (both used again only later)
    uint32_t *mort = (uint32_t *)keys, *mort_s = (uint32_t *)pairs_s;
    int32_t *fidx = (int32_t *)(mort + nf), *fidx_s = (int32_t *)(mort_s + nf);
    k_tri_keys<<<(nf + tb - 1) / tb, tb, 0, st>>>(m->V, m->F, nf, d_frame, d_bad, mort, fidx);
    MB_CUDA(cub::DeviceRadixSort::SortPairs(d_sort, sort_bytes, mort, mort_s, fidx, fidx_s, nf, 0, 30, st));
    note_launch();
    k_tri_slots<<<(nf + tb - 1) / tb, tb, 0, st>>>(m->V, m->F, nf, mort_s, fidx_s, d_bad, keys_s, m->t32, m->t64,
                                                    slotbox);
    if (nf > 1) {
        // links, parents and child boxes go straight into the mesh (kept for
        // an on-demand 4-wide copy, mcs_mesh_build_wide)
        MB_CUDA(cudaMemsetAsync(arrive, 0, sizeof(int) * (nf - 1), st));
        MB_CUDA(cudaMemsetAsync(m->parent, 0xFF, sizeof(int) * (nf - 1), st));
        MB_CUDA(cudaMemsetAsync(par_l, 0xFF, sizeof(int) * nf, st));
        note_launch();
        k_karras<<<(nf - 1 + tb - 1) / tb, tb, 0, st>>>(keys_s, nf, d_bad, m->child, m->parent, par_l);
        note_launch();
        k_refit<<<(nf + tb - 1) / tb, tb, 0, st>>>(nf, m->child, m->parent, par_l, slotbox, m->nodebox, arrive,
                                                     d_bad + 1, d_bad);
        note_launch();
        k_pack_nodes<<<(nf - 1 + tb - 1) / tb, tb, 0, st>>>(nf, m->child, m->nodebox, d_bad, m->nodes);
    }
    // vertex -> incident faces, ascending
    note_launch();
    uint32_t *vkey = (uint32_t *)pairs, *vkey_s = (uint32_t *)pairs_s;
    int32_t *fval = (int32_t *)(vkey + 3 * (size_t)nf), *fval_s = (int32_t *)(vkey_s + 3 * (size_t)nf);
    k_incidence<<<(nf + tb - 1) / tb, tb, 0, st>>>(m->F, nf, vkey, fval);
    MB_CUDA(cub::DeviceRadixSort::SortPairs(d_sort, sort_bytes2, vkey, vkey_s, fval, fval_s, 3 * nf, 0, vbits, st));
    MB_CUDA(cudaMemsetAsync(m->vstart, 0, sizeof(int32_t) * (nv + 1), st));
    note_launch();
    k_incidence_csr<<<(3 * nf + tb - 1) / tb, tb, 0, st>>>(vkey_s, fval_s, 3 * nf, nv, d_bad, m->inc_f, m->vstart);
    MB_CUDA(cudaGetLastError());
    MB_CUDA(cudaMemcpyAsync(flags_dev, d_bad, sizeof(int) * 2, cudaMemcpyDeviceToDevice, st));
    MB_CUDA(cudaMemcpyAsync(box_dev, d_box, sizeof(double) * 6, cudaMemcpyDeviceToDevice, st));
    MB_CUDA(cudaFreeAsync(tbuf, st));
    tbuf = nullptr;
#undef MB_CUDA
    *out = m;
    return MCS_OK;
}

// the checks of a build once its flags and bounds are on the host
static mcs_status build_finish(mcs_mesh_s *m, const int *flags, const double *box) {
    if (flags[0]) {
        set_error(flags[0] & 1 ? "mcs_build_bvh: non-finite vertex coordinate" : "mcs_build_bvh: face index out of range");
        return MCS_ERR_DEGENERATE;
    }
    double side = INFINITY, scale = 0.0;
    for (int k = 0; k < 3; k++) {
        m->lo[k] = box[k];
        m->hi[k] = box[3 + k];
        side = fmin(side, box[3 + k] - box[k]);
        scale = fmax(scale, fmax(fabs(box[k]), fabs(box[3 + k])));
    }
    if (!(side > 0.0)) {
        set_error("mcs_build_bvh: the bounding box has a zero-length side");
        return MCS_ERR_DEGENERATE;
    }
    m->rmax = 0.5 * side;
    m->scale = (float)scale * (1.0f + 1e-6f);
    if (flags[1]) {
        set_error("mcs_build_bvh: internal error, malformed hierarchy");
        return MCS_ERR_DEVICE;
    }
    return MCS_OK;
}

extern "C" {

mcs_status mcs_build_bvh(const double *V, int nv, const int32_t *F, int nf, void *stream_, mcs_mesh *out) {
    NvtxRange nvtx_range("mcs_build_bvh");
    MCS_ARG(out != nullptr, "mcs_build_bvh: out is NULL");
    *out = nullptr;
    mcs_status s = build_args(V, nv, F, nf, "mcs_build_bvh");
    if (s != MCS_OK) return s;
    return mcs_build_bvh_batched(1, &V, &nv, &F, &nf, stream_, out);
}

mcs_status mcs_build_bvh_batched(int count, const double *const *V, const int *nv, const int32_t *const *F,
                                 const int *nf, void *stream_, mcs_mesh *out) {
    NvtxRange nvtx_range("mcs_build_bvh_batched");
    MCS_ARG(count >= 1 && V && nv && F && nf && out, "mcs_build_bvh_batched: NULL array or count < 1");
    for (int i = 0; i < count; i++) out[i] = nullptr;
    for (int i = 0; i < count; i++) {
        const mcs_status s = build_args(V[i], nv[i], F[i], nf[i], "mcs_build_bvh_batched");
        if (s != MCS_OK) return s;
    }
    cudaStream_t st = as_stream(stream_);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    MCS_CUDA(temp_pool(dev, &pool));
    // every build's flags (2 ints) and bounds (6 doubles) in one 64-byte slot
    void *stat = nullptr;
    MCS_CUDA(cudaMallocFromPoolAsync(&stat, 64 * (size_t)count, pool, st));
    std::vector<mcs_mesh_s *> ms(count, nullptr);
    auto free_all = [&]() {
        for (mcs_mesh_s *m : ms) mesh_free(m);
        if (stat) cudaFreeAsync(stat, st);
    };
    for (int i = 0; i < count; i++) {
        char *slot = (char *)stat + 64 * (size_t)i;
        const mcs_status s = build_enqueue(V[i], nv[i], F[i], nf[i], st, (int *)slot, (double *)(slot + 16), &ms[i]);
        if (s != MCS_OK) {
            free_all();
            return s;
        }
    }
    std::vector<unsigned char> host(64 * (size_t)count);
    cudaError_t e = cudaMemcpyAsync(host.data(), stat, host.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaFreeAsync(stat, st);
    stat = nullptr;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_all();
        return cuda_fail(e, "mcs_build_bvh_batched");
    }
    for (int i = 0; i < count; i++) {
        const unsigned char *slot = host.data() + 64 * (size_t)i;
        const mcs_status s = build_finish(ms[i], (const int *)slot, (const double *)(slot + 16));
        if (s != MCS_OK) {
            if (count > 1) set_error("mesh " + std::to_string(i) + ": " + g_err);
            free_all();
            return s;
        }
    }
    for (int i = 0; i < count; i++) out[i] = ms[i];
    // mesh creation may allocate: load here what the allocation-free
    // estimate needs, so that it loads (and allocates) nothing itself; a
    // failure here only surfaces when that entry point is called
    (void)noalloc_prepare();
    return MCS_OK;
}

mcs_status mcs_mesh_build_wide(mcs_mesh m, void *stream_) {
    MCS_ARG(m != nullptr, "mcs_mesh_build_wide: mesh is NULL");
    if (m->nf < 2 || m->nodes4) return MCS_OK;
    cudaStream_t st = as_stream(stream_);
    const int nf = m->nf, tb = 256;
    int *even = nullptr, *idx4 = nullptr, *d_err = nullptr;
    void *d_scan = nullptr;
    size_t scan_bytes = 0;
    auto cleanup = [&]() { cudaFree(even); cudaFree(idx4); cudaFree(d_scan); cudaFree(d_err); };
    cudaError_t e = cudaMalloc(&even, sizeof(int) * (nf - 1));
    if (e == cudaSuccess) e = cudaMalloc(&idx4, sizeof(int) * nf);
    if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(int));
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, even, idx4, nf - 1, st);
    if (e == cudaSuccess) e = cudaMalloc(&d_scan, scan_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "mcs_mesh_build_wide: allocation"); }
    // the 4-wide copy: nodes at even depth, numbered by an exclusive scan
    note_launch();
    k_even_depth<<<(nf - 1 + tb - 1) / tb, tb, 0, st>>>(nf, m->parent, even, d_err);
    e = cub::DeviceScan::ExclusiveSum(d_scan, scan_bytes, even, idx4, nf - 1, st);
    int last[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[0], idx4 + (nf - 2), sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[1], even + (nf - 2), sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[2], d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "mcs_mesh_build_wide"); }
    if (last[2]) {
        cleanup();
        set_error("mcs_mesh_build_wide: internal error, malformed hierarchy");
        return MCS_ERR_DEVICE;
    }
    const int n4 = last[0] + last[1];
    Node4 *nodes4 = nullptr;
    e = cudaMalloc(&nodes4, sizeof(Node4) * std::max(1, n4));
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "mcs_mesh_build_wide: allocation"); }
    note_launch();
    k_collapse4<<<(nf - 1 + tb - 1) / tb, tb, 0, st>>>(nf, m->child, m->nodebox, even, idx4, nodes4);
    e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) { cudaFree(nodes4); return cuda_fail(e, "mcs_mesh_build_wide"); }
    m->nodes4 = nodes4;
    m->n4 = n4;
    return MCS_OK;
}

int mcs_mesh_has_wide(mcs_mesh m) { return m && (m->nf < 2 || m->nodes4 != nullptr); }

mcs_status mcs_vertex_rows(mcs_mesh m, double *pos, double *nrm, double *area, void *stream_) {
    MCS_ARG(m != nullptr, "mcs_vertex_rows: mesh is NULL");
    MCS_ARG(pos && nrm && area, "mcs_vertex_rows: NULL output");
    cudaStream_t st = as_stream(stream_);
    note_launch();
    k_vertex_rows<<<(m->nv + 255) / 256, 256, 0, st>>>(m->V, m->F, m->inc_f, m->vstart, m->nv, pos, nrm, area);
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

mcs_status mcs_closest_points(mcs_mesh m, const double *P, int n, int prec, int layout, double *d2, int32_t *tri,
                              double *bary, void *stream_) {
    MCS_ARG(m != nullptr, "mcs_closest_points: mesh is NULL");
    MCS_ARG(n >= 0, "mcs_closest_points: n < 0");
    MCS_ARG(prec == 32 || prec == 64, "mcs_closest_points: prec must be 32 or 64");
    MCS_ARG(layout == 2 || layout == 4, "mcs_closest_points: layout must be 2 or 4");
    MCS_ARG(layout == 2 || mcs_mesh_has_wide(m), "mcs_closest_points: layout 4 needs mcs_mesh_build_wide first");
    if (n == 0) return MCS_OK;
    MCS_ARG(P && d2 && tri && bary, "mcs_closest_points: NULL pointer");
    cudaStream_t st = as_stream(stream_);
    int *d_err = m->err;
    MCS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    note_launch();
    const int g = (n + 127) / 128;
    if (layout == 4) {
        if (prec == 64) k_closest_points<double, true><<<g, 128, 0, st>>>(m->dev(), P, n, d2, tri, bary, d_err);
        else k_closest_points<float, true><<<g, 128, 0, st>>>(m->dev(), P, n, d2, tri, bary, d_err);
    } else {
        if (prec == 64) k_closest_points<double, false><<<g, 128, 0, st>>>(m->dev(), P, n, d2, tri, bary, d_err);
        else k_closest_points<float, false><<<g, 128, 0, st>>>(m->dev(), P, n, d2, tri, bary, d_err);
    }
    int err = 0;
    MCS_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MCS_CUDA(cudaStreamSynchronize(st));
    if (err) {
        set_error("mcs_closest_points: BVH traversal stack overflow");
        return MCS_ERR_DEVICE;
    }
    return MCS_OK;
}

mcs_status mcs_philox_words(uint64_t start, uint64_t n, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                            uint32_t *out, void *stream_) {
    MCS_ARG(out != nullptr || n == 0, "mcs_philox_words: out is NULL");
    if (n == 0) return MCS_OK;
    note_launch();
    k_philox<<<num_sms() * 4, 256, 0, as_stream(stream_)>>>(start, n, c2, c3, k0, k1, out);
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

}  // extern "C"
