// rows.cu -- sample rows for the point basis (Sec. 4.4, point-based Galerkin
// basis: points sampled on the surface; farthest-point sampling stands in for
// the paper's blue-noise sampling):
//   FPS        greedy farthest-point sampling over face centroids from face 0,
//              FP64, one cooperative persistent kernel with a bounded grid
//              barrier per selection; each face keeps its nearest sample
//              (first selected on ties) -> tri2bin;
//   areas      each sample's quadrature area = area of the faces it owns,
//              summed in ascending face order (stable sort + segments);
//   normals    unit face normal of the sampled face, oriented outward by the
//              generalized winding number of the other faces (App. A item 1):
//              keep n when GWN(x - delta n) > GWN(x + delta n),
//              delta = sqrt(area)/4; winding numbers in FP32, brute force.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>

#include "mcs_internal.h"

namespace mcs {
namespace rows {

constexpr int kErrBarrier = 128;

__device__ __forceinline__ uint64_t gtime_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// grid-wide barrier for a cooperative launch; every wait is bounded (~2 s),
// after which the error word is set and the block carries on
__device__ void grid_barrier(unsigned *count, unsigned *gen, unsigned nblocks, int *err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = gen;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            *count = 0;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t t0 = gtime_ns();
            while (*vgen == g) {
                if (gtime_ns() - t0 > 2000000000ull) {
                    atomicOr(err, kErrBarrier);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

__global__ void k_centroids(const double *V, const int32_t *F, int nf, double *cen, double *farea, double *mind,
                            int32_t *owner) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const double *a = V + 3 * F[3 * f], *b = V + 3 * F[3 * f + 1], *c = V + 3 * F[3 * f + 2];
    for (int i = 0; i < 3; i++) cen[3 * f + i] = ((a[i] + b[i]) + c[i]) / 3.0;
    const double ab0 = b[0] - a[0], ab1 = b[1] - a[1], ab2 = b[2] - a[2];
    const double ac0 = c[0] - a[0], ac1 = c[1] - a[1], ac2 = c[2] - a[2];
    const double N0 = ab1 * ac2 - ab2 * ac1, N1 = ab2 * ac0 - ab0 * ac2, N2 = ab0 * ac1 - ab1 * ac0;
    farea[f] = 0.5 * sqrt(N0 * N0 + N1 * N1 + N2 * N2);
    mind[f] = INFINITY;
    owner[f] = -1;
}

struct FpsArgs {
    const double *cen;
    double *mind;
    int32_t *owner;
    int32_t *sel;
    double *cand_v;     // 2 x gridDim candidates (double-buffered)
    int *cand_i;
    unsigned *bar;      // count, generation
    int *err;
    int nf, ns;
};

// greedy farthest-point sampling; sel[0] = 0
__global__ void __launch_bounds__(256) k_fps(FpsArgs a) {
    __shared__ double rv[256];
    __shared__ int ri[256];
    __shared__ int s_next;
    const unsigned nb = gridDim.x;
    int cur = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.sel[0] = 0;
    for (int i = 0; i < a.ns; i++) {
        const double qx = a.cen[3 * cur], qy = a.cen[3 * cur + 1], qz = a.cen[3 * cur + 2];
        double bv = -1.0;
        int bi = 0x7FFFFFFF;
        for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < a.nf; f += nb * blockDim.x) {
            const double d0 = a.cen[3 * f] - qx, d1 = a.cen[3 * f + 1] - qy, d2 = a.cen[3 * f + 2] - qz;
            const double d = d0 * d0 + d1 * d1 + d2 * d2;
            double md = a.mind[f];
            if (d < md) {
                md = d;
                a.mind[f] = d;
                a.owner[f] = i;
            }
            if (md > bv) { bv = md; bi = f; }
        }
        if (i + 1 == a.ns) break;
        rv[threadIdx.x] = bv;
        ri[threadIdx.x] = bi;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const double ov = rv[threadIdx.x + s];
                const int oi = ri[threadIdx.x + s];
                if (ov > rv[threadIdx.x] || (ov == rv[threadIdx.x] && oi < ri[threadIdx.x])) {
                    rv[threadIdx.x] = ov;
                    ri[threadIdx.x] = oi;
                }
            }
            __syncthreads();
        }
        const int par = i & 1;
        if (threadIdx.x == 0) {
            a.cand_v[par * nb + blockIdx.x] = rv[0];
            a.cand_i[par * nb + blockIdx.x] = ri[0];
        }
        __threadfence();
        grid_barrier(a.bar, a.bar + 1, nb, a.err);
        // every block folds the candidates the same way
        if (threadIdx.x == 0) {
            double v = -1.0;
            int idx = 0x7FFFFFFF;
            for (unsigned b = 0; b < nb; b++) {
                const double ov = ((volatile double *)a.cand_v)[par * nb + b];
                const int oi = ((volatile int *)a.cand_i)[par * nb + b];
                if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
            }
            s_next = idx;
            if (blockIdx.x == 0) a.sel[i + 1] = idx;
        }
        __syncthreads();
        cur = s_next;
    }
}

__global__ void k_owner_keys(const int32_t *owner, int nf, int32_t *keys, int32_t *vals) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    keys[f] = owner[f];
    vals[f] = f;
}
// start of each owner's segment in the sorted list
__global__ void k_segments(const int32_t *skeys, int nf, int ns, int32_t *start) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nf) return;
    const int k = skeys[e];
    const int kp = e == 0 ? -1 : skeys[e - 1];
    for (int w = kp + 1; w <= k; w++) start[w] = e;
    if (e == nf - 1)
        for (int w = k + 1; w <= ns; w++) start[w] = nf;
}
__global__ void k_sample_rows(const double *V, const int32_t *F, const double *cen, const double *farea,
                              const int32_t *sel, const int32_t *sfaces, const int32_t *start, int ns, double *pos,
                              double *nrm, double *area) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    double s = 0.0;
    for (int e = start[i]; e < start[i + 1]; e++) s += farea[sfaces[e]];
    area[i] = s;
    const int f = sel[i];
    const double *a = V + 3 * F[3 * f], *b = V + 3 * F[3 * f + 1], *c = V + 3 * F[3 * f + 2];
    const double ab0 = b[0] - a[0], ab1 = b[1] - a[1], ab2 = b[2] - a[2];
    const double ac0 = c[0] - a[0], ac1 = c[1] - a[1], ac2 = c[2] - a[2];
    const double N0 = ab1 * ac2 - ab2 * ac1, N1 = ab2 * ac0 - ab0 * ac2, N2 = ab0 * ac1 - ab1 * ac0;
    const double l = sqrt(N0 * N0 + N1 * N1 + N2 * N2);
    nrm[3 * i] = l > 0.0 ? N0 / l : 0.0;
    nrm[3 * i + 1] = l > 0.0 ? N1 / l : 0.0;
    nrm[3 * i + 2] = l > 0.0 ? N2 / l : 0.0;
    for (int k = 0; k < 3; k++) pos[3 * i + k] = cen[3 * f + k];
}

// query points x -/+ delta n of every sample (FP32), and the face each excludes
__global__ void k_gwn_points(const double *pos, const double *nrm, const double *farea, const int32_t *sel, int ns,
                             float4 *q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const double delta = 0.25 * sqrt(farea[sel[i]]);
    for (int side = 0; side < 2; side++) {
        const double sg = side == 0 ? -1.0 : 1.0;
        q[2 * i + side] = make_float4((float)(pos[3 * i] + sg * delta * nrm[3 * i]),
                                      (float)(pos[3 * i + 1] + sg * delta * nrm[3 * i + 1]),
                                      (float)(pos[3 * i + 2] + sg * delta * nrm[3 * i + 2]), __int_as_float(sel[i]));
    }
}

constexpr int kGwnChunks = 16;
// partial[c][j] = sum over faces of chunk c (except the excluded one) of the
// signed solid angle (Van Oosterom & Strackee 1983) seen from query j
__global__ void __launch_bounds__(256) k_gwn(const double *V, const int32_t *F, int nf, const float4 *q, int nq,
                                             float *partial) {
    __shared__ float tri[256][9];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = (nf + kGwnChunks - 1) / kGwnChunks;
    const int f0 = blockIdx.y * chunk, f1 = min(nf, f0 + chunk);
    float4 p = j < nq ? q[j] : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    const int excl = __float_as_int(p.w);
    float acc = 0.f;
    for (int t0 = f0; t0 < f1; t0 += 256) {
        const int f = t0 + threadIdx.x;
        if (f < f1) {
            for (int k = 0; k < 3; k++) {
                const double *v = V + 3 * F[3 * f + k];
                tri[threadIdx.x][3 * k] = (float)v[0];
                tri[threadIdx.x][3 * k + 1] = (float)v[1];
                tri[threadIdx.x][3 * k + 2] = (float)v[2];
            }
        }
        __syncthreads();
        const int cnt = min(256, f1 - t0);
        for (int t = 0; t < cnt; t++) {
            if (t0 + t == excl) continue;
            const float ax = tri[t][0] - p.x, ay = tri[t][1] - p.y, az = tri[t][2] - p.z;
            const float bx = tri[t][3] - p.x, by = tri[t][4] - p.y, bz = tri[t][5] - p.z;
            const float cx = tri[t][6] - p.x, cy = tri[t][7] - p.y, cz = tri[t][8] - p.z;
            const float la = sqrtf(ax * ax + ay * ay + az * az), lb = sqrtf(bx * bx + by * by + bz * bz),
                        lc = sqrtf(cx * cx + cy * cy + cz * cz);
            const float det = ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx);
            const float den = la * lb * lc + (ax * bx + ay * by + az * bz) * lc + (bx * cx + by * cy + bz * cz) * la +
                              (cx * ax + cy * ay + cz * az) * lb;
            acc += 2.f * atan2f(det, den);
        }
        __syncthreads();
    }
    if (j < nq) partial[(size_t)blockIdx.y * nq + j] = acc;
}

__global__ void k_orient(const float *partial, int ns, double *nrm, float *gap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const int nq = 2 * ns;
    float gi = 0.f, go = 0.f;
    for (int c = 0; c < kGwnChunks; c++) {
        gi += partial[(size_t)c * nq + 2 * i];
        go += partial[(size_t)c * nq + 2 * i + 1];
    }
    const float inv4pi = 0.07957747154594767f;
    gi *= inv4pi;
    go *= inv4pi;
    if (gap) gap[i] = gi - go;
    if (!(gi > go))
        for (int k = 0; k < 3; k++) nrm[3 * i + k] = -nrm[3 * i + k];
}

struct Layout {
    size_t cen, farea, mind, owner, cand_v, cand_i, bar, err, keys, vals, skeys, svals, start, q, partial, sort, total;
    size_t sort_bytes;
};
static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
static Layout layout(int nf, int ns, int nblocks) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o = a256(o + b); return at; };
    L.cen = take(sizeof(double) * 3 * nf);
    L.farea = take(sizeof(double) * nf);
    L.mind = take(sizeof(double) * nf);
    L.owner = take(sizeof(int32_t) * nf);
    L.cand_v = take(sizeof(double) * 2 * nblocks);
    L.cand_i = take(sizeof(int) * 2 * nblocks);
    L.bar = take(sizeof(unsigned) * 2);
    L.err = take(sizeof(int));
    L.keys = take(sizeof(int32_t) * nf);
    L.vals = take(sizeof(int32_t) * nf);
    L.skeys = take(sizeof(int32_t) * nf);
    L.svals = take(sizeof(int32_t) * nf);
    L.start = take(sizeof(int32_t) * (ns + 1));
    L.q = take(sizeof(float4) * 2 * ns);
    L.partial = take(sizeof(float) * kGwnChunks * 2 * ns);
    size_t sb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, sb, (int32_t *)nullptr, (int32_t *)nullptr, (int32_t *)nullptr,
                                    (int32_t *)nullptr, nf, 0, 32);
    L.sort_bytes = sb;
    L.sort = take(sb);
    L.total = o;
    return L;
}

static int fps_blocks() {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fps, 256, 0);
    return num_sms() * std::max(1, std::min(occ, 4));
}

}  // namespace rows
}  // namespace mcs

using namespace mcs;
using namespace mcs::rows;

extern "C" {

size_t mcs_sample_rows_workspace_size(mcs_mesh m, int n) {
    if (!m || n <= 0) return 0;
    return layout(m->nf, n, fps_blocks()).total;
}

mcs_status mcs_sample_rows(mcs_mesh m, int n, int orient, int32_t *sel, double *pos, double *nrm, double *area,
                           int32_t *tri2bin, float *orient_gap, void *workspace, size_t workspace_bytes,
                           void *stream_) {
    MCS_ARG(m != nullptr, "mcs_sample_rows: mesh is NULL");
    MCS_ARG(n >= 1 && n <= m->nf, "mcs_sample_rows: need 1 <= n <= nf");
    MCS_ARG(sel && pos && nrm && area && tri2bin, "mcs_sample_rows: NULL output");
    const int nb = fps_blocks();
    const Layout L = layout(m->nf, n, nb);
    MCS_ARG(workspace && workspace_bytes >= L.total, "mcs_sample_rows: workspace too small");
    MCS_ARG(((uintptr_t)workspace & 255) == 0, "mcs_sample_rows: workspace must be 256-byte aligned");
    int coop = 0, dev = 0;
    MCS_CUDA(cudaGetDevice(&dev));
    MCS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    MCS_ARG(coop, "mcs_sample_rows: the device does not support cooperative launches");
    cudaStream_t st = as_stream(stream_);
    char *w = (char *)workspace;
    double *cen = (double *)(w + L.cen), *farea = (double *)(w + L.farea), *mind = (double *)(w + L.mind);
    int32_t *owner = tri2bin;  // the owner of each face is the output column map
    int *err = (int *)(w + L.err);
    unsigned *bar = (unsigned *)(w + L.bar);
    const int nf = m->nf, tb = 256;
    MCS_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
    MCS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    note_launch();
    k_centroids<<<(nf + tb - 1) / tb, tb, 0, st>>>(m->V, m->F, nf, cen, farea, mind, owner);
    FpsArgs a;
    a.cen = cen; a.mind = mind; a.owner = owner; a.sel = sel;
    a.cand_v = (double *)(w + L.cand_v); a.cand_i = (int *)(w + L.cand_i);
    a.bar = bar; a.err = err; a.nf = nf; a.ns = n;
    void *args[] = {&a};
    note_launch();
    MCS_CUDA(cudaLaunchCooperativeKernel((void *)k_fps, dim3(nb), dim3(256), args, 0, st));
    // quadrature areas: faces sorted (stably) by owner, summed in ascending face order
    int32_t *keys = (int32_t *)(w + L.keys), *vals = (int32_t *)(w + L.vals);
    int32_t *skeys = (int32_t *)(w + L.skeys), *svals = (int32_t *)(w + L.svals);
    int32_t *start = (int32_t *)(w + L.start);
    note_launch();
    k_owner_keys<<<(nf + tb - 1) / tb, tb, 0, st>>>(owner, nf, keys, vals);
    size_t sb = L.sort_bytes;
    MCS_CUDA(cub::DeviceRadixSort::SortPairs(w + L.sort, sb, keys, skeys, vals, svals, nf, 0, 32, st));
    MCS_CUDA(cudaMemsetAsync(start, 0, sizeof(int32_t) * (n + 1), st));
    note_launch();
    k_segments<<<(nf + tb - 1) / tb, tb, 0, st>>>(skeys, nf, n, start);
    note_launch();
    k_sample_rows<<<(n + tb - 1) / tb, tb, 0, st>>>(m->V, m->F, cen, farea, sel, svals, start, n, pos, nrm, area);
    if (orient) {
        float4 *q = (float4 *)(w + L.q);
        float *partial = (float *)(w + L.partial);
        note_launch();
        k_gwn_points<<<(n + tb - 1) / tb, tb, 0, st>>>(pos, nrm, farea, sel, n, q);
        note_launch();
        k_gwn<<<dim3((2 * n + 255) / 256, kGwnChunks), 256, 0, st>>>(m->V, m->F, nf, q, 2 * n, partial);
        note_launch();
        k_orient<<<(n + tb - 1) / tb, tb, 0, st>>>(partial, n, nrm, orient_gap);
    }
    MCS_CUDA(cudaGetLastError());
    int herr = 0;
    MCS_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MCS_CUDA(cudaStreamSynchronize(st));
    if (herr) {
        set_error("mcs_sample_rows: a grid barrier wait timed out");
        return MCS_ERR_DEVICE;
    }
    return MCS_OK;
}

}  // extern "C"
