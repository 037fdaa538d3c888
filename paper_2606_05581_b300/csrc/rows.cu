// rows.cu -- sample rows for the point basis (Sec. 4.4, point-based Galerkin
// basis: points sampled on the surface; farthest-point sampling stands in for
// the paper's blue-noise sampling):
//   FPS        greedy farthest-point sampling over face centroids from face 0,
//              FP32 on the float-rounded centroids: one block (small meshes),
//              one thread-block cluster with a hardware barrier and a
//              distributed-shared-memory exchange per selection (large
//              meshes), or a cooperative grid with a bounded grid barrier
//              (beyond the cluster's shared memory); each face keeps its
//              nearest sample (first selected on ties) -> tri2bin;
//   areas      each sample's quadrature area = area of the faces it owns,
//              summed in ascending face order (stable sort + segments);
//   normals    unit face normal of the sampled face, oriented outward by the
//              generalized winding number of the other faces (App. A item 1):
//              keep n when GWN(x - delta n) > GWN(x + delta n),
//              delta = sqrt(area)/4; FP32 solid angles, summed over the BVH
//              with certified far-field bounds, brute force where the bound
//              does not decide.
#include <cooperative_groups.h>
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "mcs_internal.h"

namespace mcs {
namespace rows {

constexpr int kErrBarrier = 128;

__device__ __forceinline__ uint64_t gtime_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// grid-wide barrier for a cooperative launch: `count` only grows (it starts
// at zero); arrival number a belongs to barrier a / nblocks, which opens once
// the count reaches the end of that barrier's arrivals.  Every wait is
// bounded (~2 s), after which the error word is set and the block carries on.
__device__ void grid_barrier(unsigned *count, unsigned nblocks, int *err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned target = (atomicAdd(count, 1u) / nblocks + 1u) * nblocks;
        volatile unsigned *vc = count;
        const uint64_t t0 = gtime_ns();
        for (unsigned spins = 1; *vc < target; spins++) {
            // the clock is read every 64 polls
            if ((spins & 63) == 0 && gtime_ns() - t0 > 2000000000ull) {
                atomicOr(err, kErrBarrier);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
}

__global__ void k_centroids(const double *V, const int32_t *F, int nf, double *cen, double *farea) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const double *a = V + 3 * F[3 * f], *b = V + 3 * F[3 * f + 1], *c = V + 3 * F[3 * f + 2];
    for (int i = 0; i < 3; i++) cen[3 * f + i] = ((a[i] + b[i]) + c[i]) / 3.0;
    const double ab0 = b[0] - a[0], ab1 = b[1] - a[1], ab2 = b[2] - a[2];
    const double ac0 = c[0] - a[0], ac1 = c[1] - a[1], ac2 = c[2] - a[2];
    const double N0 = ab1 * ac2 - ab2 * ac1, N1 = ab2 * ac0 - ab0 * ac2, N2 = ab0 * ac1 - ab1 * ac0;
    farea[f] = 0.5 * sqrt(N0 * N0 + N1 * N1 + N2 * N2);
}

struct FpsArgs {
    const float *cen;   // float-rounded face centroids (by face id)
    float *cen_s;       // the same in BVH slot order (spatially coherent ranges)
    float *mind;        // squared distance to the nearest sample, by slot
    int32_t *owner;     // nearest sample, by slot
    const int32_t *face;  // face id of each slot
    int32_t *sel;
    float *cand_v;      // 2 x gridDim candidates (double-buffered)
    int *cand_i;
    unsigned *bar;      // barrier arrivals (monotonic)
    int *err;
    int nf, ns;
};

// float-rounded centroids, by face and in slot order; distances start at +inf
__global__ void k_fps_prep(DevMesh m, const double *cen, float *cenf, float *cen_s, float *mind, int32_t *owner,
                           int32_t *face) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m.nf) return;
    const int f = m.t64[s].id;
    for (int k = 0; k < 3; k++) {
        const float c = (float)cen[3 * f + k];
        cen_s[3 * s + k] = c;
        cenf[3 * f + k] = c;
    }
    mind[s] = INFINITY;
    owner[s] = -1;
    face[s] = f;
}
__global__ void k_fps_scatter(int nf, const int32_t *face, const int32_t *owner_s, int32_t *owner) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nf) owner[face[s]] = owner_s[s];
}

__device__ __forceinline__ bool fps_better(float v, int i, float bv, int bi) {
    return v > bv || (v == bv && i < bi);
}

// block-wide argmax of (v, lowest i on ties); every thread gets the result
__device__ void fps_block_max(float &v, int &i, float *rv, int *ri) {
    rv[threadIdx.x] = v;
    ri[threadIdx.x] = i;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s && fps_better(rv[threadIdx.x + s], ri[threadIdx.x + s], rv[threadIdx.x], ri[threadIdx.x])) {
            rv[threadIdx.x] = rv[threadIdx.x + s];
            ri[threadIdx.x] = ri[threadIdx.x + s];
        }
        __syncthreads();
    }
    v = rv[0];
    i = ri[0];
    __syncthreads();
}

constexpr int kFpsThreads = 1024;
constexpr int kFpsSmallFaces = 1 << 18;  // meshes up to this size use the one-block kernel

__device__ __forceinline__ void warp_argmax(float &v, int &i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        const int oi = __shfl_xor_sync(0xFFFFFFFFu, i, o);
        if (fps_better(ov, oi, v, i)) { v = ov; i = oi; }
    }
}

// Greedy farthest-point sampling, sel[0] = face 0, by a cooperative grid of
// kFpsThreads-thread blocks (one per SM at most).  Every warp of the grid
// owns a contiguous range of BVH slots (a compact region of space); after
// each new sample q a warp rescans its range only when q can be nearer than
// the range's largest distance: when the squared distance from q to the
// range's centroid box exceeds that distance (with a relative margin far
// above the float rounding of either), no distance in the range can drop and
// the range keeps its candidate.  The warps' candidates are folded per block,
// the blocks' across the grid after a grid barrier.  The result is the plain
// greedy choice.
__global__ void __launch_bounds__(kFpsThreads) k_fps(FpsArgs a) {
    constexpr int NW = kFpsThreads / 32;
    __shared__ float wv[2][NW];
    __shared__ int wi[2][NW];
    const unsigned nb = gridDim.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = blockIdx.x * NW + w, nw = (int)nb * NW;
    const int chunk = (a.nf + nw - 1) / nw;
    const int s0 = min(a.nf, gw * chunk), s1 = min(a.nf, s0 + chunk);
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int s = s0 + lane; s < s1; s += 32)
        for (int k = 0; k < 3; k++) {
            lo[k] = fminf(lo[k], a.cen_s[3 * s + k]);
            hi[k] = fmaxf(hi[k], a.cen_s[3 * s + k]);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 3; k++) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], o));
        }
    float cv = INFINITY;  // the range's largest distance (its candidate's value)
    int ci = 0x7FFFFFFF;
    int cur = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.sel[0] = 0;
    for (int i = 0; i < a.ns; i++) {
        const float qx = a.cen[3 * cur], qy = a.cen[3 * cur + 1], qz = a.cen[3 * cur + 2];
        const float e0 = fmaxf(fmaxf(lo[0] - qx, 0.0f), qx - hi[0]);
        const float e1 = fmaxf(fmaxf(lo[1] - qy, 0.0f), qy - hi[1]);
        const float e2 = fmaxf(fmaxf(lo[2] - qz, 0.0f), qz - hi[2]);
        const float lb2 = e0 * e0 + e1 * e1 + e2 * e2;
        if (s0 < s1 && !(lb2 * (1.0f - 1e-5f) > cv)) {
            float bv = -1.0f;
            int bi = 0x7FFFFFFF;
            for (int s = s0 + lane; s < s1; s += 32) {
                const float d0 = a.cen_s[3 * s] - qx, d1 = a.cen_s[3 * s + 1] - qy, d2 = a.cen_s[3 * s + 2] - qz;
                const float d = d0 * d0 + d1 * d1 + d2 * d2;
                float md = a.mind[s];
                if (d < md) {
                    md = d;
                    a.mind[s] = d;
                    a.owner[s] = i;
                }
                const int f = a.face[s];
                if (fps_better(md, f, bv, bi)) { bv = md; bi = f; }
            }
            warp_argmax(bv, bi);
            cv = bv;
            ci = bi;
        }
        if (i + 1 == a.ns) break;
        const int par = i & 1;
        if (lane == 0) {
            wv[par][w] = s0 < s1 ? cv : -1.0f;
            wi[par][w] = ci;
        }
        __syncthreads();
        if (w == 0) {
            float v = lane < NW ? wv[par][lane] : -1.0f;
            int idx = lane < NW ? wi[par][lane] : 0x7FFFFFFF;
            warp_argmax(v, idx);
            if (lane == 0) {
                a.cand_v[par * nb + blockIdx.x] = v;
                a.cand_i[par * nb + blockIdx.x] = idx;
            }
        }
        __threadfence();
        grid_barrier(a.bar, nb, a.err);
        // every warp folds the blocks' candidates (any order gives the same winner)
        float v = -1.0f;
        int idx = 0x7FFFFFFF;
        for (unsigned b = lane; b < nb; b += 32) {
            const float ov = __ldcg(a.cand_v + par * nb + b);
            const int oi = __ldcg(a.cand_i + par * nb + b);
            if (fps_better(ov, oi, v, idx)) { v = ov; idx = oi; }
        }
        warp_argmax(v, idx);
        if (blockIdx.x == 0 && threadIdx.x == 0) a.sel[i + 1] = idx;
        cur = idx;
    }
}

// The same greedy sampling by ONE thread-block cluster of kFpsThreads-thread
// CTAs.  CTA k owns a contiguous range of BVH slots, split into sub-ranges of
// kFpsSub slots whose centroid boxes and largest distances (candidates) live
// in its shared memory; after each new sample q a sub-range is rescanned only
// when q can be nearer than its largest distance (the culling test of k_fps,
// at a finer grain).  The CTAs' candidates are exchanged through distributed
// shared memory, one hardware cluster barrier per selection (double-buffered,
// so a CTA never overwrites a candidate another CTA may still be reading).
constexpr int kFpsSub = 128;
constexpr int kFpsClusterMaxSub = 4096;  // sub-ranges per CTA (3 x 16 B each, dynamic shared memory)

// warp-wide argmax of (v, lowest i on ties); the winner's centroid is then
// taken from the lowest lane that holds the winning pair
__device__ __forceinline__ void warp_argmax_xyz(float &v, int &i, float &x, float &y, float &z) {
    const float v0 = v;
    const int i0 = i;
    warp_argmax(v, i);
    const unsigned hold = __ballot_sync(0xFFFFFFFFu, v0 == v && i0 == i);
    const int src = hold ? __ffs(hold) - 1 : 0;
    x = __shfl_sync(0xFFFFFFFFu, x, src);
    y = __shfl_sync(0xFFFFFFFFu, y, src);
    z = __shfl_sync(0xFFFFFFFFu, z, src);
}

__global__ void __launch_bounds__(kFpsThreads) k_fps_cluster(FpsArgs a) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    constexpr int NW = kFpsThreads / 32;
    constexpr int PER_LANE = kFpsSub / 32;
    // per sub-range: lo4 = (box lo, candidate value), hi4 = (box hi, candidate
    // face bits), cc4 = (candidate centroid, -)
    extern __shared__ float4 sub[];
    __shared__ float4 wc[NW];  // warp candidates: centroid, value
    __shared__ int wi[NW];
    // every CTA's candidate, pushed here by that CTA before the cluster
    // barrier (double-buffered by selection parity): the fold after the
    // barrier reads local shared memory only
    __shared__ float4 all_c[2][16];
    __shared__ int all_i[2][16];
    const unsigned rank = cl.block_rank(), ncta = cl.num_blocks();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int per = (a.nf + (int)ncta - 1) / (int)ncta;
    const int s0 = min(a.nf, (int)rank * per), s1 = min(a.nf, s0 + per);
    const int nsub = (s1 - s0 + kFpsSub - 1) / kFpsSub;
    float4 *lo4 = sub, *hi4 = sub + nsub, *cc4 = sub + 2 * nsub;
    // warp w owns sub-ranges w, w + NW, w + 2 NW, ...: neighbouring sub-ranges
    // (the ones a new sample tends to reach together) go to different warps
    const int nown = w < nsub ? (nsub - w + NW - 1) / NW : 0;
    for (int l = 0; l < nown; l++) {
        const int j = w + NW * l;
        const int b0 = s0 + j * kFpsSub, b1 = min(s1, b0 + kFpsSub);
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int s = b0 + lane; s < b1; s += 32)
            for (int k = 0; k < 3; k++) {
                lo[k] = fminf(lo[k], a.cen_s[3 * s + k]);
                hi[k] = fmaxf(hi[k], a.cen_s[3 * s + k]);
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            for (int k = 0; k < 3; k++) {
                lo[k] = fminf(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], o));
                hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], o));
            }
        if (lane == 0) {
            lo4[j] = make_float4(lo[0], lo[1], lo[2], INFINITY);
            hi4[j] = make_float4(hi[0], hi[1], hi[2], __int_as_float(0x7FFFFFFF));
            cc4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncwarp();
    if (rank == 0 && threadIdx.x == 0) a.sel[0] = 0;
    float qx = a.cen[0], qy = a.cen[1], qz = a.cen[2];
    for (int i = 0; i < a.ns; i++) {
        float bv = -1.0f, bx = 0.f, by = 0.f, bz = 0.f;
        int bi = 0x7FFFFFFF;
        for (int r0 = 0; r0 < nown; r0 += 32) {
            const int j = w + NW * (r0 + lane);
            bool need = false;
            if (r0 + lane < nown) {
                const float4 l = lo4[j], h = hi4[j];
                const float e0 = fmaxf(fmaxf(l.x - qx, 0.0f), qx - h.x);
                const float e1 = fmaxf(fmaxf(l.y - qy, 0.0f), qy - h.y);
                const float e2 = fmaxf(fmaxf(l.z - qz, 0.0f), qz - h.z);
                need = !((e0 * e0 + e1 * e1 + e2 * e2) * (1.0f - 1e-5f) > l.w);
            }
            unsigned m = __ballot_sync(0xFFFFFFFFu, need);
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int jb = w + NW * (r0 + b);
                const int b0 = s0 + jb * kFpsSub, b1 = min(s1, b0 + kFpsSub);
                float v = -1.0f, vx = 0.f, vy = 0.f, vz = 0.f;
                int vi = 0x7FFFFFFF;
                // all of the lane's slots at once: their loads are independent
                float cx[PER_LANE], cy[PER_LANE], cz[PER_LANE], md[PER_LANE];
                int fc[PER_LANE];
#pragma unroll
                for (int k = 0; k < PER_LANE; k++) {
                    const int s = b0 + lane + 32 * k;
                    if (s < b1) {
                        cx[k] = a.cen_s[3 * s];
                        cy[k] = a.cen_s[3 * s + 1];
                        cz[k] = a.cen_s[3 * s + 2];
                        md[k] = a.mind[s];
                        fc[k] = a.face[s];
                    }
                }
#pragma unroll
                for (int k = 0; k < PER_LANE; k++) {
                    const int s = b0 + lane + 32 * k;
                    if (s < b1) {
                        const float d0 = cx[k] - qx, d1 = cy[k] - qy, d2 = cz[k] - qz;
                        const float d = d0 * d0 + d1 * d1 + d2 * d2;
                        if (d < md[k]) {
                            md[k] = d;
                            a.mind[s] = d;
                            a.owner[s] = i;
                        }
                        if (fps_better(md[k], fc[k], v, vi)) { v = md[k]; vi = fc[k]; vx = cx[k]; vy = cy[k]; vz = cz[k]; }
                    }
                }
                warp_argmax_xyz(v, vi, vx, vy, vz);
                if (lane == b) {
                    lo4[jb].w = v;
                    hi4[jb].w = __int_as_float(vi);
                    cc4[jb] = make_float4(vx, vy, vz, 0.f);
                }
            }
            __syncwarp();
            if (r0 + lane < nown) {
                const float v = lo4[j].w;
                const int vi = __float_as_int(hi4[j].w);
                if (fps_better(v, vi, bv, bi)) {
                    const float4 c = cc4[j];
                    bv = v; bi = vi; bx = c.x; by = c.y; bz = c.z;
                }
            }
        }
        warp_argmax_xyz(bv, bi, bx, by, bz);
        if (i + 1 == a.ns) break;
        const int par = i & 1;
        if (lane == 0) {
            wc[w] = make_float4(bx, by, bz, bv);
            wi[w] = bi;
        }
        __syncthreads();
        if (w == 0) {
            const float4 c = wc[lane];
            float v = c.w, x = c.x, y = c.y, z = c.z;
            int idx = wi[lane];
            warp_argmax_xyz(v, idx, x, y, z);
            // lane r stores this CTA's candidate into CTA r's slot; the
            // barrier (release on arrive, acquire on wait) orders the stores
            if (lane < (int)ncta) {
                *cl.map_shared_rank(&all_c[par][rank], lane) = make_float4(x, y, z, v);
                *cl.map_shared_rank(&all_i[par][rank], lane) = idx;
            }
        }
        cl.sync();
        // every warp folds the CTAs' candidates (any order gives the same winner)
        float v = -1.0f, x = 0.f, y = 0.f, z = 0.f;
        int idx = 0x7FFFFFFF;
        if (lane < (int)ncta) {
            const float4 c = all_c[par][lane];
            v = c.w; x = c.x; y = c.y; z = c.z;
            idx = all_i[par][lane];
        }
        warp_argmax_xyz(v, idx, x, y, z);
        if (rank == 0 && threadIdx.x == 0) a.sel[i + 1] = idx;
        qx = x; qy = y; qz = z;
    }
    // no CTA leaves while another may still read its shared memory
    cl.sync();
}

// The same greedy sampling by ONE block of kFpsThreads threads (no grid
// barrier): warp w owns a contiguous slot range and skips it when the new
// sample cannot be nearer than the range's largest distance; the warps'
// candidates are folded by every warp from a double-buffered shared array.
__device__ void fps_one_block(const FpsArgs &a) {
    constexpr int NW = kFpsThreads / 32;
    __shared__ float cand_v[2][NW];
    __shared__ int cand_i[2][NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int chunk = (a.nf + NW - 1) / NW;
    const int s0 = min(a.nf, w * chunk), s1 = min(a.nf, s0 + chunk);
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int s = s0 + lane; s < s1; s += 32)
        for (int k = 0; k < 3; k++) {
            lo[k] = fminf(lo[k], a.cen_s[3 * s + k]);
            hi[k] = fmaxf(hi[k], a.cen_s[3 * s + k]);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 3; k++) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], o));
        }
    float cv = INFINITY;
    int ci = 0x7FFFFFFF;
    int cur = 0;
    if (threadIdx.x == 0) a.sel[0] = 0;
    for (int i = 0; i < a.ns; i++) {
        const float qx = a.cen[3 * cur], qy = a.cen[3 * cur + 1], qz = a.cen[3 * cur + 2];
        const float e0 = fmaxf(fmaxf(lo[0] - qx, 0.0f), qx - hi[0]);
        const float e1 = fmaxf(fmaxf(lo[1] - qy, 0.0f), qy - hi[1]);
        const float e2 = fmaxf(fmaxf(lo[2] - qz, 0.0f), qz - hi[2]);
        const float lb2 = e0 * e0 + e1 * e1 + e2 * e2;
        if (s0 < s1 && !(lb2 * (1.0f - 1e-5f) > cv)) {
            float bv = -1.0f;
            int bi = 0x7FFFFFFF;
            for (int s = s0 + lane; s < s1; s += 32) {
                const float d0 = a.cen_s[3 * s] - qx, d1 = a.cen_s[3 * s + 1] - qy, d2 = a.cen_s[3 * s + 2] - qz;
                const float d = d0 * d0 + d1 * d1 + d2 * d2;
                float md = a.mind[s];
                if (d < md) {
                    md = d;
                    a.mind[s] = d;
                    a.owner[s] = i;
                }
                const int f = a.face[s];
                if (fps_better(md, f, bv, bi)) { bv = md; bi = f; }
            }
            warp_argmax(bv, bi);
            cv = bv;
            ci = bi;
        }
        if (i + 1 == a.ns) break;
        const int par = i & 1;
        if (lane == 0) {
            cand_v[par][w] = s0 < s1 ? cv : -1.0f;
            cand_i[par][w] = ci;
        }
        __syncthreads();
        float v = lane < NW ? cand_v[par][lane] : -1.0f;
        int idx = lane < NW ? cand_i[par][lane] : 0x7FFFFFFF;
        warp_argmax(v, idx);
        if (threadIdx.x == 0) a.sel[i + 1] = idx;
        cur = idx;
    }
}
// The same greedy sampling by ONE block with k_fps_cluster's sub-range
// culling: the mesh's slots split into sub-ranges of kFpsSub whose centroid
// boxes and largest distances live in this block's shared memory (`sub`,
// 3 x 16 B per sub-range), warp w owning sub-ranges w, w + NW, ...; after each
// new sample only the sub-ranges it can reach are rescanned, and the warps'
// candidates are folded through double-buffered shared memory.  The choice is
// that of fps_one_block (largest distance, lowest face on ties); the finer
// culling rescans a few sub-ranges per selection instead of whole warp ranges.
__device__ void fps_subrange_block(const FpsArgs &a, float4 *sub) {
    constexpr int NW = kFpsThreads / 32;
    constexpr int PER_LANE = kFpsSub / 32;
    static_assert(NW == 32, "one warp candidate per lane in the fold");
    __shared__ float4 wc[2][NW];
    __shared__ int wi[2][NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int s1 = a.nf;
    const int nsub = (a.nf + kFpsSub - 1) / kFpsSub;
    float4 *lo4 = sub, *hi4 = sub + nsub, *cc4 = sub + 2 * nsub;
    const int nown = w < nsub ? (nsub - w + NW - 1) / NW : 0;
    for (int l = 0; l < nown; l++) {
        const int j = w + NW * l;
        const int b0 = j * kFpsSub, b1 = min(s1, b0 + kFpsSub);
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int s = b0 + lane; s < b1; s += 32)
            for (int k = 0; k < 3; k++) {
                lo[k] = fminf(lo[k], a.cen_s[3 * s + k]);
                hi[k] = fmaxf(hi[k], a.cen_s[3 * s + k]);
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            for (int k = 0; k < 3; k++) {
                lo[k] = fminf(lo[k], __shfl_xor_sync(0xFFFFFFFFu, lo[k], o));
                hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xFFFFFFFFu, hi[k], o));
            }
        if (lane == 0) {
            lo4[j] = make_float4(lo[0], lo[1], lo[2], INFINITY);
            hi4[j] = make_float4(hi[0], hi[1], hi[2], __int_as_float(0x7FFFFFFF));
            cc4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncwarp();
    if (threadIdx.x == 0) a.sel[0] = 0;
    float qx = a.cen[0], qy = a.cen[1], qz = a.cen[2];
    for (int i = 0; i < a.ns; i++) {
        float bv = -1.0f, bx = 0.f, by = 0.f, bz = 0.f;
        int bi = 0x7FFFFFFF;
        for (int r0 = 0; r0 < nown; r0 += 32) {
            const int j = w + NW * (r0 + lane);
            bool need = false;
            if (r0 + lane < nown) {
                const float4 l = lo4[j], h = hi4[j];
                const float e0 = fmaxf(fmaxf(l.x - qx, 0.0f), qx - h.x);
                const float e1 = fmaxf(fmaxf(l.y - qy, 0.0f), qy - h.y);
                const float e2 = fmaxf(fmaxf(l.z - qz, 0.0f), qz - h.z);
                need = !((e0 * e0 + e1 * e1 + e2 * e2) * (1.0f - 1e-5f) > l.w);
            }
            unsigned m = __ballot_sync(0xFFFFFFFFu, need);
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int jb = w + NW * (r0 + b);
                const int b0 = jb * kFpsSub, b1 = min(s1, b0 + kFpsSub);
                float v = -1.0f, vx = 0.f, vy = 0.f, vz = 0.f;
                int vi = 0x7FFFFFFF;
                float cx[PER_LANE], cy[PER_LANE], cz[PER_LANE], md[PER_LANE];
                int fc[PER_LANE];
#pragma unroll
                for (int k = 0; k < PER_LANE; k++) {
                    const int s = b0 + lane + 32 * k;
                    if (s < b1) {
                        cx[k] = a.cen_s[3 * s];
                        cy[k] = a.cen_s[3 * s + 1];
                        cz[k] = a.cen_s[3 * s + 2];
                        md[k] = a.mind[s];
                        fc[k] = a.face[s];
                    }
                }
#pragma unroll
                for (int k = 0; k < PER_LANE; k++) {
                    const int s = b0 + lane + 32 * k;
                    if (s < b1) {
                        const float d0 = cx[k] - qx, d1 = cy[k] - qy, d2 = cz[k] - qz;
                        const float d = d0 * d0 + d1 * d1 + d2 * d2;
                        if (d < md[k]) {
                            md[k] = d;
                            a.mind[s] = d;
                            a.owner[s] = i;
                        }
                        if (fps_better(md[k], fc[k], v, vi)) { v = md[k]; vi = fc[k]; vx = cx[k]; vy = cy[k]; vz = cz[k]; }
                    }
                }
                warp_argmax_xyz(v, vi, vx, vy, vz);
                if (lane == b) {
                    lo4[jb].w = v;
                    hi4[jb].w = __int_as_float(vi);
                    cc4[jb] = make_float4(vx, vy, vz, 0.f);
                }
            }
            __syncwarp();
            if (r0 + lane < nown) {
                const float v = lo4[j].w;
                const int vi = __float_as_int(hi4[j].w);
                if (fps_better(v, vi, bv, bi)) {
                    const float4 c = cc4[j];
                    bv = v; bi = vi; bx = c.x; by = c.y; bz = c.z;
                }
            }
        }
        warp_argmax_xyz(bv, bi, bx, by, bz);
        if (i + 1 == a.ns) break;
        // the block's winner: every warp folds the warps' candidates; the two
        // buffers alternate, so a warp writing the next candidates never
        // overwrites ones another warp may still be reading
        const int par = i & 1;
        if (lane == 0) {
            wc[par][w] = make_float4(bx, by, bz, bv);
            wi[par][w] = bi;
        }
        __syncthreads();
        const float4 c = wc[par][lane];
        float v = c.w, x = c.x, y = c.y, z = c.z;
        int idx = wi[par][lane];
        warp_argmax_xyz(v, idx, x, y, z);
        if (threadIdx.x == 0) a.sel[i + 1] = idx;
        qx = x; qy = y; qz = z;
    }
}

// bytes of dynamic shared memory fps_subrange_block needs for nf faces
static size_t fps_sub_smem(int nf) { return sizeof(float4) * 3 * (size_t)((nf + kFpsSub - 1) / kFpsSub); }

__global__ void __launch_bounds__(kFpsThreads) k_fps_block(FpsArgs a) {
    extern __shared__ float4 fps_sub[];
    fps_subrange_block(a, fps_sub);
}
// many meshes at once: block b samples mesh b
__global__ void __launch_bounds__(kFpsThreads) k_fps_blocks(const FpsArgs *table) {
    extern __shared__ float4 fps_sub[];
    fps_subrange_block(table[blockIdx.x], fps_sub);
}
// the same for batches holding a mesh whose sub-ranges exceed shared memory
__global__ void __launch_bounds__(kFpsThreads) k_fps_blocks_coarse(const FpsArgs *table) {
    fps_one_block(table[blockIdx.x]);
}
// shared memory fps_subrange_block may take (sub-range boxes of up to ~570k faces)
constexpr size_t kFpsSubSmemMax = 212 * 1024;

static mcs_status fps_block_attr(const void *k, size_t smem) {
    MCS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return MCS_OK;
}
constexpr int kFpsChunk = 100;
struct FpsChunk {
    FpsArgs a[kFpsChunk];
    int count, base;
};
__global__ void k_store_fps(FpsChunk c, FpsArgs *table) {
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) table[c.base + i] = c.a[i];
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
__device__ void sample_row(const double *V, const int32_t *F, const double *cen, const double *farea,
                           const int32_t *sel, const int32_t *sfaces, const int32_t *start, int i, double *pos,
                           double *nrm, double *area) {
    // the cell's faces in ascending order, their loads issued 8 at a time
    // ahead of the additions (same summation order)
    double s = 0.0;
    const int e1 = start[i + 1];
    int e = start[i];
    for (; e + 8 <= e1; e += 8) {
        int id[8];
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) id[k] = sfaces[e + k];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = farea[id[k]];
#pragma unroll
        for (int k = 0; k < 8; k++) s += v[k];
    }
    for (; e < e1; e++) s += farea[sfaces[e]];
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
__global__ void k_sample_rows(const double *V, const int32_t *F, const double *cen, const double *farea,
                              const int32_t *sel, const int32_t *sfaces, const int32_t *start, int ns, double *pos,
                              double *nrm, double *area) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ns) sample_row(V, F, cen, farea, sel, sfaces, start, i, pos, nrm, area);
}

// query points x -/+ delta n of every sample (FP32), and the face each excludes
__device__ void gwn_point(const double *pos, const double *nrm, const double *farea, const int32_t *sel, int i,
                          float4 *q) {
    const double delta = 0.25 * sqrt(farea[sel[i]]);
    for (int side = 0; side < 2; side++) {
        const double sg = side == 0 ? -1.0 : 1.0;
        q[2 * i + side] = make_float4((float)(pos[3 * i] + sg * delta * nrm[3 * i]),
                                      (float)(pos[3 * i + 1] + sg * delta * nrm[3 * i + 1]),
                                      (float)(pos[3 * i + 2] + sg * delta * nrm[3 * i + 2]), __int_as_float(sel[i]));
    }
}
__global__ void k_gwn_points(const double *pos, const double *nrm, const double *farea, const int32_t *sel, int ns,
                             float4 *q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ns) gwn_point(pos, nrm, farea, sel, i, q);
}

// the rows (and, with q, the orientation query points) of many meshes in one
// launch: each mesh's launch would wait alone for its largest cell, whose
// area is summed face by face in ascending order
struct RowsJob {
    const double *V, *cen, *farea;
    const int32_t *F, *sel, *sfaces, *start;
    double *pos, *nrm, *area;
    float4 *q;
    int row0;
};
constexpr int kRowsChunk = 40;
struct RowsChunk {
    RowsJob j[kRowsChunk];
    int count, base;
};
__global__ void k_store_rows(RowsChunk c, RowsJob *table) {
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) table[c.base + i] = c.j[i];
}
__global__ void k_rows_batched(const RowsJob *jobs, int count, int total) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo = 0, hi = count - 1;  // the last job whose first row is <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].row0 <= g) lo = mid;
        else hi = mid - 1;
    }
    const RowsJob &J = jobs[lo];
    const int i = g - J.row0;
    sample_row(J.V, J.F, J.cen, J.farea, J.sel, J.sfaces, J.start, i, J.pos, J.nrm, J.area);
    if (J.q) gwn_point(J.pos, J.nrm, J.farea, J.sel, i, J.q);
}

// ---------------------------------------------------------------------------
// Certified hierarchical winding-number orientation.  The decision needs the
// sign of D = sum over the other faces f of Omega_f(x - delta n) -
// Omega_f(x + delta n) (= 4 pi times the GWN gap).  Far BVH nodes enter by
// their dipole term: a node's faces have vector area N = sum (b-a)x(c-a)/2,
// total area A, centre C (area-weighted centroid, clamped into the node's
// box) and radius r (farthest box corner from C); with G(v) = v / |v|^3,
//   Omega_node(p) = N . G(C - p) + R(p),
// and since G = -grad(1/|v|) has third-order derivative tensor norm 6/|v|^4,
// the remainder of the difference between the two query points (2 delta
// apart, both at least d from the box) obeys
//   |R(p-) - R(p+)| <= 2 delta * A * r * 6 / d^4.
// A node is taken by its dipole term when r <= theta d; nearer nodes are
// opened and their faces summed exactly (the brute-force formula).  E adds
// the remainder bounds and a bound on the float rounding of every term; a
// row is decided when |D| > E, since then D has the sign of the exact sum.
// Rows within the bound (and rows whose frontier overflowed) are summed by
// brute force.
// ---------------------------------------------------------------------------
struct __align__(16) GwnAgg {
    float4 na;  // N.x N.y N.z A
    float4 cr;  // C.x C.y C.z r
};
// far-field acceptance r <= theta d, measured: one 2.0M-face union (10,000
// rows) is fastest at 0.1 (0.05: +110 ms, 0.2: +4 ms, 0.3: +80 ms of
// brute-force fallback); 512 meshes of 5k-200k faces in one batched pass at
// 0.2 (0.1: +80 ms, 0.3: +6 ms, 0.5: +60 ms).  The normals are the same at
// every theta: only the share of rows left to brute force moves.
constexpr float kGwnTheta = 0.1f;
constexpr float kGwnThetaBatched = 0.2f;
constexpr double kGwnTreeMin = 268435456.0;  // 2^28 face-row pairs (~2 ms of brute force)
constexpr int kGwnWarps = 4;
constexpr int kGwnStack = 2048;  // frontier entries per warp (shared memory; ~32 x tree depth)
constexpr float kGwnUlp = 5.9604645e-08f;  // 2^-24

__device__ __forceinline__ void tri_moments(const Tri32 &t, float N[3], float &A, float S[3]) {
    N[0] = 0.5f * (t.ab.y * t.ac.z - t.ab.z * t.ac.y);
    N[1] = 0.5f * (t.ab.z * t.ac.x - t.ab.x * t.ac.z);
    N[2] = 0.5f * (t.ab.x * t.ac.y - t.ab.y * t.ac.x);
    A = sqrtf(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    S[0] = A * (t.a.x + (t.ab.x + t.ac.x) * (1.0f / 3.0f));
    S[1] = A * (t.a.y + (t.ab.y + t.ac.y) * (1.0f / 3.0f));
    S[2] = A * (t.a.z + (t.ab.z + t.ac.z) * (1.0f / 3.0f));
}

// node aggregates bottom-up: threads start at the nodes with two leaf
// children; the last internal child to finish continues to the parent
// moments of the internal nodes above internal node i, when both of i's
// children are leaves (the last of each node's two arrivals continues up)
__device__ void gwn_agg_from(const DevMesh &m, const int *child, const int *parent, int *arrive, GwnAgg *agg, int *err,
                             int i) {
    const int ni = m.nf - 1;
    if (i >= ni || child[2 * i] >= 0 || child[2 * i + 1] >= 0) return;
    int p = i;
    for (int level = 0;; level++) {
        if (level > 70) { atomicOr(err, kErrTree); return; }
        float N[3] = {0.f, 0.f, 0.f}, S[3] = {0.f, 0.f, 0.f}, A = 0.f;
        for (int side = 0; side < 2; side++) {
            const int c = child[2 * p + side];
            float n3[3], s3[3], a;
            if (c < 0) {
                tri_moments(m.t32[~c], n3, a, s3);
            } else {
                const float4 na = __ldcg(&agg[c].na), cr = __ldcg(&agg[c].cr);
                n3[0] = na.x; n3[1] = na.y; n3[2] = na.z; a = na.w;
                s3[0] = a * cr.x; s3[1] = a * cr.y; s3[2] = a * cr.z;
            }
            for (int k = 0; k < 3; k++) { N[k] += n3[k]; S[k] += s3[k]; }
            A += a;
        }
        const Node nd = m.nodes[p];
        const float lo[3] = {fminf(nd.a.x, nd.b.z), fminf(nd.a.y, nd.b.w), fminf(nd.a.z, nd.c.x)};
        const float hi[3] = {fmaxf(nd.a.w, nd.c.y), fmaxf(nd.b.x, nd.c.z), fmaxf(nd.b.y, nd.c.w)};
        float C[3], r2 = 0.f;
        for (int k = 0; k < 3; k++) {
            C[k] = A > 0.f ? S[k] / A : 0.5f * (lo[k] + hi[k]);
            C[k] = fminf(fmaxf(C[k], lo[k]), hi[k]);
            const float e = fmaxf(C[k] - lo[k], hi[k] - C[k]);
            r2 += e * e;
        }
        GwnAgg g;
        g.na = make_float4(N[0], N[1], N[2], A);
        g.cr = make_float4(C[0], C[1], C[2], sqrtf(r2) * (1.0f + 1e-6f));
        __stcg(&agg[p].na, g.na);
        __stcg(&agg[p].cr, g.cr);
        __threadfence();
        if (p == 0) return;
        const int q = parent[p];
        if (q < 0 || q >= ni) { atomicOr(err, kErrTree); return; }
        const int need = (child[2 * q] >= 0) + (child[2 * q + 1] >= 0);
        if (need == 2 && atomicAdd(&arrive[q], 1) == 0) return;
        __threadfence();
        p = q;
    }
}
__global__ void k_gwn_agg(DevMesh m, const int *child, const int *parent, int *arrive, GwnAgg *agg, int *err) {
    gwn_agg_from(m, child, parent, arrive, agg, err, blockIdx.x * blockDim.x + threadIdx.x);
}

// solid angle of triangle (a, a + ab, a + ac) seen from p (Van Oosterom &
// Strackee), and a bound on its float rounding
__device__ __forceinline__ float tri_omega(const Tri32 &t, float px, float py, float pz, float &err) {
    const float ax = t.a.x - px, ay = t.a.y - py, az = t.a.z - pz;
    const float bx = ax + t.ab.x, by = ay + t.ab.y, bz = az + t.ab.z;
    const float cx = ax + t.ac.x, cy = ay + t.ac.y, cz = az + t.ac.z;
    const float la = sqrtf(ax * ax + ay * ay + az * az), lb = sqrtf(bx * bx + by * by + bz * bz),
                lc = sqrtf(cx * cx + cy * cy + cz * cz);
    const float det = ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx);
    const float den = la * lb * lc + (ax * bx + ay * by + az * bz) * lc + (bx * cx + by * cy + bz * cz) * la +
                      (cx * ax + cy * ay + cz * az) * lb;
    // det and den carry at most ~16 roundings of size ulp * la lb lc; the
    // angle moves by that over |(det, den)|, atan2f adds a few ulp of pi
    const float mag = sqrtf(det * det + den * den);
    const float l3 = la * lb * lc;
    err = (mag > 1024.f * kGwnUlp * l3) ? (128.f * kGwnUlp) * l3 / mag + 16.f * kGwnUlp : 8.0f;
    return 2.f * atan2f(det, den);
}

// one row's two points summed over the tree by one warp, its frontier in the
// warp's shared stack stk (kGwnStack entries) with the depth in *top
__device__ void gwn_tree_row(const DevMesh &m, const GwnAgg *agg, const float4 *q, int row, float *Dout, float *Eout,
                             int *ovf, int *stk, int *top, float theta) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const float4 qm = q[2 * row], qp = q[2 * row + 1];
    const int excl = __float_as_int(qm.w);
    const float xm = 0.5f * (qm.x + qp.x), ym = 0.5f * (qm.y + qp.y), zm = 0.5f * (qm.z + qp.z);
    const float sx = qp.x - qm.x, sy = qp.y - qm.y, sz = qp.z - qm.z;
    // half the segment, rounded up; every point of the segment lies within it of (xm, ym, zm)
    const float hd = 0.5f * sqrtf(sx * sx + sy * sy + sz * sz) * (1.0f + 1e-5f) + 1e-30f;
    double D = 0.0;  // FP64 running sum: its rounding stays far below E
    float E = 0.f;
    bool over = false;
    if (lane == 0) { stk[0] = 0; *top = 1; }
    __syncwarp();
    for (int guard = 0;; guard++) {
        const int t = *top;
        if (t == 0) break;
        if (guard > 4 * m.nf + 64) { over = true; break; }
        const int take = min(32, t);
        const int node = lane < take ? stk[t - 1 - lane] : -1;
        __syncwarp();
        int push[2] = {-1, -1};
        if (node >= 0) {
            const Node nd = m.nodes[node];
            const float bx[2][6] = {{nd.a.x, nd.a.y, nd.a.z, nd.a.w, nd.b.x, nd.b.y},
                                    {nd.b.z, nd.b.w, nd.c.x, nd.c.y, nd.c.z, nd.c.w}};
            const int ch[2] = {nd.d.x, nd.d.y};
#pragma unroll
            for (int side = 0; side < 2; side++) {
                const int c = ch[side];
                if (c < 0) {
                    const Tri32 tr = m.t32[~c];
                    if (__float_as_int(tr.a.w) == excl) continue;
                    float e1, e2;
                    const float o1 = tri_omega(tr, qm.x, qm.y, qm.z, e1);
                    const float o2 = tri_omega(tr, qp.x, qp.y, qp.z, e2);
                    D += (double)(o1 - o2);
                    E += e1 + e2 + 2.f * kGwnUlp * (fabsf(o1) + fabsf(o2));
                    continue;
                }
                const float dx = fmaxf(fmaxf(bx[side][0] - xm, 0.f), xm - bx[side][3]);
                const float dy = fmaxf(fmaxf(bx[side][1] - ym, 0.f), ym - bx[side][4]);
                const float dz = fmaxf(fmaxf(bx[side][2] - zm, 0.f), zm - bx[side][5]);
                const float d = sqrtf(dx * dx + dy * dy + dz * dz) * (1.0f - 1e-5f) - hd;
                const float4 na = agg[c].na, cr = agg[c].cr;
                if (d > 0.f && cr.w <= theta * d) {
                    const float v1x = cr.x - qm.x, v1y = cr.y - qm.y, v1z = cr.z - qm.z;
                    const float v2x = cr.x - qp.x, v2y = cr.y - qp.y, v2z = cr.z - qp.z;
                    const float i1 = rsqrtf(v1x * v1x + v1y * v1y + v1z * v1z);
                    const float i2 = rsqrtf(v2x * v2x + v2y * v2y + v2z * v2z);
                    const float g1 = i1 * i1 * i1, g2 = i2 * i2 * i2;
                    D += (double)(na.x * (v1x * g1 - v2x * g2) + na.y * (v1y * g1 - v2y * g2) +
                                  na.z * (v1z * g1 - v2z * g2));
                    const float d2 = d * d;
                    const float nn = sqrtf(na.x * na.x + na.y * na.y + na.z * na.z);
                    E += 12.f * hd * na.w * cr.w / (d2 * d2) * (1.0f + 1e-4f) +
                         64.f * kGwnUlp * nn * (i1 * i1 + i2 * i2);
                } else {
                    push[side] = c;
                }
            }
        }
        const int k = (push[0] >= 0) + (push[1] >= 0);
        int incl = k;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        const int base = t - take;
        if (base + total > kGwnStack) { over = true; break; }
        int at = base + incl - k;
        if (push[0] >= 0) stk[at++] = push[0];
        if (push[1] >= 0) stk[at++] = push[1];
        __syncwarp();
        if (lane == 0) *top = base + total;
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        D += __shfl_xor_sync(FULL, D, o);
        E += __shfl_xor_sync(FULL, E, o);
    }
    if (lane == 0) {
        // D rounded to float once; E (a sum of positive terms) rounded up generously
        Dout[row] = (float)D;
        Eout[row] = E * (1.0f + 1e-3f) + 2.f * kGwnUlp * (float)fabs(D);
        ovf[row] = over ? 1 : 0;
    }
}
// rows in the given order (order[i]: the row the i-th warp sums; NULL: 0..n-1)
__global__ void __launch_bounds__(32 * kGwnWarps) k_gwn_tree(DevMesh m, const GwnAgg *agg, const float4 *q, int n,
                                                            float *Dout, float *Eout, int *ovf, const int *order) {
    __shared__ int stk[kGwnWarps][kGwnStack];
    __shared__ int top[kGwnWarps];
    const int w = threadIdx.x >> 5;
    const int g = blockIdx.x * kGwnWarps + w;
    if (g >= n) return;  // warp-uniform
    const int row = order ? order[g] : g;
    gwn_tree_row(m, agg, q, row, Dout, Eout, ovf, stk[w], &top[w], kGwnTheta);
}

// The tree pass of many meshes in two launches (a mesh's 1024 rows alone
// would keep a few warps per SM busy): each mesh is one job; a thread finds
// its job by binary search of the jobs' first internal node (aggregation) or
// first row (sums).
struct GwnJob {
    DevMesh m;
    const int *child, *parent;
    int *arrive, *err, *ovf;
    GwnAgg *agg;
    const float4 *q;
    float *D, *E;
    int n, node0, row0;
};
constexpr int kGwnChunk = 24;
struct GwnChunk {
    GwnJob j[kGwnChunk];
    int count, base;
};
__global__ void k_store_gwn(GwnChunk c, GwnJob *table) {
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) table[c.base + i] = c.j[i];
}
// the last job whose first index (node0 or row0) is <= g
template <bool ROWS>
__device__ __forceinline__ int gwn_job_of(const GwnJob *jobs, int count, int g) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((ROWS ? jobs[mid].row0 : jobs[mid].node0) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__global__ void k_gwn_agg_batched(const GwnJob *jobs, int count, int total_nodes) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total_nodes) return;
    const GwnJob &J = jobs[gwn_job_of<false>(jobs, count, g)];
    gwn_agg_from(J.m, J.child, J.parent, J.arrive, J.agg, J.err, g - J.node0);
}
__global__ void __launch_bounds__(32 * kGwnWarps) k_gwn_tree_batched(const GwnJob *jobs, int count, int total_rows) {
    __shared__ int stk[kGwnWarps][kGwnStack];
    __shared__ int top[kGwnWarps];
    const int w = threadIdx.x >> 5;
    const int g = blockIdx.x * kGwnWarps + w;
    if (g >= total_rows) return;  // warp-uniform
    const GwnJob &J = jobs[gwn_job_of<true>(jobs, count, g)];
    gwn_tree_row(J.m, J.agg, J.q, g - J.row0, J.D, J.E, J.ovf, stk[w], &top[w], kGwnThetaBatched);
}

// decided rows take the sign of D; the rest go to the brute-force list
__device__ __forceinline__ void gwn_decide_row(int i, int force_all, const float *D, const float *E, const int *ovf,
                                               double *nrm, float *gap, int *fb_list, int *fb_count) {
    if (!force_all && !ovf[i] && fabsf(D[i]) > E[i]) {
        if (gap) gap[i] = D[i] * 0.07957747154594767f;
        if (D[i] < 0.f)
            for (int k = 0; k < 3; k++) nrm[3 * i + k] = -nrm[3 * i + k];
        return;
    }
    fb_list[atomicAdd(fb_count, 1)] = i;
}
__global__ void k_gwn_decide(int n, int force_all, const float *D, const float *E, const int *ovf, double *nrm,
                             float *gap, int *fb_list, int *fb_count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) gwn_decide_row(i, force_all, D, E, ovf, nrm, gap, fb_list, fb_count);
}

// brute-force sums of the listed rows; the face range is split into as many
// chunks as fill the grid (at least 16), from the device-side row count
__device__ __forceinline__ int fb_chunks(int cnt, int nf, int grid) {
    const int qg = (2 * cnt + 255) / 256;
    int ch = max(16, (grid + qg - 1) / qg);
    return max(1, min(ch, (nf + 255) / 256));
}
// units u = b, b + grid, ... of one mesh's brute force (grid: the launch's
// x extent, which fixes the chunks and so the summation order)
__device__ void gwn_fb_units(const double *V, const int32_t *F, int nf, const float4 *q, const int *fb_list,
                             const int *fb_count, float *partial, int b, int grid, float (*tri)[9]) {
    const int cnt = *fb_count;
    if (cnt == 0) return;
    const int nq = 2 * cnt, qg = (nq + 255) / 256;
    const int chunks = fb_chunks(cnt, nf, grid);
    const int csize = (nf + chunks - 1) / chunks;
    for (int u = b; u < qg * chunks; u += grid) {
        const int g = u % qg, c = u / qg;
        const int j = g * 256 + threadIdx.x;
        const float4 p = j < nq ? q[2 * fb_list[j >> 1] + (j & 1)] : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        const int excl = __float_as_int(p.w);
        const int f0 = min(nf, c * csize), f1 = min(nf, f0 + csize);
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
            const int nt = min(256, f1 - t0);
            for (int t = 0; t < nt; t++) {
                if (t0 + t == excl) continue;
                const float ax = tri[t][0] - p.x, ay = tri[t][1] - p.y, az = tri[t][2] - p.z;
                const float bx = tri[t][3] - p.x, by = tri[t][4] - p.y, bz = tri[t][5] - p.z;
                const float cx = tri[t][6] - p.x, cy = tri[t][7] - p.y, cz = tri[t][8] - p.z;
                const float la = sqrtf(ax * ax + ay * ay + az * az), lb = sqrtf(bx * bx + by * by + bz * bz),
                            lc = sqrtf(cx * cx + cy * cy + cz * cz);
                const float det = ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx);
                const float den = la * lb * lc + (ax * bx + ay * by + az * bz) * lc +
                                  (bx * cx + by * cy + bz * cz) * la + (cx * ax + cy * ay + cz * az) * lb;
                acc += 2.f * atan2f(det, den);
            }
            __syncthreads();
        }
        if (j < nq) partial[(size_t)c * nq + j] = acc;
    }
}
__global__ void __launch_bounds__(256) k_gwn_fb(const double *V, const int32_t *F, int nf, const float4 *q,
                                                const int *fb_list, const int *fb_count, float *partial) {
    __shared__ float tri[256][9];
    gwn_fb_units(V, F, nf, q, fb_list, fb_count, partial, blockIdx.x, gridDim.x, tri);
}
__device__ void orient_fb_row(int k, const float *partial, int nf, int grid, const int *fb_list, const int *fb_count,
                              double *nrm, float *gap) {
    const int cnt = *fb_count;
    if (k >= cnt) return;
    const int nq = 2 * cnt, chunks = fb_chunks(cnt, nf, grid);
    float gi = 0.f, go = 0.f;
    for (int c = 0; c < chunks; c++) {
        gi += partial[(size_t)c * nq + 2 * k];
        go += partial[(size_t)c * nq + 2 * k + 1];
    }
    const float inv4pi = 0.07957747154594767f;
    gi *= inv4pi;
    go *= inv4pi;
    const int i = fb_list[k];
    if (gap) gap[i] = gi - go;
    if (!(gi > go))
        for (int d = 0; d < 3; d++) nrm[3 * i + d] = -nrm[3 * i + d];
}
__global__ void k_orient_fb(const float *partial, int nf, int grid, const int *fb_list, const int *fb_count,
                            double *nrm, float *gap) {
    orient_fb_row(blockIdx.x * blockDim.x + threadIdx.x, partial, nf, grid, fb_list, fb_count, nrm, gap);
}

// the decisions and brute-force sums of many meshes in one launch each: a
// 2-D grid with the mesh in y, and for the brute force the single-mesh
// launch's x extent, so that every mesh keeps its chunks and summation order
struct OrientJob {
    const double *V;
    const int32_t *F;
    const float4 *q;
    const float *D, *E;
    const int *ovf;
    double *nrm;
    float *gap, *partial;
    int *fb_list, *fb_count;
    int nf, n, force_all;
};
constexpr int kOrientChunk = 36;
struct OrientChunk {
    OrientJob j[kOrientChunk];
    int count, base;
};
__global__ void k_store_orient(OrientChunk c, OrientJob *table) {
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) table[c.base + i] = c.j[i];
}
__global__ void k_zero_fb(const OrientJob *jobs, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) *jobs[i].fb_count = 0;
}
__global__ void k_gwn_decide_batched(const OrientJob *jobs, int count) {
    for (int y = blockIdx.y; y < count; y += gridDim.y) {
        const OrientJob &J = jobs[y];
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i < J.n) gwn_decide_row(i, J.force_all, J.D, J.E, J.ovf, J.nrm, J.gap, J.fb_list, J.fb_count);
    }
}
__global__ void __launch_bounds__(256) k_gwn_fb_batched(const OrientJob *jobs, int count) {
    __shared__ float tri[256][9];
    for (int y = blockIdx.y; y < count; y += gridDim.y) {
        const OrientJob &J = jobs[y];
        gwn_fb_units(J.V, J.F, J.nf, J.q, J.fb_list, J.fb_count, J.partial, blockIdx.x, gridDim.x, tri);
    }
}
__global__ void k_orient_fb_batched(const OrientJob *jobs, int count, int grid) {
    for (int y = blockIdx.y; y < count; y += gridDim.y) {
        const OrientJob &J = jobs[y];
        orient_fb_row(blockIdx.x * blockDim.x + threadIdx.x, J.partial, J.nf, grid, J.fb_list, J.fb_count, J.nrm,
                      J.gap);
    }
}

struct Layout {
    size_t cen, cen_s, cenf, face, farea, mind, owner, cand_v, cand_i, bar, err, keys, vals, skeys, svals, start, q, partial, sort,
        agg, arrive, gD, gE, govf, fb_list, fb_count, total;
    size_t sort_bytes;
};
static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
// brute-force blocks for the undecided rows, and the partial sums they need:
// at most max(16 chunks x 2 ns queries, 256 x (grid + grid/16 + 2)) floats
static int gwn_fb_grid() { return num_sms() * 8; }
static size_t gwn_partial_floats(int ns) {
    const size_t g = (size_t)gwn_fb_grid();
    return std::max((size_t)32 * ns, 256 * (g + g / 16 + 2));
}
static Layout layout(int nf, int ns, int nblocks) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o = a256(o + b); return at; };
    L.cen = take(sizeof(double) * 3 * nf);
    L.cen_s = take(sizeof(float) * 3 * nf);
    L.cenf = take(sizeof(float) * 3 * nf);
    L.face = take(sizeof(int32_t) * nf);
    L.farea = take(sizeof(double) * nf);
    L.mind = take(sizeof(float) * nf);
    L.owner = take(sizeof(int32_t) * nf);
    L.cand_v = take(sizeof(float) * 2 * nblocks);
    L.cand_i = take(sizeof(int) * 2 * nblocks);
    L.bar = take(sizeof(unsigned) * 2);
    L.err = take(sizeof(int));
    L.keys = take(sizeof(int32_t) * nf);
    L.vals = take(sizeof(int32_t) * nf);
    L.skeys = take(sizeof(int32_t) * nf);
    L.svals = take(sizeof(int32_t) * nf);
    L.start = take(sizeof(int32_t) * (ns + 1));
    L.q = take(sizeof(float4) * 2 * ns);
    L.partial = take(sizeof(float) * gwn_partial_floats(ns));
    L.agg = take(sizeof(GwnAgg) * (size_t)std::max(1, nf - 1));
    L.arrive = take(sizeof(int) * (size_t)std::max(1, nf - 1));
    L.gD = take(sizeof(float) * ns);
    L.gE = take(sizeof(float) * ns);
    L.govf = take(sizeof(int) * ns);
    L.fb_list = take(sizeof(int) * ns);
    L.fb_count = take(sizeof(int));
    size_t sb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, sb, (int32_t *)nullptr, (int32_t *)nullptr, (int32_t *)nullptr,
                                    (int32_t *)nullptr, nf, 0, 32);
    L.sort_bytes = sb;
    L.sort = take(sb);
    L.total = o;
    return L;
}

// blocks of the FPS launch: about 16 faces per thread (small meshes keep the
// grid barrier cheap), at most 4 resident blocks per SM
static int fps_blocks(int nf) {
    const int want = (nf + kFpsThreads * 16 - 1) / (kFpsThreads * 16);
    return std::max(1, std::min(num_sms(), want));
}

// cluster FPS: the largest cluster size (16 if the device allows it, else 8)
// that can be resident with this much dynamic shared memory; 0 if neither
static int fps_cluster_size(int nf, size_t *smem_out) {
    for (int cs : {16, 8}) {
        const int per = (nf + cs - 1) / cs;
        const int nsub = (per + kFpsSub - 1) / kFpsSub;
        if (nsub > kFpsClusterMaxSub) continue;
        const size_t smem = sizeof(float4) * 3 * (size_t)nsub;
        if (cs > 8 && cudaFuncSetAttribute(k_fps_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                          cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (cudaFuncSetAttribute(k_fps_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(kFpsThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = cs;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, (void *)k_fps_cluster, &cfg) == cudaSuccess && nc >= 1) {
            *smem_out = smem;
            return cs;
        }
        cudaGetLastError();
    }
    return 0;
}

static mcs_status launch_fps_cluster(const FpsArgs &a, int cs, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kFpsThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = cs;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    note_launch();
    MCS_CUDA(cudaLaunchKernelEx(&cfg, k_fps_cluster, a));
    return MCS_OK;
}

static mcs_status sample_check(const mcs_sample_item &it, const char *fn) {
    const std::string f(fn);
    MCS_ARG(it.mesh != nullptr, f + ": mesh is NULL");
    MCS_ARG(it.n >= 1 && it.n <= it.mesh->nf, f + ": need 1 <= n <= nf");
    MCS_ARG(it.sel && it.pos && it.nrm && it.area && it.tri2bin, f + ": NULL output");
    return MCS_OK;
}

// centroids, areas and the slot-order copies; the FPS arguments of the mesh
static mcs_status sample_prepare(const mcs_sample_item &it, char *w, const Layout &L, int nb, cudaStream_t st,
                                 FpsArgs *out) {
    mcs_mesh m = it.mesh;
    const int nf = m->nf, tb = 256;
    double *cen = (double *)(w + L.cen), *farea = (double *)(w + L.farea);
    float *mind = (float *)(w + L.mind);
    int *err = (int *)(w + L.err);
    unsigned *bar = (unsigned *)(w + L.bar);
    MCS_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
    MCS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    note_launch();
    k_centroids<<<(nf + tb - 1) / tb, tb, 0, st>>>(m->V, m->F, nf, cen, farea);
    float *cen_s = (float *)(w + L.cen_s), *cenf = (float *)(w + L.cenf);
    int32_t *face = (int32_t *)(w + L.face), *owner_s = (int32_t *)(w + L.owner);
    note_launch();
    k_fps_prep<<<(nf + tb - 1) / tb, tb, 0, st>>>(m->dev(), cen, cenf, cen_s, mind, owner_s, face);
    FpsArgs &a = *out;
    a.cen = cenf; a.cen_s = cen_s; a.mind = mind; a.owner = owner_s; a.face = face; a.sel = it.sel;
    a.cand_v = (float *)(w + L.cand_v); a.cand_i = (int *)(w + L.cand_i);
    a.bar = bar; a.err = err; a.nf = nf; a.ns = it.n;
    (void)nb;
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

// Morton code (10 bits per axis in the mesh's box) of each row's two query
// points' midpoint
__device__ __forceinline__ uint32_t spread10_rows(uint32_t x) {
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}
__global__ void k_gwn_row_keys(const float4 *q, int n, float lx, float ly, float lz, float ix, float iy, float iz,
                               uint32_t *keys, int32_t *idx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = q[2 * i], b = q[2 * i + 1];
    const float c[3] = {0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z)};
    const float l[3] = {lx, ly, lz}, v[3] = {ix, iy, iz};
    uint32_t u[3];
    for (int k = 0; k < 3; k++) {
        const float f = fminf(fmaxf((c[k] - l[k]) * v[k], 0.f), 1.f);
        u[k] = (uint32_t)(f * 1023.f);
    }
    keys[i] = spread10_rows(u[0]) | (spread10_rows(u[1]) << 1) | (spread10_rows(u[2]) << 2);
    idx[i] = i;
}

// orientation pieces of sample_finish: the two points of each row, the
// tree pass of one mesh, and the decision (brute force for the rest)
static void orient_points(const mcs_sample_item &it, char *w, const Layout &L, cudaStream_t st) {
    const int tb = 256;
    note_launch();
    k_gwn_points<<<(it.n + tb - 1) / tb, tb, 0, st>>>(it.pos, it.nrm, (double *)(w + L.farea), it.sel, it.n,
                                                       (float4 *)(w + L.q));
}
static mcs_status orient_tree(const mcs_sample_item &it, char *w, const Layout &L, cudaStream_t st) {
    mcs_mesh m = it.mesh;
    const int nf = m->nf, n = it.n, tb = 256;
    GwnAgg *agg = (GwnAgg *)(w + L.agg);
    int *arrive = (int *)(w + L.arrive);
    cudaMemsetAsync(arrive, 0, sizeof(int) * (nf - 1), st);
    note_launch();
    k_gwn_agg<<<(nf - 1 + tb - 1) / tb, tb, 0, st>>>(m->dev(), m->child, m->parent, arrive, agg, (int *)(w + L.err));
    // rows by the Morton code of their points (in the owner sort's arrays, free
    // by now): warps resident together sum nearby rows and share the nodes
    // they open in the caches; each row's sum is unchanged
    const float4 *q = (const float4 *)(w + L.q);
    uint32_t *keys = (uint32_t *)(w + L.keys), *skeys = (uint32_t *)(w + L.skeys);
    int32_t *idx = (int32_t *)(w + L.vals), *order = (int32_t *)(w + L.svals);
    float lo[3], inv[3];
    for (int k = 0; k < 3; k++) {
        lo[k] = (float)m->lo[k];
        inv[k] = (float)(1.0 / (m->hi[k] - m->lo[k]));
    }
    note_launch();
    k_gwn_row_keys<<<(n + tb - 1) / tb, tb, 0, st>>>(q, n, lo[0], lo[1], lo[2], inv[0], inv[1], inv[2], keys, idx);
    size_t sb = L.sort_bytes;
    MCS_CUDA(cub::DeviceRadixSort::SortPairs(w + L.sort, sb, keys, skeys, idx, order, n, 0, 30, st));
    note_launch();
    k_gwn_tree<<<(n + kGwnWarps - 1) / kGwnWarps, 32 * kGwnWarps, 0, st>>>(
        m->dev(), agg, q, n, (float *)(w + L.gD), (float *)(w + L.gE), (int *)(w + L.govf), order);
    return MCS_OK;
}
static void orient_decide(const mcs_sample_item &it, char *w, const Layout &L, cudaStream_t st, bool tree) {
    mcs_mesh m = it.mesh;
    const int nf = m->nf, n = it.n, tb = 256;
    const float4 *q = (const float4 *)(w + L.q);
    float *partial = (float *)(w + L.partial);
    int *fb_list = (int *)(w + L.fb_list), *fb_count = (int *)(w + L.fb_count);
    cudaMemsetAsync(fb_count, 0, sizeof(int), st);
    note_launch();
    k_gwn_decide<<<(n + tb - 1) / tb, tb, 0, st>>>(n, tree ? 0 : 1, (float *)(w + L.gD), (float *)(w + L.gE),
                                                    (int *)(w + L.govf), it.nrm, it.orient_gap, fb_list, fb_count);
    const int grid = gwn_fb_grid();
    note_launch();
    k_gwn_fb<<<grid, 256, 0, st>>>(m->V, m->F, nf, q, fb_list, fb_count, partial);
    note_launch();
    k_orient_fb<<<(n + tb - 1) / tb, tb, 0, st>>>(partial, nf, grid, fb_list, fb_count, it.nrm, it.orient_gap);
}

// owners by face, quadrature areas, row points and normals (+ orientation)
// rows = false leaves the row kernel (k_sample_rows) to the caller's batched launch
static mcs_status sample_finish(const mcs_sample_item &it, int orient, char *w, const Layout &L, cudaStream_t st,
                                bool rows = true) {
    mcs_mesh m = it.mesh;
    const int nf = m->nf, n = it.n, tb = 256;
    double *cen = (double *)(w + L.cen), *farea = (double *)(w + L.farea);
    int32_t *face = (int32_t *)(w + L.face), *owner_s = (int32_t *)(w + L.owner);
    int32_t *owner = it.tri2bin;  // the owner of each face is the output column map
    note_launch();
    k_fps_scatter<<<(nf + tb - 1) / tb, tb, 0, st>>>(nf, face, owner_s, owner);
    // quadrature areas: faces sorted (stably) by owner, summed in ascending face order
    int32_t *keys = (int32_t *)(w + L.keys), *vals = (int32_t *)(w + L.vals);
    int32_t *skeys = (int32_t *)(w + L.skeys), *svals = (int32_t *)(w + L.svals);
    int32_t *start = (int32_t *)(w + L.start);
    note_launch();
    k_owner_keys<<<(nf + tb - 1) / tb, tb, 0, st>>>(owner, nf, keys, vals);
    size_t sb = L.sort_bytes;
    // owners lie in [0, n): radix passes over their bits only (the workspace
    // was sized for all 32, an upper bound)
    const int obits = n > 1 ? 32 - __builtin_clz((unsigned)(n - 1)) : 1;
    MCS_CUDA(cub::DeviceRadixSort::SortPairs(w + L.sort, sb, keys, skeys, vals, svals, nf, 0, obits, st));
    MCS_CUDA(cudaMemsetAsync(start, 0, sizeof(int32_t) * (n + 1), st));
    note_launch();
    k_segments<<<(nf + tb - 1) / tb, tb, 0, st>>>(skeys, nf, n, start);
    if (rows) {
        note_launch();
        k_sample_rows<<<(n + tb - 1) / tb, tb, 0, st>>>(m->V, m->F, cen, farea, it.sel, svals, start, n, it.pos,
                                                        it.nrm, it.area);
    }
    if (orient) {
        // orient 3: hierarchical sums, brute force for the rows within their
        // bound; orient 2: brute force for every row; orient 1: the first
        // when faces x rows reach kGwnTreeMin, else the second (small meshes
        // pay more for the extra launches than for the brute-force sums)
        const bool tree = nf >= 2 && (orient == 3 || (orient == 1 && (double)nf * n >= kGwnTreeMin));
        orient_points(it, w, L, st);
        if (tree) {
            const mcs_status s = orient_tree(it, w, L, st);
            if (s != MCS_OK) return s;
        }
        orient_decide(it, w, L, st, tree);
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

}  // namespace rows
}  // namespace mcs

using namespace mcs;
using namespace mcs::rows;

extern "C" {

size_t mcs_sample_rows_workspace_size(mcs_mesh m, int n) {
    if (!m || n <= 0) return 0;
    return layout(m->nf, n, fps_blocks(m->nf)).total;
}

mcs_status mcs_sample_rows(mcs_mesh m, int n, int orient, int32_t *sel, double *pos, double *nrm, double *area,
                           int32_t *tri2bin, float *orient_gap, void *workspace, size_t workspace_bytes,
                           void *stream_) {
    NvtxRange nvtx_range("mcs_sample_rows");
    mcs_sample_item it;
    it.mesh = m;
    it.n = n;
    it.sel = sel;
    it.pos = pos;
    it.nrm = nrm;
    it.area = area;
    it.tri2bin = tri2bin;
    it.orient_gap = orient_gap;
    mcs_status s = sample_check(it, "mcs_sample_rows");
    if (s != MCS_OK) return s;
    const int nb = fps_blocks(m->nf);
    const Layout L = layout(m->nf, n, nb);
    MCS_ARG(workspace && workspace_bytes >= L.total, "mcs_sample_rows: workspace too small");
    MCS_ARG(((uintptr_t)workspace & 255) == 0, "mcs_sample_rows: workspace must be 256-byte aligned");
    cudaStream_t st = as_stream(stream_);
    char *w = (char *)workspace;
    FpsArgs a;
    if ((s = sample_prepare(it, w, L, nb, st, &a)) != MCS_OK) return s;
    size_t csmem = 0;
    const int cs = m->nf > kFpsSmallFaces ? fps_cluster_size(m->nf, &csmem) : 0;
    if (m->nf <= kFpsSmallFaces) {
        const size_t smem = fps_sub_smem(m->nf);
        if ((s = fps_block_attr((const void *)k_fps_block, smem)) != MCS_OK) return s;
        note_launch();
        k_fps_block<<<1, kFpsThreads, smem, st>>>(a);
    } else if (cs > 0) {
        if ((s = launch_fps_cluster(a, cs, csmem, st)) != MCS_OK) return s;
    } else {
        int coop = 0, dev = 0;
        MCS_CUDA(cudaGetDevice(&dev));
        MCS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        MCS_ARG(coop, "mcs_sample_rows: the device does not support cooperative launches");
        void *args[] = {&a};
        note_launch();
        MCS_CUDA(cudaLaunchCooperativeKernel((void *)k_fps, dim3(nb), dim3(kFpsThreads), args, 0, st));
    }
    if ((s = sample_finish(it, orient, w, L, st)) != MCS_OK) return s;
    int herr = 0;
    MCS_CUDA(cudaMemcpyAsync(&herr, w + L.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MCS_CUDA(cudaStreamSynchronize(st));
    if (herr) {
        set_error((herr & kErrBarrier) ? "mcs_sample_rows: a grid barrier wait timed out"
                                       : "mcs_sample_rows: the BVH aggregate pass exceeded its depth bound");
        return MCS_ERR_DEVICE;
    }
    return MCS_OK;
}

size_t mcs_sample_rows_batched_workspace_size(const mcs_sample_item *items, int count) {
    if (!items || count <= 0) return 0;
    size_t o = a256(sizeof(FpsArgs) * (size_t)count) + a256(sizeof(GwnJob) * (size_t)count) +
               a256(sizeof(RowsJob) * (size_t)count) + a256(sizeof(OrientJob) * (size_t)count);
    for (int i = 0; i < count; i++) {
        if (!items[i].mesh || items[i].n <= 0) return 0;
        o += a256(layout(items[i].mesh->nf, items[i].n, 1).total);
    }
    return o;
}

mcs_status mcs_sample_rows_batched(const mcs_sample_item *items, int count, int orient, void *workspace,
                                   size_t workspace_bytes, void *stream_) {
    NvtxRange nvtx_range("mcs_sample_rows_batched");
    MCS_ARG(items != nullptr && count > 0, "mcs_sample_rows_batched: no items");
    for (int i = 0; i < count; i++) {
        const mcs_status s = sample_check(items[i], "mcs_sample_rows_batched");
        if (s != MCS_OK) return s;
    }
    const size_t need = mcs_sample_rows_batched_workspace_size(items, count);
    MCS_ARG(workspace && workspace_bytes >= need, "mcs_sample_rows_batched: workspace too small");
    MCS_ARG(((uintptr_t)workspace & 255) == 0, "mcs_sample_rows_batched: workspace must be 256-byte aligned");
    cudaStream_t st = as_stream(stream_);
    char *w = (char *)workspace;
    FpsArgs *table = (FpsArgs *)w;
    size_t o = a256(sizeof(FpsArgs) * (size_t)count);
    GwnJob *gtable = (GwnJob *)(w + o);
    o += a256(sizeof(GwnJob) * (size_t)count);
    RowsJob *rtable = (RowsJob *)(w + o);
    o += a256(sizeof(RowsJob) * (size_t)count);
    OrientJob *otable = (OrientJob *)(w + o);
    o += a256(sizeof(OrientJob) * (size_t)count);
    std::vector<FpsArgs> args(count);
    std::vector<Layout> lay(count);
    std::vector<size_t> base(count);
    mcs_status s;
    for (int i = 0; i < count; i++) {
        lay[i] = layout(items[i].mesh->nf, items[i].n, 1);
        base[i] = o;
        o += a256(lay[i].total);
        if ((s = sample_prepare(items[i], w + base[i], lay[i], 1, st, &args[i])) != MCS_OK) return s;
    }
    // every mesh's farthest-point sampling in one launch, one block per mesh
    for (int b0 = 0; b0 < count; b0 += kFpsChunk) {
        FpsChunk c;
        c.count = std::min(kFpsChunk, count - b0);
        c.base = b0;
        for (int i = 0; i < c.count; i++) c.a[i] = args[b0 + i];
        note_launch();
        k_store_fps<<<1, 128, 0, st>>>(c, table);
    }
    size_t smem = 0;
    for (int i = 0; i < count; i++) smem = std::max(smem, fps_sub_smem(items[i].mesh->nf));
    note_launch();
    if (smem <= kFpsSubSmemMax) {
        if ((s = fps_block_attr((const void *)k_fps_blocks, smem)) != MCS_OK) return s;
        k_fps_blocks<<<count, kFpsThreads, smem, st>>>(table);
    } else {
        k_fps_blocks_coarse<<<count, kFpsThreads, 0, st>>>(table);
    }
    for (int i = 0; i < count; i++)
        if ((s = sample_finish(items[i], 0, w + base[i], lay[i], st, false)) != MCS_OK) return s;
    // every mesh's rows (and query points when orienting) in one launch
    {
        std::vector<RowsJob> rj(count);
        int total = 0;
        for (int i = 0; i < count; i++) {
            const Layout &L = lay[i];
            char *wb = w + base[i];
            RowsJob &j = rj[i];
            j.V = items[i].mesh->V;
            j.F = items[i].mesh->F;
            j.cen = (const double *)(wb + L.cen);
            j.farea = (const double *)(wb + L.farea);
            j.sel = items[i].sel;
            j.sfaces = (const int32_t *)(wb + L.svals);
            j.start = (const int32_t *)(wb + L.start);
            j.pos = items[i].pos;
            j.nrm = items[i].nrm;
            j.area = items[i].area;
            j.q = orient ? (float4 *)(wb + L.q) : nullptr;
            j.row0 = total;
            total += items[i].n;
        }
        for (int b0 = 0; b0 < count; b0 += kRowsChunk) {
            RowsChunk c;
            c.count = std::min(kRowsChunk, count - b0);
            c.base = b0;
            for (int k = 0; k < c.count; k++) c.j[k] = rj[b0 + k];
            note_launch();
            k_store_rows<<<1, 128, 0, st>>>(c, rtable);
        }
        note_launch();
        k_rows_batched<<<(total + 255) / 256, 256, 0, st>>>(rtable, count, total);
    }
    if (orient) {
        // the tree pass (orient 3, or orient 1 when the batch's faces x rows
        // reach kGwnTreeMin) for all meshes in two launches, then each mesh's
        // decision and brute force for its undecided rows
        double pairs = 0.0;
        for (int i = 0; i < count; i++) pairs += (double)items[i].mesh->nf * items[i].n;
        const bool tree = orient == 3 || (orient == 1 && pairs >= kGwnTreeMin);
        std::vector<GwnJob> jobs;
        int nodes = 0, nrows = 0;
        for (int i = 0; i < count; i++) {
            mcs_mesh m = items[i].mesh;
            if (!tree || m->nf < 2) continue;
            char *wb = w + base[i];
            const Layout &L = lay[i];
            MCS_CUDA(cudaMemsetAsync(wb + L.arrive, 0, sizeof(int) * (m->nf - 1), st));
            GwnJob j;
            j.m = m->dev();
            j.child = m->child;
            j.parent = m->parent;
            j.arrive = (int *)(wb + L.arrive);
            j.err = (int *)(wb + L.err);
            j.ovf = (int *)(wb + L.govf);
            j.agg = (GwnAgg *)(wb + L.agg);
            j.q = (const float4 *)(wb + L.q);
            j.D = (float *)(wb + L.gD);
            j.E = (float *)(wb + L.gE);
            j.n = items[i].n;
            j.node0 = nodes;
            j.row0 = nrows;
            nodes += m->nf - 1;
            nrows += items[i].n;
            jobs.push_back(j);
        }
        if (!jobs.empty()) {
            const int nj = (int)jobs.size();
            for (int b0 = 0; b0 < nj; b0 += kGwnChunk) {
                GwnChunk c;
                c.count = std::min(kGwnChunk, nj - b0);
                c.base = b0;
                for (int k = 0; k < c.count; k++) c.j[k] = jobs[b0 + k];
                note_launch();
                k_store_gwn<<<1, 128, 0, st>>>(c, gtable);
            }
            note_launch();
            k_gwn_agg_batched<<<(nodes + 255) / 256, 256, 0, st>>>(gtable, nj, nodes);
            note_launch();
            k_gwn_tree_batched<<<(nrows + kGwnWarps - 1) / kGwnWarps, 32 * kGwnWarps, 0, st>>>(gtable, nj, nrows);
        }
        // decisions, brute force for the undecided rows, and their signs:
        // one launch each for all meshes
        std::vector<OrientJob> oj(count);
        int nmax = 0;
        for (int i = 0; i < count; i++) {
            const Layout &L = lay[i];
            char *wb = w + base[i];
            OrientJob &j = oj[i];
            j.V = items[i].mesh->V;
            j.F = items[i].mesh->F;
            j.q = (const float4 *)(wb + L.q);
            j.D = (const float *)(wb + L.gD);
            j.E = (const float *)(wb + L.gE);
            j.ovf = (const int *)(wb + L.govf);
            j.nrm = items[i].nrm;
            j.gap = items[i].orient_gap;
            j.partial = (float *)(wb + L.partial);
            j.fb_list = (int *)(wb + L.fb_list);
            j.fb_count = (int *)(wb + L.fb_count);
            j.nf = items[i].mesh->nf;
            j.n = items[i].n;
            j.force_all = (tree && j.nf >= 2) ? 0 : 1;
            nmax = std::max(nmax, j.n);
        }
        for (int b0 = 0; b0 < count; b0 += kOrientChunk) {
            OrientChunk c;
            c.count = std::min(kOrientChunk, count - b0);
            c.base = b0;
            for (int k = 0; k < c.count; k++) c.j[k] = oj[b0 + k];
            note_launch();
            k_store_orient<<<1, 128, 0, st>>>(c, otable);
        }
        const int gy = std::min(count, 65535), G = gwn_fb_grid();
        const dim3 rgrid((nmax + 255) / 256, gy);
        note_launch();
        k_zero_fb<<<(count + 255) / 256, 256, 0, st>>>(otable, count);
        note_launch();
        k_gwn_decide_batched<<<rgrid, 256, 0, st>>>(otable, count);
        note_launch();
        k_gwn_fb_batched<<<dim3(G, gy), 256, 0, st>>>(otable, count);
        note_launch();
        k_orient_fb_batched<<<rgrid, 256, 0, st>>>(otable, count, G);
    }
    MCS_CUDA(cudaStreamSynchronize(st));
    return MCS_OK;
}

}  // extern "C"
