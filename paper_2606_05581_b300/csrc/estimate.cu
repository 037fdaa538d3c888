// estimate.cu -- the Monte Carlo DtN estimator on the device.
//
//   row schedule   Morton (Z-order) sort of the row points (Sec. 5)
//   tangent balls  bisection on the inward normal (Alg. 2 LargestTangentBall,
//                  Sec. 5: 10 iterations; App. A item 3: radius clamp), FP64
//   exterior frame inversion centre, Kelvin-inverted AABB clamp and the empty
//                  ball at the inverted origin (Sec. 4.3, App. A item 3)
//   walks          persistent kernel: each lane takes walks from a global
//                  queue (warp-aggregated atomics) and steps them one
//                  closest-point query at a time, so a finished lane refills
//                  at once instead of idling behind the warp's longest walk
//   histogram      one block per row: warp-aggregated (__match_any_sync)
//                  shared-memory counts -> padded CSR, fused with the row
//                  normalisation W_vu = omega_v cf_u H_vu / W scattered into
//                  Lambda (the deferred, batched outer products of Sec. 5)
//   assembly       Wsym = (W + W^T)/2 in place by tile pairs, then the
//                  Laplacian diagonal (+ killing measure)
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mcs_internal.h"

namespace mcs {

struct RowBall {
    double c[3];   // empty-ball centre (inverted coordinates for the exterior)
    double n[3];   // pole direction: the row normal (inverted normal for the exterior)
    double rho;    // empty-ball radius
    double M;      // jump mass (1/w0 - 1) / (2 rho)
    double kfac;   // |s~|^3 for exterior rows, 1 otherwise
    double r;      // accepted bisection radius
    int valid;
    int pad;
};

struct Ctrl {
    unsigned long long queue, kqueue;
    unsigned long long steps, capped, lost, kill_steps, kill_capped, kill_lost;
    unsigned long long nodes, tris;
    // first walk that met a query without a triangle: kind (1 interior,
    // 2 exterior), killing flag, walk id, step and query point
    int diag_set, diag_kind, diag_killing, diag_step;
    unsigned long long diag_walk;
    double diag_p[3];
    int err;
    int discarded;
    double origin[3];
    double rmax_ext;
    double rho0max;
    double esc2;   // |x~|^2 beyond which an exterior walk has left the exterior's image
    float origin_f[3], rho0max_f, esc2_f;  // the same, rounded once for FP32 walks
    int argmax_row;
    int pad;
};

struct Frame {
    double onemk, iw0, eps, rho_min_factor, rmax;
    int bisect_iters;
    int start_mode;  // 2: naive rows (the walk starts at s - inset n)
    double inset;
};

__device__ __forceinline__ double dist64(const DevMesh &m, double x, double y, double z, int *err) {
    Hit<double> h;
    closest<double>(m, x, y, z, -1, h, err);
    return sqrt(h.d2);
}

// ---------------------------------------------------------------- row schedule
// Z-order key of row v: 30-bit Morton code of its point in the mesh box, then v
__device__ unsigned long long row_key(const double *pos, int v, double lx, double ly, double lz, double ix, double iy,
                                      double iz) {
    auto q = [](double x, double lo, double inv) {
        const double f = fmin(fmax((x - lo) * inv, 0.0), 1.0);
        return min((uint32_t)(f * 1024.0), 1023u);
    };
    auto spread = [](uint32_t x) {
        x &= 0x3FFu;
        x = (x | (x << 16)) & 0x030000FFu;
        x = (x | (x << 8)) & 0x0300F00Fu;
        x = (x | (x << 4)) & 0x030C30C3u;
        x = (x | (x << 2)) & 0x09249249u;
        return x;
    };
    const uint32_t code = (spread(q(pos[3 * v], lx, ix)) << 2) | (spread(q(pos[3 * v + 1], ly, iy)) << 1) |
                          spread(q(pos[3 * v + 2], lz, iz));
    return ((unsigned long long)code << 32) | (unsigned)v;
}
__global__ void k_row_keys(const double *pos, int R, double lx, double ly, double lz, double ix, double iy, double iz,
                           unsigned long long *keys) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= R) return;
    keys[v] = row_key(pos, v, lx, ly, lz, ix, iy, iz);
}
__global__ void k_order_from_keys(const unsigned long long *keys, int R, int32_t *order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < R) order[i] = (int32_t)(keys[i] & 0xFFFFFFFFull);
}

// ---------------------------------------------------------------- tangent balls
// One warp per row: every query of the row is answered by the whole warp
// (warp_query); a bisection test only asks whether some triangle lies closer
// than (1 - kappa) r, which is the oracle's dist >= (1 - kappa) r decision.
constexpr int kTanWarps = 4;

// Tangent-ball queries are FP64 decisions (the oracle's); an FP32 query on
// the float triangles answers them first whenever it is clear of a band of
// half-width E = 2^-16 (scale + |p|inf) around the threshold -- E bounds the
// float rounding of the point, of the triangle vertices and of the distance
// arithmetic many times over -- and the FP64 query decides the rest.
__device__ __forceinline__ double fp32_band(const DevMesh &m, double x, double y, double z) {
    return 1.52587890625e-05 * ((double)m.scale + fmax(fabs(x), fmax(fabs(y), fabs(z))));
}

// the FP32 warp queries of the tangent balls, one copy each out of line: the
// kernels' hot code then fits the instruction cache better (their top stall
// was instruction fetch; 64-mesh batch setup 30.4 -> 28.0 ms)
__device__ __noinline__ bool wq32_collect(const DevMesh &m, float x, float y, float z, float thr, Hit<float> &h,
                                          int *front, int *err, float lo, int *cand, int *ncand) {
    return warp_query<float, kCollect>(m, x, y, z, thr, h, front, err, lo, cand, ncand);
}
__device__ __noinline__ void wq32_full(const DevMesh &m, float x, float y, float z, Hit<float> &h, int *front, int *err) {
    warp_query<float, kFull>(m, x, y, z, 0.0f, h, front, err);
}

// dist(p) in FP64 (the exact argmin distance): an FP32 query bounds it by
// bound = its distance + 2E.  Every triangle at the FP64 minimum (the
// argmin and its ties) has a float distance below bound + E, so with cand
// given an FP32 pass collects those triangles and they are tested in FP64,
// one per lane, under the FP64 query's (d^2, id) order; otherwise (or when
// more than kCandMax qualify) the FP64 query searches within the bound
__device__ __forceinline__ double wdist(const DevMesh &m, double x, double y, double z, int *front, int *err,
                                        int *cand = nullptr) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    Hit<double> h;
    const float xf = (float)x, yf = (float)y, zf = (float)z;
    double bound = 0.0;
    if (isfinite(xf) && isfinite(yf) && isfinite(zf)) {
        Hit<float> hf;
        wq32_full(m, xf, yf, zf, hf, front, err);
        const double E = fp32_band(m, x, y, z);
        if (hf.slot >= 0 && isfinite(hf.d2)) bound = sqrt((double)hf.d2) + 2.0 * E;
        if (cand && bound > 0.0) {
            int *ncand = cand + kCandMax;
            if (lane == 0) *ncand = 0;
            __syncwarp();
            Hit<float> hc;
            wq32_collect(m, xf, yf, zf, (float)(bound + E), hc, front, err, 0.0f, cand, ncand);
            __syncwarp();
            const int nc = *ncand;
            if (nc >= 1 && nc <= kCandMax) {
                double d2 = INFINITY;
                int id = 0x7FFFFFFF;
                for (int k = lane; k < nc; k += 32) {
                    double b[3];
                    int kid;
                    const double e2 = Slot<double>::test(m, cand[k], x, y, z, b, kid);
                    if (e2 < d2 || (e2 == d2 && kid < id)) { d2 = e2; id = kid; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double od2 = __shfl_xor_sync(FULL, d2, o);
                    const int oid = __shfl_xor_sync(FULL, id, o);
                    if (od2 < d2 || (od2 == d2 && oid < id)) { d2 = od2; id = oid; }
                }
                __syncwarp();
                return sqrt(d2);
            }
            __syncwarp();
        }
    }
    warp_query<double, kFull>(m, x, y, z, bound, h, front, err);
    if (h.slot < 0 && bound > 0.0) warp_query<double, kFull>(m, x, y, z, 0.0, h, front, err);
    return sqrt(h.d2);
}
// dist(p) >= thr, decided as the FP64 query would: an FP32 query stops at the
// first triangle nearer than thr - E (not clear) and otherwise collects the
// triangles whose float distance lies in [thr - E, thr + E); only those can
// be nearer than thr in FP64, and they are tested in FP64, one per lane
__device__ __forceinline__ bool wclear(const DevMesh &m, double x, double y, double z, double thr, int *front,
                                       int *cand, int *err) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const float xf = (float)x, yf = (float)y, zf = (float)z;
    const double E = fp32_band(m, x, y, z);
    if (isfinite(xf) && isfinite(yf) && isfinite(zf) && thr > 2.0 * E) {
        int *ncand = cand + kCandMax;
        if (lane == 0) *ncand = 0;
        __syncwarp();
        Hit<float> hf;
        if (wq32_collect(m, xf, yf, zf, (float)(thr + E), hf, front, err, (float)(thr - E), cand, ncand))
            return false;
        __syncwarp();
        const int nc = *ncand;
        if (nc <= kCandMax) {
            bool below = false;
            for (int k = lane; k < nc; k += 32) {
                double b[3];
                int id;
                below = below || sqrt(Slot<double>::test(m, cand[k], x, y, z, b, id)) < thr;
            }
            const bool any = __any_sync(FULL, below);
            __syncwarp();
            return !any;
        }
    }
    Hit<double> h;
    return !warp_query<double, kBelow>(m, x, y, z, thr, h, front, err);
}

// interior tangent ball of row v, by one warp
__device__ void tangent_int_row(const DevMesh &m, const double *pos, const double *nrm, int v, const Frame &fr,
                                RowBall *ball, Ctrl *ctrl, int *front, int *cand) {
    int err = 0;
    const double s0 = pos[3 * v], s1 = pos[3 * v + 1], s2 = pos[3 * v + 2];
    const double n0 = nrm[3 * v], n1 = nrm[3 * v + 1], n2 = nrm[3 * v + 2];
    const bool nz = (n0 != 0.0 || n1 != 0.0 || n2 != 0.0);
    RowBall b;
    b.c[0] = b.c[1] = b.c[2] = 0.0;
    b.n[0] = n0; b.n[1] = n1; b.n[2] = n2;
    b.rho = 0.0; b.r = 0.0; b.kfac = 1.0;
    if (nz && fr.start_mode == 2) {
        // naive estimator (Alg. 1): the ball of the first walk-on-spheres step
        // from the inset point
        b.c[0] = s0 - fr.inset * n0; b.c[1] = s1 - fr.inset * n1; b.c[2] = s2 - fr.inset * n2;
        b.rho = wdist(m, b.c[0], b.c[1], b.c[2], front, &err, cand);
        b.r = fr.inset;
    } else if (nz) {
        const double rmax = fr.rmax;
        double r;
        if (wclear(m, s0 - rmax * n0, s1 - rmax * n1, s2 - rmax * n2, fr.onemk * rmax, front, cand, &err)) {
            r = rmax;
        } else {
            double lo = 0.0, hi = rmax;
            for (int it = 0; it < fr.bisect_iters; it++) {
                const double mid = 0.5 * (lo + hi);
                if (wclear(m, s0 - mid * n0, s1 - mid * n1, s2 - mid * n2, fr.onemk * mid, front, cand, &err)) lo = mid;
                else hi = mid;
            }
            r = lo;
        }
        b.c[0] = s0 - r * n0; b.c[1] = s1 - r * n1; b.c[2] = s2 - r * n2;
        b.rho = wdist(m, b.c[0], b.c[1], b.c[2], front, &err, cand);
        b.r = r;
    }
    b.valid = nz && (b.rho >= fr.rho_min_factor * fr.eps);
    b.M = b.valid ? (fr.start_mode == 2 ? 1.0 / fr.inset : (fr.iw0 - 1.0) / (2.0 * b.rho)) : 0.0;
    b.pad = 0;
    if ((threadIdx.x & 31) == 0) {
        ball[v] = b;
        if (err) atomicOr(&ctrl->err, err);
    }
}

// rows v = i * stride, i = 0, 1, ... (stride 1: every row)
__global__ void __launch_bounds__(32 * kTanWarps) k_tangent_int(DevMesh m, const double *pos, const double *nrm, int R,
                                                                int stride, Frame fr, RowBall *ball, Ctrl *ctrl) {
    __shared__ int fronts[kTanWarps][32];
    __shared__ int cands[kTanWarps][kCandMax + 1];
    const int v = (blockIdx.x * kTanWarps + (threadIdx.x >> 5)) * stride;
    if (v >= R) return;
    tangent_int_row(m, pos, nrm, v, fr, ball, ctrl, fronts[threadIdx.x >> 5], cands[threadIdx.x >> 5]);
}

// largest empty radius over rows 0, stride, 2 stride, ..., lowest row on ties
// -> inversion centre (any interior point serves; Sec. 4.3)
// one block; sv, si: shared arrays of blockDim.x entries (a power of two)
__device__ void origin_argmax_block(const RowBall *ball, int R, int stride, Ctrl *ctrl, double *sv, int *si) {
    double best = -1.0;
    int bi = 0x7FFFFFFF;
    for (int v = threadIdx.x * stride; v < R; v += blockDim.x * stride) {
        const double r = ball[v].rho;
        if (r > best) { best = r; bi = v; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double o = sv[threadIdx.x + s];
            const int oi = si[threadIdx.x + s];
            if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = o;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int v = si[0];
        ctrl->argmax_row = sv[0] > 0.0 ? v : -1;
        if (!(sv[0] > 0.0)) {
            ctrl->err |= kErrNoOrigin;
            ctrl->origin[0] = ctrl->origin[1] = ctrl->origin[2] = 0.0;
        } else {
            ctrl->origin[0] = ball[v].c[0];
            ctrl->origin[1] = ball[v].c[1];
            ctrl->origin[2] = ball[v].c[2];
        }
    }
}
__global__ void k_origin_argmax(const RowBall *ball, int R, int stride, Ctrl *ctrl) {
    __shared__ double sv[1024];
    __shared__ int si[1024];
    origin_argmax_block(ball, R, stride, ctrl, sv, si);
}
__global__ void k_set_origin(Ctrl *ctrl, double x, double y, double z) {
    ctrl->origin[0] = x; ctrl->origin[1] = y; ctrl->origin[2] = z;
}

// Kelvin-inverted AABB of the vertices (radius clamp), the radius of the
// empty ball at the inverted origin, 1 / max |v - o|, and the escape bound:
// the inversion centre o lies in a bounded component of the complement of
// the surface and B(o, dist(o)) holds no surface point, so no exterior point
// is closer to o than dist(o) and the exterior's image satisfies
// |x~| <= 1 / dist(o); a walk at |x~| > 2 / dist(o) is in o's own component
// (a pocket of a self-overlapping surface) and is retired without a hit
constexpr int kFrameThreads = 256;
// one block of kFrameThreads threads, after the origin is set
// auto_ball: the rows' interior balls when the origin is the centre of the
// ball of ctrl->argmax_row (its empty radius is dist(o)); null otherwise
__device__ void ext_frame_block(const DevMesh &m, const double *V, int nv, Ctrl *ctrl, const RowBall *auto_ball) {
    __shared__ double sm[7][kFrameThreads];
    const double o0 = ctrl->origin[0], o1 = ctrl->origin[1], o2 = ctrl->origin[2];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, mr = 0.0;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        const double d0 = V[3 * v] - o0, d1 = V[3 * v + 1] - o1, d2 = V[3 * v + 2] - o2;
        const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        const double inv = 1.0 / r2;
        const double p[3] = {d0 * inv, d1 * inv, d2 * inv};
        for (int k = 0; k < 3; k++) { mn[k] = fmin(mn[k], p[k]); mx[k] = fmax(mx[k], p[k]); }
        mr = fmax(mr, sqrt(r2));
    }
    for (int k = 0; k < 3; k++) { sm[k][threadIdx.x] = mn[k]; sm[3 + k][threadIdx.x] = mx[k]; }
    sm[6][threadIdx.x] = mr;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int k = 0; k < 3; k++) {
                sm[k][threadIdx.x] = fmin(sm[k][threadIdx.x], sm[k][threadIdx.x + s]);
                sm[3 + k][threadIdx.x] = fmax(sm[3 + k][threadIdx.x], sm[3 + k][threadIdx.x + s]);
            }
            sm[6][threadIdx.x] = fmax(sm[6][threadIdx.x], sm[6][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double side = sm[3][0] - sm[0][0];
        if (sm[4][0] - sm[1][0] < side) side = sm[4][0] - sm[1][0];
        if (sm[5][0] - sm[2][0] < side) side = sm[5][0] - sm[2][0];
        ctrl->rmax_ext = 0.5 * side;
        ctrl->rho0max = 1.0 / sm[6][0];
    }
    // dist(o): the origin ball's empty radius, else by one warp (a single
    // thread would visit every triangle alone when o is equidistant from many
    // of them, as at a sphere's centre)
    __shared__ int front[32];
    if (threadIdx.x < 32) {
        int err = 0;
        const int am = ctrl->argmax_row;
        const double d = auto_ball ? (am >= 0 ? auto_ball[am].rho : 0.0) : wdist(m, o0, o1, o2, front, &err);
        if (threadIdx.x == 0) {
            ctrl->esc2 = d > 0.0 ? 4.0 / (d * d) : INFINITY;
            ctrl->origin_f[0] = (float)o0;
            ctrl->origin_f[1] = (float)o1;
            ctrl->origin_f[2] = (float)o2;
            ctrl->rho0max_f = (float)ctrl->rho0max;
            ctrl->esc2_f = (float)ctrl->esc2;
            if (err) atomicOr(&ctrl->err, err);
        }
    }
}
__global__ void __launch_bounds__(kFrameThreads) k_ext_frame(DevMesh m, const double *V, int nv, Ctrl *ctrl,
                                                            const RowBall *auto_ball) {
    ext_frame_block(m, V, nv, ctrl, auto_ball);
}

// exterior tangent ball: an inverted ball B(c~, r') (not containing 0) is the
// image of the primal ball with centre c~/(|c~|^2 - r'^2) and radius
// r'/(|c~|^2 - r'^2); the accepted ball is replaced by the image of the primal
// empty ball B(C, dist(C)) at the same primal centre, which contains
// B(c~, (1 - kappa) r) and so passes within kappa r of s~
__device__ bool inv_ball_ok(const DevMesh &m, const double st[3], const double nt[3], double r, const double o[3],
                            double onemk, int *front, int *cand, int *err) {
    const double ct0 = st[0] - r * nt[0], ct1 = st[1] - r * nt[1], ct2 = st[2] - r * nt[2];
    const double cc = ct0 * ct0 + ct1 * ct1 + ct2 * ct2;
    // the slack is taken on the inverted radius, where the ball lives: the
    // shrunk ball B(c~, (1 - kappa) r) must be empty.  (On the primal image
    // radius, which grows without bound as the ball nears 0, it would let the
    // ball swallow other components.)
    const double rk = onemk * r;
    const double den = cc - rk * rk;
    // clear of the inversion centre by a margin that keeps the primal image
    // ball (centre ~ 1/den) within FP64 resolution
    if (!(den > 1e-6 * cc)) return false;
    const double inv = 1.0 / den;
    const double C0 = ct0 * inv, C1 = ct1 * inv, C2 = ct2 * inv;
    const double Rp = rk * inv;
    return wclear(m, C0 + o[0], C1 + o[1], C2 + o[2], Rp, front, cand, err);
}

// exterior tangent ball of row v, by one warp
__device__ void tangent_ext_row(const DevMesh &m, const double *pos, const double *nrm, int v, const Frame &fr,
                                RowBall *ball, Ctrl *ctrl, int *front, int *cand) {
    int err = 0;
    const double o[3] = {ctrl->origin[0], ctrl->origin[1], ctrl->origin[2]};
    const double rmax = ctrl->rmax_ext;
    const double n0 = nrm[3 * v], n1 = nrm[3 * v + 1], n2 = nrm[3 * v + 2];
    const bool nz = (n0 != 0.0 || n1 != 0.0 || n2 != 0.0);
    const double sp0 = pos[3 * v] - o[0], sp1 = pos[3 * v + 1] - o[1], sp2 = pos[3 * v + 2] - o[2];
    const double r2s = sp0 * sp0 + sp1 * sp1 + sp2 * sp2;
    const double inv = 1.0 / r2s;
    const double sn = sp0 * n0 + sp1 * n1 + sp2 * n2;
    const double t = (2.0 * sn) * inv;
    const double st[3] = {sp0 * inv, sp1 * inv, sp2 * inv};
    const double nt[3] = {sp0 * t - n0, sp1 * t - n1, sp2 * t - n2};
    RowBall b;
    b.c[0] = b.c[1] = b.c[2] = 0.0;
    b.n[0] = nt[0]; b.n[1] = nt[1]; b.n[2] = nt[2];
    b.rho = 0.0; b.r = 0.0;
    b.kfac = 1.0 / (r2s * sqrt(r2s));
    if (nz) {
        double r;
        if (inv_ball_ok(m, st, nt, rmax, o, fr.onemk, front, cand, &err)) {
            r = rmax;
        } else {
            double lo = 0.0, hi = rmax;
            for (int it = 0; it < fr.bisect_iters; it++) {
                const double mid = 0.5 * (lo + hi);
                if (inv_ball_ok(m, st, nt, mid, o, fr.onemk, front, cand, &err)) lo = mid;
                else hi = mid;
            }
            r = lo;
        }
        b.r = r;
        if (r > 0.0) {
            const double ct0 = st[0] - r * nt[0], ct1 = st[1] - r * nt[1], ct2 = st[2] - r * nt[2];
            const double cc = ct0 * ct0 + ct1 * ct1 + ct2 * ct2;
            const double rk = fr.onemk * r;
            const double den = cc - rk * rk;
            if (den > 1e-6 * cc) {
                const double invd = 1.0 / den;
                const double C0 = ct0 * invd, C1 = ct1 * invd, C2 = ct2 * invd;
                const double D = wdist(m, C0 + o[0], C1 + o[1], C2 + o[2], front, &err, cand);
                const double CC = C0 * C0 + C1 * C1 + C2 * C2;
                const double den2 = CC - D * D;
                // |C|^2 - D^2 cancels when the empty ball nearly reaches the centre
                if (den2 > 1e-8 * CC) {
                    const double inv2 = 1.0 / den2;
                    b.c[0] = C0 * inv2; b.c[1] = C1 * inv2; b.c[2] = C2 * inv2;
                    b.rho = D * inv2;
                }
            }
        }
    }
    b.valid = nz && (b.rho >= fr.rho_min_factor * fr.eps);
    b.M = b.valid ? (fr.iw0 - 1.0) / (2.0 * b.rho) : 0.0;
    b.pad = 0;
    if ((threadIdx.x & 31) == 0) {
        ball[v] = b;
        if (err) atomicOr(&ctrl->err, err);
    }
}

__global__ void __launch_bounds__(32 * kTanWarps) k_tangent_ext(DevMesh m, const double *pos, const double *nrm, int R,
                                                                Frame fr, RowBall *ball, Ctrl *ctrl) {
    __shared__ int fronts[kTanWarps][32];
    __shared__ int cands[kTanWarps][kCandMax + 1];
    const int v = blockIdx.x * kTanWarps + (threadIdx.x >> 5);
    if (v >= R) return;
    tangent_ext_row(m, pos, nrm, v, fr, ball, ctrl, fronts[threadIdx.x >> 5], cands[threadIdx.x >> 5]);
}

// ---------------------------------------------------------------- walks
// One job = the walks of one mesh: its row walks (R x W, in Z-order row
// position order) followed by its killing walks.  A launch serves a table of
// jobs through one global queue; each lane looks its job up on refill.
struct WalkJob {
    DevMesh m;
    const RowBall *ball;
    const int32_t *order;
    const int32_t *tri2bin;
    int32_t *exits;        // R x W, by sorted row position
    int32_t *exit_tri;     // optional, R x W by canonical row
    double *exit_bary;     // optional, R x W x 3 by canonical row: barycentrics of the exit point
    double *walk_w;        // optional, R x W by canonical row: the walk's weight q
    int start_mode;        // 0 importance-sampled ball, 1 uniform ball (weighted), 2 naive inset
    int32_t *H0;           // killing histogram
    Ctrl *ctrl;            // the mesh's control block (origin, Kelvin frame)
    unsigned long long n_rows_walks;  // R * W
    unsigned long long n_kill;        // killing walks after the row walks
    double box_c[3];                  // interior: centre of the vertices' bounding box
    double esc_int2;                  // interior: squared box diagonal (reading R18)
    float box_cf[3], esc_int2f;       // the same, rounded once for FP32 walks
    int R, W;
    uint32_t k0, k1;
    int ext;
    int row_stride;                   // sorted row positions 0, s, 2s, ... (autotuner samples; else 1)
};

struct MultiArgs {
    const WalkJob *jobs;
    const unsigned long long *offs;   // offs[j]: first queue index of job j; offs[n] = total
    int n_jobs;
    unsigned long long *queue;
    Ctrl *stats;                      // counters of the whole launch (with one job: that job's block)
    double eps, iw0;
    float eps2f;
    int max_steps;
    WalkJob j0;                       // the job of a one-job launch (kernel parameter space)
};

// a job constant in the walk's precision (FP32 walks read the copy rounded once)
template <typename T> __device__ __forceinline__ T pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

template <bool MULTI> __device__ __forceinline__ const WalkJob &job_of(const MultiArgs &a, int i) {
    if constexpr (MULTI) return a.jobs[i];
    else return a.j0;
}

__device__ __forceinline__ int exit_bin(const WalkJob &J, int f, double b0, double b1, double b2) {
    if (J.tri2bin) return J.tri2bin[f];
    const int i0 = J.m.F[3 * f], i1 = J.m.F[3 * f + 1], i2 = J.m.F[3 * f + 2];
    int best = 0;
    double bm = b0;
    int im = i0;
    if (b1 > bm || (b1 == bm && i1 < im)) { best = 1; bm = b1; im = i1; }
    if (b2 > bm || (b2 == bm && i2 < im)) { best = 2; bm = b2; im = i2; }
    return best == 0 ? i0 : (best == 1 ? i1 : i2);
}

// FP64 re-check of an FP32 query against the float triangle in `slot`, widened exactly
__device__ __forceinline__ double recheck64(const DevMesh &m, int slot, double x, double y, double z, double *b) {
    const Tri32 t = m.t32[slot];
    return tri_closest<double>(x, y, z, (double)t.a.x, (double)t.a.y, (double)t.a.z, (double)t.ab.x, (double)t.ab.y,
                               (double)t.ab.z, (double)t.ac.x, (double)t.ac.y, (double)t.ac.z, b);
}

__device__ void record_nohit(Ctrl *c, int kind, int killing, unsigned long long g, int step, double x, double y,
                             double z) {
    if (atomicCAS(&c->diag_set, 0, 1) == 0) {
        c->diag_kind = kind;
        c->diag_killing = killing;
        c->diag_walk = g;
        c->diag_step = step;
        c->diag_p[0] = x; c->diag_p[1] = y; c->diag_p[2] = z;
    }
}

template <typename T> struct WalkState {
    V3<T> x;
    unsigned long long g;   // walk id (Philox counter)
    unsigned long long li;  // index within the job
    int k;                  // next step number
    int prev;               // previous closest slot
    int v;                  // canonical row (-1: killing walk)
    int job;
    int kill;
    uint32_t k1;            // Philox key word (killing walks use their own)
};

// MODE: 0 interior jobs only, 1 exterior jobs only, 2 both (the job decides), 3
// one interior job with a start mode of the variance study (mcs_params.start_mode).
// WIDE: closest-point queries on the 4-wide BVH, else on the binary one
// (identical results; the node layout is an autotuner knob).
// FP32 walks are capped at 48 registers for 10 resident blocks per SM: the
// traversal is latency-bound, and the extra warps outweigh the spills
// (measured on the two-sphere exterior workload: 80 registers 300 ms,
// 64: 267 ms, 56: 256 ms, 48: 252 ms, 40: 250-256 ms; identical hit counts).
// TRAV: 0 binary BVH, one lane per query; 1 4-wide BVH, one lane per query;
// 2 4-wide BVH, a group of 4 lanes per query (the group runs one walk, every
// lane holding its state; lane 0 of the group writes results and counters)
// Binary traversal: a round of node visits ends when at most kLeafStop lanes
// can still visit without testing their queued triangles, and the traversal
// stops for service once kServe lanes wait for a decision, a query or a walk;
// with at most kLeafStop live lanes (a launch's tail) queries run to the end
// per lane.  Measured on the two-sphere exterior launch / a 64-mesh batch,
// FP32, against 162 / 666 ms for one whole query per lane and loop pass:
// kServe 8: 169 / 663; 16: 156 / 613; 24: 165 / 641; 28: 178 / 692;
// kLeafStop 0 (every lane queued) 206 / 822 at kServe 8, 4 or 12 no better
// than 8; an L1 prefetch of queued triangles no gain; with the tail rules
// 149 / 568, and with decisions before refills 148 / 550 (kServe 24: 147 /
// 546, slower on short launches; the 2M-face union, whose walks take ~2
// steps: 80 ms per query loop, 86 with refills first, 76); the tree pointer
// held per query rather than read from the job per node: 556 -> 549 on the
// 64-mesh batch
constexpr int kLeafStop = 8;
constexpr int kServe = 16;

template <typename T, int MODE, bool COUNT, bool MULTI, int TRAV>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 4 : 10) k_walks(const __grid_constant__ MultiArgs a) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    constexpr bool GROUP = TRAV == 2;
    const int gr = GROUP ? (lane & 3) : 0;                         // lane within its group
    const unsigned gmask = GROUP ? (0xFu << (lane & ~3)) : (1u << lane);
    const bool writer = gr == 0;                                   // writes results and counts
    const T epsT = sizeof(T) == 8 ? (T)a.eps : (T)a.eps2f;  // FP32: re-check below 2 eps
    WalkState<T> s;
    s.x = V3<T>{(T)0, (T)0, (T)0};
    s.g = 0; s.li = 0; s.k = 1; s.prev = -1; s.v = -1; s.job = 0; s.kill = 0; s.k1 = 0;
    bool active = false, more = true;
    // counters of the lane's current job since its last flush
    long long n_steps = 0, n_ksteps = 0, n_capped = 0, n_kcapped = 0, n_lost = 0;
    int err = 0;
    int cj = -1;
    Work work{0ull, 0ull};
    const unsigned long long total = MULTI ? a.offs[a.n_jobs] : a.j0.n_rows_walks + a.j0.n_kill;
    // with several jobs, a lane adds its counters (and error bits) to a job's
    // block when it leaves that job
    auto flush = [&]() {
        if (cj < 0) return;
        Ctrl *c = job_of<MULTI>(a, cj).ctrl;
        if (n_steps) atomicAdd(&c->steps, (unsigned long long)n_steps);
        if (n_ksteps) atomicAdd(&c->kill_steps, (unsigned long long)n_ksteps);
        if (n_capped) atomicAdd(&c->capped, (unsigned long long)n_capped);
        if (n_kcapped) atomicAdd(&c->kill_capped, (unsigned long long)n_kcapped);
        if (n_lost) atomicAdd(&c->lost, (unsigned long long)n_lost);
        if (err) atomicOr(&c->err, err);
        n_steps = n_ksteps = n_capped = n_kcapped = n_lost = 0;
        err = 0;
    };

    // x <- x + step u with the step's Philox direction
    auto advance = [&](T step, const WalkJob &J) {
        const V3<T> u = direction<T>(J.k0, s.k1, s.g, (uint32_t)s.k);
        s.x.x = s.x.x + step * u.x;
        s.x.y = s.x.y + step * u.y;
        s.x.z = s.x.z + step * u.z;
        s.k++;
    };

    auto finish = [&](const WalkJob &J, int bin, int f, bool capped, bool lost, double b0 = 0.0, double b1 = 0.0,
                      double b2 = 0.0) {
        active = false;
        if (!writer) return;
        if (s.kill) n_kcapped += capped; else n_capped += capped;
        n_lost += lost;
        if (bin >= J.R) { err |= kErrBin; bin = -1; }
        if (s.kill) {
            if (bin >= 0) atomicAdd(&J.H0[bin], 1);
        } else {
            const int rp = (int)(s.li / (unsigned long long)J.W) * J.row_stride, j = (int)(s.li % (unsigned long long)J.W);
            J.exits[(size_t)rp * J.W + j] = bin;
            if (J.exit_tri) J.exit_tri[(size_t)s.v * J.W + j] = f;
            if (J.exit_bary) {
                double *eb = J.exit_bary + ((size_t)s.v * J.W + j) * 3;
                eb[0] = b0; eb[1] = b1; eb[2] = b2;
            }
        }
    };

    // the query point of the walk's next step (exterior: the primal image of
    // x~); false when the walk ended, or stepped, without a query
    auto query_point = [&](const WalkJob &J, bool ext, T &qx, T &qy, T &qz) -> bool {
        qx = s.x.x; qy = s.x.y; qz = s.x.z;
        if (!ext) {
            // farther from the box centre than the box diagonal: the walk is in
            // the unbounded component and is retired without a hit
            const T e0 = s.x.x - pick<T>(J.box_c[0], J.box_cf[0]), e1 = s.x.y - pick<T>(J.box_c[1], J.box_cf[1]),
                    e2 = s.x.z - pick<T>(J.box_c[2], J.box_cf[2]);
            if (e0 * e0 + e1 * e1 + e2 * e2 > pick<T>(J.esc_int2, J.esc_int2f)) {
                finish(J, -1, -1, false, true);
                return false;
            }
        } else {
            const Ctrl &C = *J.ctrl;
            const T r2 = s.x.x * s.x.x + s.x.y * s.x.y + s.x.z * s.x.z;
            if (r2 > pick<T>(C.esc2, C.esc2_f)) { finish(J, -1, -1, false, true); return false; }  // escaped
            if (r2 == (T)0) {
                // the empty ball around the inverted origin; no query
                if (s.k == a.max_steps) { finish(J, -1, -1, true, true); return false; }
                advance(pick<T>(C.rho0max, C.rho0max_f), J);
                return false;
            }
            const T inv = (T)1 / r2;
            qx = s.x.x * inv + pick<T>(C.origin[0], C.origin_f[0]);
            qy = s.x.y * inv + pick<T>(C.origin[1], C.origin_f[1]);
            qz = s.x.z * inv + pick<T>(C.origin[2], C.origin_f[2]);
        }
        return true;
    };

    // after the closest-point query h: the walk exits in the epsilon-shell (or at
    // the step cap), or steps
    auto decide = [&](const WalkJob &J, bool ext, const Hit<T> &h) {
        if (writer) {
            if (s.kill) n_ksteps++; else n_steps++;
        }
        if (h.slot < 0 || h.id < 0 || h.id >= J.m.nf) {
            err |= kErrNoHit;
            if (writer) record_nohit(J.ctrl, ext ? 2 : 1, s.kill, s.g, s.k, (double)s.x.x, (double)s.x.y, (double)s.x.z);
            finish(J, -1, -1, true, true);
            return;
        }
        const T d = rsq<T>(h.d2);
        if (!ext) {
            if (d < epsT || s.k == a.max_steps) {
                if (sizeof(T) == 8) {
                    finish(J, exit_bin(J, h.id, (double)h.b0, (double)h.b1, (double)h.b2), h.id, !(d < epsT), false,
                           (double)h.b0, (double)h.b1, (double)h.b2);
                    return;
                }
                // sample rows without recorded barycentrics need only the
                // decision d64 < eps (the bin is tri2bin[f]); the FP32
                // distance, from the same point to the same float triangle,
                // settles it below a band E of rounding under eps (E bounds
                // the float rounding of the point and the test many times
                // over); inside the band the FP64 re-check decides
                if (J.tri2bin && !J.exit_bary) {
                    const double E = 1.52587890625e-05 * ((double)J.m.scale +
                                                         fmax(fabs((double)s.x.x), fmax(fabs((double)s.x.y), fabs((double)s.x.z))));
                    if ((double)d + E < a.eps) {
                        finish(J, J.tri2bin[h.id], h.id, false, false);
                        return;
                    }
                }
                double b[3];
                const double d64 = sqrt(recheck64(J.m, h.slot, (double)s.x.x, (double)s.x.y, (double)s.x.z, b));
                if (d64 < a.eps || s.k == a.max_steps) {
                    finish(J, exit_bin(J, h.id, b[0], b[1], b[2]), h.id, !(d64 < a.eps), false, b[0], b[1], b[2]);
                    return;
                }
            }
            s.prev = h.slot;
            advance(d, J);
            return;
        }
        // exterior: the step radius in inverted coordinates (reading R7)
        const double r0max64 = J.ctrl->rho0max;
        const T r2 = s.x.x * s.x.x + s.x.y * s.x.y + s.x.z * s.x.z;
        const T inv = (T)1 / r2;
        const T xp0 = s.x.x * inv, xp1 = s.x.y * inv, xp2 = s.x.z * inv;
        const T nx = rsq<T>(xp0 * xp0 + xp1 * xp1 + xp2 * xp2);
        const T ri = d / (nx * (nx + d));
        const T r0 = pick<T>(r0max64, J.ctrl->rho0max_f) - rsq<T>(r2);
        const T rho = ri > r0 ? ri : r0;
        if (rho < epsT || s.k == a.max_steps) {
            if (sizeof(T) == 8) {
                finish(J, exit_bin(J, h.id, (double)h.b0, (double)h.b1, (double)h.b2), h.id, !(rho < epsT), false,
                       (double)h.b0, (double)h.b1, (double)h.b2);
                return;
            }
            const double o64[3] = {J.ctrl->origin[0], J.ctrl->origin[1], J.ctrl->origin[2]};
            const double xd0 = (double)s.x.x, xd1 = (double)s.x.y, xd2 = (double)s.x.z;
            const double r2d = xd0 * xd0 + xd1 * xd1 + xd2 * xd2;
            const double invd = 1.0 / r2d;
            const double xpd0 = xd0 * invd, xpd1 = xd1 * invd, xpd2 = xd2 * invd;
            double b[3];
            const double dd = sqrt(recheck64(J.m, h.slot, xpd0 + o64[0], xpd1 + o64[1], xpd2 + o64[2], b));
            const double nxd = sqrt(xpd0 * xpd0 + xpd1 * xpd1 + xpd2 * xpd2);
            const double rid = dd / (nxd * (nxd + dd));
            const double r0d = r0max64 - sqrt(r2d);
            const double rhod = rid > r0d ? rid : r0d;
            if (rhod < a.eps || s.k == a.max_steps) {
                finish(J, exit_bin(J, h.id, b[0], b[1], b[2]), h.id, !(rhod < a.eps), false, b[0], b[1], b[2]);
                return;
            }
        }
        s.prev = h.slot;
        advance(rho, J);
    };

    // lanes without a walk take the next ones from the global queue
    auto refill = [&]() {
        const bool need = !active && more;
        // groups: one queue entry per group, taken by its lane 0
        const unsigned nm = __ballot_sync(FULL, need && writer);
        if (nm) {
            const int leader = __ffs(nm) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(a.queue, (unsigned long long)__popc(nm));
            base = __shfl_sync(FULL, base, leader);
            unsigned long long wi = base + __popc(nm & ((1u << (lane & ~(GROUP ? 3 : 0))) - 1u));
            if (GROUP) wi = __shfl_sync(FULL, wi, lane & ~3);
            if (need) {
                if (wi >= total) {
                    more = false;
                } else {
                    int lo = 0;
                    if (MULTI) {
                        int hi = a.n_jobs - 1;  // last job with offs <= wi
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (a.offs[mid] <= wi) lo = mid; else hi = mid - 1;
                        }
                    }
                    const WalkJob &J = job_of<MULTI>(a, lo);
                    if (MULTI && lo != cj) { flush(); cj = lo; }
                    s.job = lo;
                    s.li = MULTI ? wi - a.offs[lo] : wi;
                    s.k = 1;
                    s.prev = -1;
                    if (s.li >= J.n_rows_walks) {
                        s.kill = 1;
                        s.k1 = J.k1 ^ kKillKeyXor;
                        s.g = s.li - J.n_rows_walks;
                        s.v = -1;
                        s.x = V3<T>{(T)0, (T)0, (T)0};
                        active = true;
                    } else {
                        s.kill = 0;
                        s.k1 = J.k1;
                        const int rp = (int)(s.li / (unsigned long long)J.W) * J.row_stride,
                                  j = (int)(s.li % (unsigned long long)J.W);
                        const int v = J.order[rp];
                        const RowBall &b = J.ball[v];
                        s.v = v;
                        if (!b.valid) {
                            J.exits[(size_t)rp * J.W + j] = -1;
                            if (J.exit_tri) J.exit_tri[(size_t)v * J.W + j] = -1;
                            if (J.exit_bary) {
                                double *eb = J.exit_bary + ((size_t)v * J.W + j) * 3;
                                eb[0] = eb[1] = eb[2] = 0.0;
                            }
                            if (J.walk_w) J.walk_w[(size_t)v * J.W + j] = 0.0;
                        } else {
                            s.g = (unsigned long long)v * (unsigned long long)J.W + (unsigned long long)j;
                            const unsigned long long gp = s.g - (unsigned long long)(j & 1);
                            if constexpr (MODE == 3) {
                                // interior walks with the variance study's start modes
                                double q = 1.0;
                                s.x = start_point<T>(J.k0, s.k1, gp, j & 1, (T)a.iw0,
                                                     V3<T>{(T)b.c[0], (T)b.c[1], (T)b.c[2]}, (T)b.rho,
                                                     V3<T>{(T)b.n[0], (T)b.n[1], (T)b.n[2]}, J.start_mode, a.iw0,
                                                     &q);
                                if (J.walk_w && writer) J.walk_w[(size_t)v * J.W + j] = q;
                            } else {
                                s.x = start_point<T>(J.k0, s.k1, gp, j & 1, (T)a.iw0,
                                                     V3<T>{(T)b.c[0], (T)b.c[1], (T)b.c[2]}, (T)b.rho,
                                                     V3<T>{(T)b.n[0], (T)b.n[1], (T)b.n[2]});
                                if (J.walk_w && writer) J.walk_w[(size_t)v * J.W + j] = 1.0;
                            }
                            active = true;
                        }
                    }
                }
            }
        }
    };

    if constexpr (TRAV == 0) {
        // Binary BVH: the warp interleaves its lanes' queries.  A lane whose
        // query completes waits (its walk's decision, next query point, or next
        // walk) while the others keep traversing, until kServe lanes wait; the
        // traversal itself alternates node visits with rounds of queued
        // triangle tests (bq_*), so neither the warp's longest query nor a
        // few lanes' triangle tests hold the rest back.
        int qstack[kStackDepth];
        float qsdist[kStackDepth];
        BinQuery<T> q;
        q.nq = 0;
        Hit<T> h;
        int phase = 0;  // 0: the walk needs its next query, 1: query in flight, 2: query complete
        while (true) {
            // service: decisions first, so that a lane whose walk ends takes
            // its next walk (and that walk's first query) in the same round
            if (active && phase == 2) {
                phase = 0;
                const WalkJob &J = job_of<MULTI>(a, s.job);
                decide(J, MODE == 1 || (MODE == 2 && J.ext), h);
            }
            refill();
            if (!__any_sync(FULL, active || more)) break;
            if (active && phase == 0) {
                const WalkJob &J = job_of<MULTI>(a, s.job);
                T qx, qy, qz;
                if (query_point(J, MODE == 1 || (MODE == 2 && J.ext), qx, qy, qz))
                    phase = bq_begin<T, COUNT>(J.m, q, h, qx, qy, qz, s.prev, &work) ? 1 : 2;
            }
            const int live = __popc(__ballot_sync(FULL, active || more));
            if (live <= kLeafStop) {
                // the launch's tail: too few walks to interleave; each query
                // runs to completion (the same visits and tests, per lane)
                if (phase == 1) {
                    const DevMesh &m = job_of<MULTI>(a, s.job).m;
                    do {
                        while (q.nq > 0) bq_flush<T, COUNT>(m, q, h, &work);
                    } while (bq_step<T, COUNT>(q, qstack, qsdist, &err, &work));
                    phase = 2;
                }
                continue;
            }
            while (__any_sync(FULL, phase == 1)) {
                while (true) {
                    if (phase == 1 && q.nq == 0 &&
                        !bq_step<T, COUNT>(q, qstack, qsdist, &err, &work))
                        phase = 2;
                    if (__popc(__ballot_sync(FULL, phase == 1 && q.nq == 0)) <= kLeafStop) break;
                }
                while (__any_sync(FULL, q.nq > 0))
                    if (q.nq > 0) bq_flush<T, COUNT>(job_of<MULTI>(a, s.job).m, q, h, &work);
                // serve at kServe waiting lanes, or at half the live ones once
                // fewer than 2 kServe lanes hold or can take a walk (the
                // launch's tail, where waiting for kServe would stall walks)
                if (__popc(__ballot_sync(FULL, phase != 1 && (active || more))) >= min(kServe, (live + 1) >> 1))
                    break;
            }
        }
    } else {
        while (true) {
            refill();
            if (!__any_sync(FULL, active || more)) break;
            if (!active) continue;
            // ---- one walk-on-spheres step: the query point (exterior: the
            // primal image of x~), the closest-point query, the decision
            const WalkJob &J = job_of<MULTI>(a, s.job);
            const bool ext = MODE == 1 || (MODE == 2 && J.ext);
            T qx, qy, qz;
            if (!query_point(J, ext, qx, qy, qz)) continue;
            Hit<T> h;
            if constexpr (TRAV == 2) closest_g4<T, COUNT>(J.m, qx, qy, qz, s.prev, h, &err, &work, gmask, gr);
            else closest4<T, COUNT>(J.m, qx, qy, qz, s.prev, h, &err, &work);
            decide(J, ext, h);
        }
    }
    if constexpr (MULTI) {
        flush();
        if (COUNT) {
            for (int off = 16; off > 0; off >>= 1) {
                work.nodes += __shfl_down_sync(FULL, work.nodes, off);
                work.tris += __shfl_down_sync(FULL, work.tris, off);
            }
            if (lane == 0) {
                atomicAdd(&a.stats->nodes, work.nodes);
                atomicAdd(&a.stats->tris, work.tris);
            }
        }
    } else {
        // one job (a.stats is its block): per-warp reduction of the counters
        for (int off = 16; off > 0; off >>= 1) {
            n_steps += __shfl_down_sync(FULL, n_steps, off);
            n_ksteps += __shfl_down_sync(FULL, n_ksteps, off);
            n_capped += __shfl_down_sync(FULL, n_capped, off);
            n_kcapped += __shfl_down_sync(FULL, n_kcapped, off);
            n_lost += __shfl_down_sync(FULL, n_lost, off);
            err |= __shfl_down_sync(FULL, err, off);
            if (COUNT) {
                work.nodes += __shfl_down_sync(FULL, work.nodes, off);
                work.tris += __shfl_down_sync(FULL, work.tris, off);
            }
        }
        if (lane == 0) {
            if (COUNT) {
                atomicAdd(&a.stats->nodes, work.nodes);
                atomicAdd(&a.stats->tris, work.tris);
            }
            atomicAdd(&a.stats->steps, (unsigned long long)n_steps);
            atomicAdd(&a.stats->kill_steps, (unsigned long long)n_ksteps);
            atomicAdd(&a.stats->capped, (unsigned long long)n_capped);
            atomicAdd(&a.stats->kill_capped, (unsigned long long)n_kcapped);
            atomicAdd(&a.stats->lost, (unsigned long long)n_lost);
            if (err) atomicOr(&a.stats->err, err);
        }
    }
}

// job tables are written by a kernel (capturable; kernel parameters are copied at launch)
constexpr int kJobChunk = 96;
struct JobChunk {
    WalkJob j[kJobChunk];
    unsigned long long offs[kJobChunk + 1];
    int count, base, last;
};
__global__ void k_store_jobs(JobChunk c, WalkJob *jobs, unsigned long long *offs) {
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) {
        jobs[c.base + i] = c.j[i];
        offs[c.base + i] = c.offs[i];
    }
    if (threadIdx.x == 0 && c.last) offs[c.base + c.count] = c.offs[c.count];
}

// ---------------------------------------------------------------- histogram + assembly
__global__ void k_fill_zero(double *p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = 0.0;
}

__global__ void k_colfactor(const double *pos, int R, const Ctrl *ctrl, double *cf) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= R) return;
    const double d0 = pos[3 * u] - ctrl->origin[0], d1 = pos[3 * u + 1] - ctrl->origin[1],
                 d2 = pos[3 * u + 2] - ctrl->origin[2];
    cf[u] = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

constexpr int kHistThreads = 256;

// one block per sorted row position: shared-memory hit counts of the row's W
// exit bins with warp aggregation, then the row's nonzero bins in ascending
// order -> padded CSR, and W_vu = omega_v cf_u H_vu / W into Lambda
typedef cub::BlockScan<int, kHistThreads> HistScan;

// the histogram of sorted row position rp, by one block of kHistThreads
__device__ void row_histogram(int rp, const int32_t *exits, const int32_t *order, const RowBall *ball,
                              const double *area, const double *cf, int R, int W, int cap, int32_t *hbin,
                              int32_t *hcnt, int32_t *hnnz, double *Lambda, double *omega_out, Ctrl *ctrl, int *hist,
                              typename HistScan::TempStorage &scan_tmp) {
    typedef HistScan Scan;
    const int v = order[rp];
    const RowBall &b = ball[v];
    const double omega = b.valid ? area[v] * b.M * b.kfac : 0.0;
    if (threadIdx.x == 0 && omega_out) omega_out[v] = omega;
    if (!b.valid) {
        if (threadIdx.x == 0) { hnnz[v] = 0; atomicAdd(&ctrl->discarded, 1); }
        return;
    }
    for (int i = threadIdx.x; i < R; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int32_t *ex = exits + (size_t)rp * W;
    const int Wr = (W + 31) & ~31;
    for (int j = threadIdx.x; j < Wr; j += blockDim.x) {
        const int bin = j < W ? ex[j] : -1;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, bin);
        if (bin >= 0 && bin < R && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
    }
    __syncthreads();
    const int chunk = (R + blockDim.x - 1) / blockDim.x;
    const int lo = min(R, (int)threadIdx.x * chunk), hi = min(R, lo + chunk);
    int cnt = 0;
    for (int u = lo; u < hi; u++) cnt += hist[u] != 0;
    int off, total;
    Scan(scan_tmp).ExclusiveSum(cnt, off, total);
    int32_t *ob = hbin + (size_t)v * cap, *oc = hcnt + (size_t)v * cap;
    double *Lrow = Lambda ? Lambda + (size_t)v * R : nullptr;
    for (int u = lo; u < hi; u++) {
        const int h = hist[u];
        if (h) {
            ob[off] = u;
            oc[off] = h;
            off++;
            if (Lrow) Lrow[u] = ((omega * (double)h) / (double)W) * (cf ? cf[u] : 1.0);
        }
    }
    if (threadIdx.x == 0) hnnz[v] = total;
}

__global__ void __launch_bounds__(kHistThreads) k_histogram(const int32_t *exits, const int32_t *order,
                                                           const RowBall *ball, const double *area, const double *cf,
                                                           int R, int W, int cap, int32_t *hbin, int32_t *hcnt,
                                                           int32_t *hnnz, double *Lambda, double *omega_out,
                                                           Ctrl *ctrl) {
    extern __shared__ int hist[];
    __shared__ typename HistScan::TempStorage scan_tmp;
    row_histogram(blockIdx.x, exits, order, ball, area, cf, R, W, cap, hbin, hcnt, hnnz, Lambda, omega_out, ctrl,
                  hist, scan_tmp);
}

// Rows beyond the shared-memory histogram (R ints per block): the row's W exit
// bins are radix-sorted within the block (keys bin + 1; bin -1, no exit, is 0;
// padding 2^end_bit - 1 > R), then every run of equal valid keys is one
// (bin, count) pair.  A run's first item writes its bin and index into the
// row's own CSR slots, its last item (after a barrier) turns the index into the
// count: no array of R or W entries in shared memory.  Bins ascend and the
// counts, omega and Lambda entries are those of row_histogram.
constexpr int kHistDenseMaxRows = 51200;
template <int ITEMS>
__global__ void __launch_bounds__(kHistThreads) k_histogram_sorted(const int32_t *exits, const int32_t *order,
                                                                  const RowBall *ball, const double *area,
                                                                  const double *cf, int R, int W, int cap,
                                                                  int32_t *hbin, int32_t *hcnt, int32_t *hnnz,
                                                                  double *Lambda, double *omega_out, Ctrl *ctrl,
                                                                  int end_bit) {
    typedef cub::BlockRadixSort<unsigned, kHistThreads, ITEMS> Sort;
    __shared__ union {
        typename Sort::TempStorage sort;
        typename HistScan::TempStorage scan;
    } tmp;
    __shared__ unsigned first_s[kHistThreads], last_s[kHistThreads];
    const int t = threadIdx.x, rp = blockIdx.x;
    const int v = order[rp];
    const RowBall &b = ball[v];
    const double omega = b.valid ? area[v] * b.M * b.kfac : 0.0;
    if (t == 0 && omega_out) omega_out[v] = omega;
    if (!b.valid) {
        if (t == 0) { hnnz[v] = 0; atomicAdd(&ctrl->discarded, 1); }
        return;
    }
    const int32_t *ex = exits + (size_t)rp * W;
    const unsigned pad = (1u << end_bit) - 1u;
    unsigned key[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        const int j = k * kHistThreads + t;  // any arrangement: the sort orders them
        key[k] = j < W ? (unsigned)(ex[j] + 1) : pad;
    }
    Sort(tmp.sort).Sort(key, 0, end_bit);  // blocked: thread t holds sorted items t * ITEMS + k
    first_s[t] = key[0];
    last_s[t] = key[ITEMS - 1];
    __syncthreads();
    const unsigned prev = t > 0 ? last_s[t - 1] : 0u, next = t + 1 < kHistThreads ? first_s[t + 1] : 0u;
    unsigned st = 0, en = 0;  // run starts / ends among this thread's items (bit k)
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        const bool valid = key[k] >= 1u && key[k] <= (unsigned)R;
        const unsigned p = k > 0 ? key[k - 1] : prev, n = k + 1 < ITEMS ? key[k + 1] : next;
        if (valid && key[k] != p) st |= 1u << k;
        if (valid && key[k] != n) en |= 1u << k;
    }
    int sbase, total, ebase;
    HistScan(tmp.scan).ExclusiveSum(__popc(st), sbase, total);
    __syncthreads();
    HistScan(tmp.scan).ExclusiveSum(__popc(en), ebase);
    int32_t *ob = hbin + (size_t)v * cap, *oc = hcnt + (size_t)v * cap;
#pragma unroll
    for (int k = 0; k < ITEMS; k++)
        if (st >> k & 1u) {
            ob[sbase] = (int32_t)key[k] - 1;
            oc[sbase] = t * ITEMS + k;
            sbase++;
        }
    __syncthreads();
    double *Lrow = Lambda ? Lambda + (size_t)v * R : nullptr;
#pragma unroll
    for (int k = 0; k < ITEMS; k++)
        if (en >> k & 1u) {
            const int h = t * ITEMS + k - oc[ebase] + 1;
            oc[ebase] = h;
            const int u = (int)key[k] - 1;
            if (Lrow) Lrow[u] = ((omega * (double)h) / (double)W) * (cf ? cf[u] : 1.0);
            ebase++;
        }
    if (t == 0) hnnz[v] = total;
}
// exits per row the sorted histogram takes (kHistThreads x 32 items)
constexpr int kHistSortMaxW = kHistThreads * 32;

// Lambda <- -(D + D^T)/2 off the diagonal, by 32 x 32 tile pairs (I <= J);
// one block of 32 x 8 threads per pair
__device__ void symmetrize_tiles(double *L, int R, int I, int J, double (*A)[33], double (*B)[33]) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += blockDim.y) {
        const int gi = I * 32 + r, gj = J * 32 + tx;
        A[r][tx] = (gi < R && gj < R) ? L[(size_t)gi * R + gj] : 0.0;
        const int hi = J * 32 + r, hj = I * 32 + tx;
        B[r][tx] = (hi < R && hj < R) ? L[(size_t)hi * R + hj] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += blockDim.y) {
        const int gi = I * 32 + r, gj = J * 32 + tx;
        if (gi < R && gj < R) {
            const double s = gi == gj ? 0.0 : -(0.5 * (A[r][tx] + B[tx][r]));
            L[(size_t)gi * R + gj] = s;
        }
    }
    if (I == J) return;
    __syncthreads();
    for (int r = ty; r < 32; r += blockDim.y) {
        const int hi = J * 32 + r, hj = I * 32 + tx;
        if (hi < R && hj < R) L[(size_t)hi * R + hj] = -(0.5 * (A[tx][r] + B[r][tx]));
    }
}
__global__ void k_symmetrize(double *L, int R) {
    __shared__ double A[32][33], B[32][33];
    const int I = blockIdx.y, J = blockIdx.x;
    if (I > J) return;
    symmetrize_tiles(L, R, I, J, A, B);
}

// Laplacian diagonal of row `warp`, by one warp:
// Lambda_vv = sum_{u != v} Wsym_vu (+ killing 4 pi cf_v H0_v / N0)
__device__ void diagonal_row(double *L, int R, int warp, const double *cf, const int32_t *H0, double inv_n0) {
    const int lane = threadIdx.x & 31;
    const double *row = L + (size_t)warp * R;
    double s = 0.0;
    for (int u = lane; u < R; u += 32) s += row[u];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, off);
    if (lane == 0) {
        double d = -s;  // row[warp] is 0 here
        if (H0) d += ((4.0 * M_PI * (cf ? cf[warp] : 1.0)) * (double)H0[warp]) * inv_n0;
        L[(size_t)warp * R + warp] = d;
    }
}
__global__ void k_to_f32(const double *L, size_t n, float *out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)L[i];
}
__global__ void k_diagonal(double *L, int R, const double *cf, const int32_t *H0, double inv_n0) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= R) return;
    diagonal_row(L, R, warp, cf, H0, inv_n0);
}

// ---------------------------------------------------------------- batched setup and finish
// Every mesh of a batch, as the batched setup and finishing kernels see it.
// Units of work are numbered across the batch; a kernel finds its mesh by a
// binary search of the per-mesh offsets, so one launch serves all meshes.
struct MeshJob {
    DevMesh m;
    const double *pos, *nrm, *area, *V;
    RowBall *ball;
    Ctrl *ctrl;
    int32_t *order, *exits, *H0;
    double *cf;                 // exterior column factors, else null
    int32_t *hbin, *hcnt, *hnnz;
    double *Lambda, *omega;
    float *Lambda32;
    Frame fr;
    double lo[3], inv[3];       // box frame of the row keys
    double origin[3];           // exterior, origin_auto == 0
    double inv_n0;              // 1 / N0 with killing walks, else 0
    int R, W, cap, nv;
    int ext, origin_auto, ostride, kill;
};

// last j with offs[j] <= g (offs ascending, offs[0] = 0)
__device__ __forceinline__ int find_job(const int *offs, int n, int g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kMeshChunk = 40;
struct MeshChunk {
    MeshJob j[kMeshChunk];
    int count, base;
};
__global__ void k_store_mesh_jobs(MeshChunk c, MeshJob *jobs) {
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) jobs[c.base + i] = c.j[i];
}
constexpr int kIntChunk = 2048;
struct IntChunk {
    int v[kIntChunk];
    int count, base;
};
__global__ void k_store_ints(IntChunk c, int *out) {
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) out[c.base + i] = c.v[i];
}

// zero H0; the Z-order key of every row (or the caller's order)
__global__ void k_b_rows(const MeshJob *jobs, const int *row0, int n, int identity, unsigned long long *keys) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= row0[n]) return;
    const int j = find_job(row0, n, g);
    const MeshJob &J = jobs[j];
    const int v = g - row0[j];
    J.H0[v] = 0;
    if (identity) J.order[v] = v;
    else keys[g] = row_key(J.pos, v, J.lo[0], J.lo[1], J.lo[2], J.inv[0], J.inv[1], J.inv[2]);
}
__global__ void k_b_order(const MeshJob *jobs, const int *row0, int n, const unsigned long long *keys_s) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= row0[n]) return;
    const int j = find_job(row0, n, g);
    jobs[j].order[g - row0[j]] = (int32_t)(keys_s[g] & 0xFFFFFFFFull);
}

// interior tangent balls: every row of interior meshes, the strided subset of
// exterior meshes with an automatic inversion centre; one warp per row
__global__ void __launch_bounds__(32 * kTanWarps) k_b_tangent_int(const MeshJob *jobs, const int *unit0, int n) {
    __shared__ int fronts[kTanWarps][32];
    __shared__ int cands[kTanWarps][kCandMax + 1];
    const int u = blockIdx.x * kTanWarps + (threadIdx.x >> 5);
    if (u >= unit0[n]) return;
    const int j = find_job(unit0, n, u);
    const MeshJob &J = jobs[j];
    const int v = (u - unit0[j]) * (J.ext ? J.ostride : 1);
    tangent_int_row(J.m, J.pos, J.nrm, v, J.fr, J.ball, J.ctrl, fronts[threadIdx.x >> 5], cands[threadIdx.x >> 5]);
}
// exterior meshes: inversion centre and inverted frame, one block each
__global__ void __launch_bounds__(kFrameThreads) k_b_frame(const MeshJob *jobs) {
    __shared__ double sv[kFrameThreads];
    __shared__ int si[kFrameThreads];
    const MeshJob &J = jobs[blockIdx.x];
    if (!J.ext) return;
    if (J.origin_auto) {
        origin_argmax_block(J.ball, J.R, J.ostride, J.ctrl, sv, si);
    } else if (threadIdx.x == 0) {
        J.ctrl->origin[0] = J.origin[0];
        J.ctrl->origin[1] = J.origin[1];
        J.ctrl->origin[2] = J.origin[2];
    }
    __syncthreads();
    ext_frame_block(J.m, J.V, J.nv, J.ctrl, J.origin_auto ? J.ball : nullptr);
}
// exterior tangent balls of every row of the exterior meshes
__global__ void __launch_bounds__(32 * kTanWarps) k_b_tangent_ext(const MeshJob *jobs, const int *unit0, int n,
                                                                  const int *ext_ids) {
    __shared__ int fronts[kTanWarps][32];
    __shared__ int cands[kTanWarps][kCandMax + 1];
    const int u = blockIdx.x * kTanWarps + (threadIdx.x >> 5);
    if (u >= unit0[n]) return;
    const int e = find_job(unit0, n, u);
    const MeshJob &J = jobs[ext_ids[e]];
    tangent_ext_row(J.m, J.pos, J.nrm, u - unit0[e], J.fr, J.ball, J.ctrl, fronts[threadIdx.x >> 5],
                    cands[threadIdx.x >> 5]);
}
__global__ void k_b_colfactor(const MeshJob *jobs, const int *row0, int n) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= row0[n]) return;
    const int j = find_job(row0, n, g);
    const MeshJob &J = jobs[j];
    if (!J.ext) return;
    const int u = g - row0[j];
    const double d0 = J.pos[3 * u] - J.ctrl->origin[0], d1 = J.pos[3 * u + 1] - J.ctrl->origin[1],
                 d2 = J.pos[3 * u + 2] - J.ctrl->origin[2];
    J.cf[u] = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

// finishing: zero Lambda (grid.y = mesh), histograms (one block per row),
// symmetrisation (one block per tile pair), Laplacian diagonals (one warp per row)
__global__ void k_b_fill_zero(const MeshJob *jobs) {
    const MeshJob &J = jobs[blockIdx.y];
    if (!J.Lambda) return;
    const size_t nn = (size_t)J.R * J.R;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x)
        J.Lambda[i] = 0.0;
}
__global__ void __launch_bounds__(kHistThreads) k_b_histogram(const MeshJob *jobs, const int *row0, int n) {
    extern __shared__ int hist[];
    __shared__ typename HistScan::TempStorage scan_tmp;
    const int j = find_job(row0, n, blockIdx.x);
    const MeshJob &J = jobs[j];
    row_histogram(blockIdx.x - row0[j], J.exits, J.order, J.ball, J.area, J.cf, J.R, J.W, J.cap, J.hbin, J.hcnt,
                  J.hnnz, J.Lambda, J.omega, J.ctrl, hist, scan_tmp);
}
__global__ void k_b_symmetrize(const MeshJob *jobs, const int *tile0, int n) {
    __shared__ double A[32][33], B[32][33];
    const int j = find_job(tile0, n, blockIdx.x);
    const MeshJob &J = jobs[j];
    if (!J.Lambda) return;
    const int nt = (J.R + 31) / 32, t = blockIdx.x - tile0[j];
    const int I = t / nt, Jt = t % nt;
    if (I > Jt) return;
    symmetrize_tiles(J.Lambda, J.R, I, Jt, A, B);
}
__global__ void k_b_to_f32(const MeshJob *jobs) {
    const MeshJob &J = jobs[blockIdx.y];
    if (!J.Lambda || !J.Lambda32) return;
    const size_t nn = (size_t)J.R * J.R;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x)
        J.Lambda32[i] = (float)J.Lambda[i];
}
__global__ void k_b_diagonal(const MeshJob *jobs, const int *row0, int n) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= row0[n]) return;
    const int j = find_job(row0, n, g);
    const MeshJob &J = jobs[j];
    if (!J.Lambda) return;
    diagonal_row(J.Lambda, J.R, g - row0[j], J.cf, J.kill ? J.H0 : nullptr, J.inv_n0);
}

// rows in the caller's order (queue-order option)
__global__ void k_order_identity(int R, int32_t *order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < R) order[i] = i;
}

// ---------------------------------------------------------------- workspace
struct Layout {
    size_t ball, keys, keys_s, order, exits, H0, cf, ctrl, sort, total;
    size_t sort_bytes;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// per-mesh scratch; `own_ctrl` adds the control block of a single-mesh
// estimate (a batch keeps its blocks in its header)
static Layout layout(int R, int W, bool own_ctrl) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
    L.ball = take(sizeof(RowBall) * R);
    L.keys = take(sizeof(unsigned long long) * R);
    L.keys_s = take(sizeof(unsigned long long) * R);
    L.order = take(sizeof(int32_t) * R);
    L.exits = take(sizeof(int32_t) * (size_t)R * W);
    L.H0 = take(sizeof(int32_t) * R);
    L.cf = take(sizeof(double) * R);
    L.ctrl = own_ctrl ? take(sizeof(Ctrl)) : 0;
    size_t sb = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, sb, (unsigned long long *)nullptr, (unsigned long long *)nullptr, R, 0, 62);
    L.sort_bytes = sb;
    L.sort = take(sb);
    L.total = o;
    return L;
}

// one mesh of an estimate: its inputs, outputs and scratch
struct Plan {
    mcs_mesh m = nullptr;
    mcs_rows rows{};
    mcs_outputs out{};
    Layout L{};
    char *ws = nullptr;
    Ctrl *ctrl = nullptr;
    bool ext = false;
    int W = 0;
    double kappa = 0.0;
    uint64_t seed = 0;
    long long killing = 0;
    int origin_auto = 1;
    double origin[3] = {0.0, 0.0, 0.0};
    Frame fr{};
    RowBall *ball() const { return (RowBall *)(ws + L.ball); }
    int32_t *order() const { return (int32_t *)(ws + L.order); }
    int32_t *exits() const { return (int32_t *)(ws + L.exits); }
    int32_t *H0() const { return out.H0 ? out.H0 : (int32_t *)(ws + L.H0); }
    double *cf() const { return ext ? (double *)(ws + L.cf) : nullptr; }
    unsigned long long walks() const { return (unsigned long long)rows.n_rows * (unsigned long long)W; }
};

static mcs_status check_common(const mcs_params *p, const std::string &f) {
    MCS_ARG(p->walks_per_row > 0 && p->walks_per_row % 2 == 0, f + ": walks_per_row must be a positive even number");
    MCS_ARG(p->eps > 0.0 && std::isfinite(p->eps), f + ": eps must be positive");
    MCS_ARG(p->cap_deg > 0.0 && p->cap_deg < 180.0, f + ": cap_deg must be in (0, 180)");
    MCS_ARG(p->bisect_iters >= 0 && p->bisect_iters <= 60, f + ": bisect_iters out of range");
    MCS_ARG(p->max_steps >= 2, f + ": max_steps must be >= 2");
    MCS_ARG(p->prec == MCS_FP32 || p->prec == MCS_FP64, f + ": prec must be 32 or 64");
    MCS_ARG(p->killing_walks >= 0, f + ": killing_walks < 0");
    MCS_ARG(p->kappa < 1.0, f + ": kappa must be < 1");
    MCS_ARG(p->threads_per_block == 0 || (p->threads_per_block % 32 == 0 && p->threads_per_block <= 128 &&
                                          p->threads_per_block > 0),
            f + ": threads_per_block must be 0 or a multiple of 32 up to 128");
    MCS_ARG(p->blocks_per_sm >= 0 && p->blocks_per_sm <= 64, f + ": blocks_per_sm out of range");
    MCS_ARG(p->queue_order >= 0 && p->queue_order <= 3, f + ": queue_order must be in [0, 3]");
    MCS_ARG(p->bvh_layout == 0 || p->bvh_layout == 2 || p->bvh_layout == 4, f + ": bvh_layout must be 0, 2 or 4");
    MCS_ARG(p->lanes_per_query == 0 || p->lanes_per_query == 1 || (p->lanes_per_query == 4 && p->bvh_layout == 4),
            f + ": lanes_per_query must be 0, 1, or 4 (with bvh_layout 4)");
    MCS_ARG(p->start_mode >= 0 && p->start_mode <= 2, f + ": start_mode must be 0, 1 or 2");
    MCS_ARG(p->start_mode != 2 || (p->inset > 0.0 && std::isfinite(p->inset)), f + ": start_mode 2 needs inset > 0");
    return MCS_OK;
}

// start modes 1 and 2 serve the Galerkin assembly of interior estimates: the
// nodal Lambda takes neither per-walk weights nor the naive form
static mcs_status check_start_mode(const mcs_params *p, int domain, const mcs_outputs *out, const std::string &f) {
    MCS_ARG(p->start_mode == 0 || (domain == MCS_INTERIOR && out->Lambda == nullptr),
            f + ": start_mode 1 and 2 are for interior estimates without Lambda (use the Galerkin assembly)");
    return MCS_OK;
}

static mcs_status check_mesh_rows(mcs_mesh m, const mcs_rows *rows, const mcs_outputs *out, int domain, int W,
                                  const std::string &f, bool batched = false) {
    MCS_ARG(m != nullptr, f + ": NULL mesh");
    const int R = rows->n_rows;
    MCS_ARG(R > 0, f + ": n_rows must be positive");
    MCS_ARG(rows->pos && rows->nrm && rows->area, f + ": NULL row arrays");
    MCS_ARG(rows->tri2bin != nullptr || R == m->nv, f + ": vertex rows need n_rows == nv");
    MCS_ARG((long long)R * W < (1LL << 40), f + ": too many walks");
    MCS_ARG(domain == MCS_INTERIOR || domain == MCS_EXTERIOR, f + ": bad domain");
    MCS_ARG(out->hist_bin && out->hist_cnt && out->hist_nnz, f + ": NULL histogram outputs");
    if (batched)
        MCS_ARG(R <= kHistDenseMaxRows, f + ": more than 51200 rows in a batch item");
    else
        MCS_ARG(R <= kHistDenseMaxRows || W <= kHistSortMaxW,
                f + ": more than 51200 rows need walks_per_row <= 8192");
    return MCS_OK;
}

static Plan make_plan(mcs_mesh m, const mcs_rows &rows, const mcs_outputs &out, const mcs_params *p, int domain,
                      uint64_t seed, int origin_auto, const double *origin, char *ws, Ctrl *ctrl, bool own_ctrl) {
    Plan pl;
    pl.m = m;
    pl.rows = rows;
    pl.out = out;
    pl.W = p->walks_per_row;
    pl.L = layout(rows.n_rows, pl.W, own_ctrl);
    pl.ws = ws;
    pl.ctrl = own_ctrl ? (Ctrl *)(ws + pl.L.ctrl) : ctrl;
    pl.ext = domain == MCS_EXTERIOR;
    pl.kappa = p->kappa >= 0.0 ? p->kappa : (rows.tri2bin ? 1e-6 : 0.05);
    pl.seed = seed;
    pl.killing = pl.ext ? p->killing_walks : 0;
    pl.origin_auto = origin_auto;
    for (int k = 0; k < 3; k++) pl.origin[k] = origin[k];
    pl.fr.onemk = 1.0 - pl.kappa;
    pl.fr.iw0 = 1.0 / sin(p->cap_deg * (M_PI / 360.0));
    pl.fr.eps = p->eps;
    pl.fr.rho_min_factor = p->rho_min_factor;
    pl.fr.rmax = m->rmax;
    pl.fr.bisect_iters = p->bisect_iters;
    pl.fr.start_mode = p->start_mode;
    pl.fr.inset = p->start_mode == 2 ? p->inset : 0.0;
    return pl;
}

// the row schedule: Z-order of the row points (Sec. 5), or the caller's order
static mcs_status enqueue_order(const Plan &pl, int row_order, cudaStream_t st) {
    const int R = pl.rows.n_rows, tb = 128, gr = (R + tb - 1) / tb;
    if (row_order & 1) {
        note_launch();
        k_order_identity<<<gr, tb, 0, st>>>(R, pl.order());
    } else {
        double inv[3];
        for (int k = 0; k < 3; k++) inv[k] = 1.0 / (pl.m->hi[k] - pl.m->lo[k]);
        unsigned long long *keys = (unsigned long long *)(pl.ws + pl.L.keys);
        unsigned long long *keys_s = (unsigned long long *)(pl.ws + pl.L.keys_s);
        note_launch();
        k_row_keys<<<gr, tb, 0, st>>>(pl.rows.pos, R, pl.m->lo[0], pl.m->lo[1], pl.m->lo[2], inv[0], inv[1], inv[2],
                                      keys);
        size_t sb = pl.L.sort_bytes;
        MCS_CUDA(cub::DeviceRadixSort::SortKeys(pl.ws + pl.L.sort, sb, keys, keys_s, R, 0, 62, st));
        note_launch();
        k_order_from_keys<<<gr, tb, 0, st>>>(keys_s, R, pl.order());
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

// control block, row schedule, tangent balls (and the exterior frame)
static mcs_status enqueue_setup(const Plan &pl, int row_order, cudaStream_t st) {
    const int R = pl.rows.n_rows;
    const DevMesh dm = pl.m->dev();
    MCS_CUDA(cudaMemsetAsync(pl.ctrl, 0, sizeof(Ctrl), st));
    MCS_CUDA(cudaMemsetAsync(pl.H0(), 0, sizeof(int32_t) * R, st));
    const mcs_status s = enqueue_order(pl, row_order, st);
    if (s != MCS_OK) return s;
    const int tb = 128, gr = (R + tb - 1) / tb;
    const int tgrid = (R + kTanWarps - 1) / kTanWarps;
    if (pl.ext) {
        if (pl.origin_auto) {
            const int ostride = (R + 255) / 256, nsub = (R + ostride - 1) / ostride;
            note_launch();
            k_tangent_int<<<(nsub + kTanWarps - 1) / kTanWarps, 32 * kTanWarps, 0, st>>>(
                dm, pl.rows.pos, pl.rows.nrm, R, ostride, pl.fr, pl.ball(), pl.ctrl);
            note_launch();
            k_origin_argmax<<<1, 1024, 0, st>>>(pl.ball(), R, ostride, pl.ctrl);
        } else {
            note_launch();
            k_set_origin<<<1, 1, 0, st>>>(pl.ctrl, pl.origin[0], pl.origin[1], pl.origin[2]);
        }
        note_launch();
        k_ext_frame<<<1, kFrameThreads, 0, st>>>(dm, pl.m->V, pl.m->nv, pl.ctrl, pl.origin_auto ? pl.ball() : nullptr);
        note_launch();
        k_tangent_ext<<<tgrid, 32 * kTanWarps, 0, st>>>(dm, pl.rows.pos, pl.rows.nrm, R, pl.fr, pl.ball(), pl.ctrl);
        note_launch();
        k_colfactor<<<gr, tb, 0, st>>>(pl.rows.pos, R, pl.ctrl, pl.cf());
    } else {
        note_launch();
        k_tangent_int<<<tgrid, 32 * kTanWarps, 0, st>>>(dm, pl.rows.pos, pl.rows.nrm, R, 1, pl.fr, pl.ball(), pl.ctrl);
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

// the job of a plan; n_row_walks < R*W truncates it to its first rows (autotuner samples)
static WalkJob make_job(const Plan &pl, unsigned long long n_row_walks, unsigned long long n_kill) {
    WalkJob J;
    J.m = pl.m->dev();
    J.ball = pl.ball();
    J.order = pl.order();
    J.tri2bin = pl.rows.tri2bin;
    J.exits = pl.exits();
    J.exit_tri = pl.out.exit_tri;
    J.exit_bary = pl.out.exit_bary;
    J.walk_w = pl.out.walk_w;
    J.start_mode = pl.fr.start_mode;
    J.H0 = pl.H0();
    J.ctrl = pl.ctrl;
    J.n_rows_walks = n_row_walks;
    J.n_kill = n_kill;
    for (int k = 0; k < 3; k++) J.box_c[k] = 0.5 * (pl.m->lo[k] + pl.m->hi[k]);
    const double s0 = pl.m->hi[0] - pl.m->lo[0], s1 = pl.m->hi[1] - pl.m->lo[1], s2 = pl.m->hi[2] - pl.m->lo[2];
    J.esc_int2 = s0 * s0 + s1 * s1 + s2 * s2;
    for (int k = 0; k < 3; k++) J.box_cf[k] = (float)J.box_c[k];
    J.esc_int2f = (float)J.esc_int2;
    J.R = pl.rows.n_rows;
    J.W = pl.W;
    J.k0 = (uint32_t)pl.seed;
    J.k1 = (uint32_t)(pl.seed >> 32);
    J.ext = pl.ext;
    J.row_stride = 1;
    return J;
}

// writes the job table and its queue offsets on the stream
static mcs_status store_jobs(const std::vector<WalkJob> &jobs, WalkJob *d_jobs, unsigned long long *d_offs,
                             cudaStream_t st) {
    unsigned long long off = 0;
    for (size_t base = 0; base < jobs.size(); base += kJobChunk) {
        JobChunk c;
        c.count = (int)std::min<size_t>(kJobChunk, jobs.size() - base);
        c.base = (int)base;
        c.last = base + c.count == jobs.size();
        for (int i = 0; i < c.count; i++) {
            c.j[i] = jobs[base + i];
            c.offs[i] = off;
            off += jobs[base + i].n_rows_walks + jobs[base + i].n_kill;
        }
        c.offs[c.count] = off;
        note_launch();
        k_store_jobs<<<1, 128, 0, st>>>(c, d_jobs, d_offs);
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

typedef void (*WalkKernel)(MultiArgs);

template <typename T, bool COUNT, int TRAV> static WalkKernel walk_kernel_mode(int mode, bool multi) {
    if (!multi)
        return mode == 0 ? k_walks<T, 0, COUNT, false, TRAV>
                         : (mode == 3 ? k_walks<T, 3, COUNT, false, TRAV> : k_walks<T, 1, COUNT, false, TRAV>);
    return mode == 0 ? k_walks<T, 0, COUNT, true, TRAV>
                     : (mode == 1 ? k_walks<T, 1, COUNT, true, TRAV> : k_walks<T, 2, COUNT, true, TRAV>);
}

template <typename T, bool COUNT> static WalkKernel walk_kernel_w(int mode, bool multi, int trav) {
    if (trav == 2) return walk_kernel_mode<T, COUNT, 2>(mode, multi);
    return trav == 1 ? walk_kernel_mode<T, COUNT, 1>(mode, multi) : walk_kernel_mode<T, COUNT, 0>(mode, multi);
}

// traversal: 0 binary, 1 4-wide one lane per query, 2 4-wide four lanes per query
static int trav_of(const mcs_params *p) {
    if (p->bvh_layout != 4) return 0;
    return p->lanes_per_query == 4 ? 2 : 1;
}

// the BVH node layout of the walk queries: binary unless the caller asks for
// 4-wide (measured: binary 304 ms, 4-wide 332 ms on the two-sphere exterior
// workload; 95 vs 107 ms on the 2M-face union)
static bool use_wide(const mcs_params *p) { return p->bvh_layout == 4; }

// mode: 0 all jobs interior, 1 all exterior, 2 mixed; multi: several jobs
static WalkKernel walk_kernel(const mcs_params *p, int mode, bool multi) {
    const int trav = trav_of(p);
    if (p->count_work)
        return p->prec == MCS_FP64 ? walk_kernel_w<double, true>(mode, multi, trav)
                                   : walk_kernel_w<float, true>(mode, multi, trav);
    return p->prec == MCS_FP64 ? walk_kernel_w<double, false>(mode, multi, trav)
                               : walk_kernel_w<float, false>(mode, multi, trav);
}

// resident blocks per SM of the walk kernel for this block size
static mcs_status walk_residency(const mcs_params *p, int mode, bool multi, int *tpb_out, int *bps_out) {
    const int tpb = p->threads_per_block > 0 ? p->threads_per_block : 128;
    int occ = 0;
    MCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, walk_kernel(p, mode, multi), tpb, 0));
    occ = std::max(1, occ);
    *tpb_out = tpb;
    *bps_out = p->blocks_per_sm > 0 ? std::min(p->blocks_per_sm, occ) : occ;
    return MCS_OK;
}

// the persistent walk launch over a job table
// n_jobs == 1: `one` is the job (passed in the kernel parameters); else the
// table at d_jobs / d_offs, written earlier on the stream
static mcs_status launch_walks(const WalkJob *d_jobs, const unsigned long long *d_offs, int n_jobs, const WalkJob *one,
                               Ctrl *stats, const mcs_params *p, int mode, int tpb, int bps, cudaStream_t st) {
    MultiArgs a;
    memset(&a, 0, sizeof a);
    if (one) a.j0 = *one;
    a.jobs = d_jobs;
    a.offs = d_offs;
    a.n_jobs = n_jobs;
    a.queue = &stats->queue;
    a.stats = stats;
    a.eps = p->eps;
    a.iw0 = 1.0 / sin(p->cap_deg * (M_PI / 360.0));
    a.eps2f = (float)(2.0 * p->eps);
    a.max_steps = p->max_steps;
    note_launch();
    walk_kernel(p, mode, n_jobs > 1)<<<num_sms() * bps, tpb, 0, st>>>(a);
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

// CUDA loads kernels lazily, at their first use, and loading one reserves
// device memory for its code; this loads every kernel that a one-mesh
// estimate can launch, so that later estimates load nothing
mcs_status preload_estimate_kernels() {
    cudaFuncAttributes fa;
    const void *fns[] = {(const void *)k_order_identity, (const void *)k_row_keys, (const void *)k_order_from_keys,
                         (const void *)k_tangent_int,    (const void *)k_origin_argmax, (const void *)k_set_origin,
                         (const void *)k_ext_frame,      (const void *)k_tangent_ext,   (const void *)k_colfactor,
                         (const void *)k_fill_zero,      (const void *)k_histogram,     (const void *)k_symmetrize,
                         (const void *)k_diagonal,       (const void *)k_to_f32};
    for (const void *f : fns) MCS_CUDA(cudaFuncGetAttributes(&fa, f));
    for (int prec = 0; prec < 2; prec++)
        for (int count = 0; count < 2; count++)
            for (int trav = 0; trav < 3; trav++)
                for (int mode : {0, 1, 3}) {
                    WalkKernel k = prec ? (count ? walk_kernel_w<double, true>(mode, false, trav)
                                                 : walk_kernel_w<double, false>(mode, false, trav))
                                        : (count ? walk_kernel_w<float, true>(mode, false, trav)
                                                 : walk_kernel_w<float, false>(mode, false, trav));
                    MCS_CUDA(cudaFuncGetAttributes(&fa, (const void *)k));
                }
    return MCS_OK;
}

static size_t hist_smem(int R) { return std::max<size_t>(sizeof(int) * (size_t)R, 1024); }

static mcs_status prepare_histogram(size_t smem) {
    MCS_CUDA(cudaFuncSetAttribute(k_histogram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return MCS_OK;
}

// histogram + row normalisation, symmetrisation, Laplacian diagonal
static mcs_status enqueue_hist(const Plan &pl, cudaStream_t st) {
    const int R = pl.rows.n_rows, W = pl.W;
    if (pl.out.Lambda) {
        note_launch();
        k_fill_zero<<<num_sms() * 8, 256, 0, st>>>(pl.out.Lambda, (size_t)R * R);
    }
    note_launch();
    if (R <= kHistDenseMaxRows) {
        k_histogram<<<R, kHistThreads, sizeof(int) * (size_t)R, st>>>(
            pl.exits(), pl.order(), pl.ball(), pl.rows.area, pl.cf(), R, W, std::min(W, R), pl.out.hist_bin,
            pl.out.hist_cnt, pl.out.hist_nnz, pl.out.Lambda, pl.out.omega, pl.ctrl);
    } else {
        // keys bin + 1 in [0, R] and the padding 2^end_bit - 1 > R
        const int end_bit = 32 - __builtin_clz((unsigned)R + 1u);
        auto *k = W <= kHistThreads * 4 ? k_histogram_sorted<4>
                                        : (W <= kHistThreads * 16 ? k_histogram_sorted<16> : k_histogram_sorted<32>);
        k<<<R, kHistThreads, 0, st>>>(pl.exits(), pl.order(), pl.ball(), pl.rows.area, pl.cf(), R, W, std::min(W, R),
                                      pl.out.hist_bin, pl.out.hist_cnt, pl.out.hist_nnz, pl.out.Lambda, pl.out.omega,
                                      pl.ctrl, end_bit);
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

static mcs_status enqueue_assembly(const Plan &pl, cudaStream_t st) {
    const int R = pl.rows.n_rows;
    if (pl.out.Lambda) {
        const int nt = (R + 31) / 32;
        note_launch();
        k_symmetrize<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(pl.out.Lambda, R);
        const bool kill = pl.ext && pl.killing > 0;
        note_launch();
        k_diagonal<<<(R * 32 + 255) / 256, 256, 0, st>>>(pl.out.Lambda, R, pl.cf(), kill ? pl.H0() : nullptr,
                                                        kill ? 1.0 / (double)pl.killing : 0.0);
        if (pl.out.Lambda32) {
            note_launch();
            k_to_f32<<<num_sms() * 8, 256, 0, st>>>(pl.out.Lambda, (size_t)R * R, pl.out.Lambda32);
        }
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

// host statistics of one control block; the status of that estimate
static mcs_status read_stats(const Ctrl &hc, const Plan *pl, unsigned long long walks, mcs_stats *stats,
                             const char *fn) {
    if (stats) {
        stats->nodes_visited = (long long)hc.nodes;
        stats->tris_tested = (long long)hc.tris;
        stats->walks = (long long)walks;
        stats->steps = (long long)hc.steps;
        stats->capped = (long long)hc.capped;
        stats->lost = (long long)hc.lost;
        stats->discarded_rows = hc.discarded;
        stats->killing_steps = (long long)hc.kill_steps;
        stats->killing_capped = (long long)hc.kill_capped;
        const bool ext = pl && pl->ext;
        for (int k = 0; k < 3; k++) stats->origin[k] = ext ? hc.origin[k] : 0.0;
        stats->rmax = pl ? (ext ? hc.rmax_ext : pl->m->rmax) : 0.0;
        stats->device_error = hc.err;
    }
    if (hc.err & kErrNoOrigin) {
        set_error(std::string(fn) + ": no interior tangent ball to place the inversion centre");
        return MCS_ERR_NO_INTERIOR_POINT;
    }
    if (hc.err & kErrNoHit) {
        char buf[320];
        snprintf(buf, sizeof buf,
                 "%s: a walk query found no triangle (kind %d, killing %d, walk %llu, step %d, "
                 "x~ = (%.9g, %.9g, %.9g)); walk retired as lost",
                 fn, hc.diag_kind, hc.diag_killing, hc.diag_walk, hc.diag_step, hc.diag_p[0], hc.diag_p[1],
                 hc.diag_p[2]);
        set_error(buf);
        return MCS_ERR_DEVICE;
    }
    if (hc.err) {
        set_error(std::string(fn) + (hc.err & kErrBin ? ": tri2bin maps a triangle outside [0, n_rows)"
                                                      : ": BVH traversal stack or iteration bound exceeded"));
        return MCS_ERR_DEVICE;
    }
    if (hc.capped || hc.kill_capped) return MCS_WARN_CAPPED;
    return hc.lost ? MCS_WARN_LOST : MCS_OK;
}

// ---------------------------------------------------------------- batches
// Batch workspace: header (job table, queue offsets, control blocks: one per
// mesh and one for the launch), then each mesh's scratch.
struct BatchLayout {
    size_t jobs, offs, ctrl, mjobs, ints, keys, keys_s, sort, total;
    size_t sort_bytes;
    std::vector<size_t> item;
};

static BatchLayout batch_layout(const mcs_batch_item *items, int n, int W) {
    BatchLayout B;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
    long long rows = 0;
    for (int i = 0; i < n; i++) rows += std::max(1, items[i].rows.n_rows);
    B.jobs = take(sizeof(WalkJob) * (size_t)n);
    B.offs = take(sizeof(unsigned long long) * (size_t)(n + 1));
    B.ctrl = take(sizeof(Ctrl) * (size_t)(n + 1));
    B.mjobs = take(sizeof(MeshJob) * (size_t)n);
    B.ints = take(sizeof(int) * (size_t)(5 * (n + 1)));  // row0, unitA, unitB, tile0, ext ids
    B.keys = take(sizeof(unsigned long long) * (size_t)rows);
    B.keys_s = take(sizeof(unsigned long long) * (size_t)rows);
    size_t sb = 0;
    cub::DeviceSegmentedRadixSort::SortKeys(nullptr, sb, (unsigned long long *)nullptr, (unsigned long long *)nullptr,
                                            (int)rows, n, (int *)nullptr, (int *)nullptr, 0, 62);
    B.sort_bytes = sb;
    B.sort = take(sb);
    B.item.resize(n);
    for (int i = 0; i < n; i++) B.item[i] = take(layout(std::max(1, items[i].rows.n_rows), W, false).total);
    B.total = o;
    return B;
}

struct Batch {
    std::vector<Plan> plans;
    WalkJob *jobs = nullptr;
    unsigned long long *offs = nullptr;
    Ctrl *ctrl = nullptr;   // n + 1 blocks: per mesh, then the launch's
    MeshJob *mjobs = nullptr;
    int *row0 = nullptr, *unitA = nullptr, *unitB = nullptr, *tile0 = nullptr, *ext_ids = nullptr;
    unsigned long long *keys = nullptr, *keys_s = nullptr;
    void *sort = nullptr;
    size_t sort_bytes = 0;
    std::vector<int> h_row0, h_unitA, h_unitB, h_tile0, h_ext;  // host copies
    int max_rows = 1;
    bool any_lambda = false, any_lambda32 = false;
    int n = 0;
    int mode = 0;           // walk kernel: 0 all interior, 1 all exterior, 2 mixed
    mcs_params p{};
    Ctrl *launch_ctrl() const { return ctrl + n; }
};

static mcs_status make_batch(const mcs_batch_item *items, int n, const mcs_params *p, void *workspace,
                             size_t workspace_bytes, Batch &b, const char *fn) {
    const std::string f(fn);
    MCS_ARG(items != nullptr && p != nullptr, f + ": NULL items or params");
    MCS_ARG(n > 0, f + ": the batch is empty");
    mcs_status s = check_common(p, f);
    if (s != MCS_OK) return s;
    for (int i = 0; i < n; i++) {
        s = check_mesh_rows(items[i].mesh, &items[i].rows, &items[i].out, items[i].domain, p->walks_per_row,
                            f + " item " + std::to_string(i), true);
        if (s != MCS_OK) return s;
        MCS_ARG(p->start_mode == 0, f + ": start_mode 1 and 2 are for single estimates (mcs_estimate_dtn)");
        MCS_ARG(!use_wide(p) || mcs_mesh_has_wide(items[i].mesh),
                f + " item " + std::to_string(i) + ": bvh_layout 4 needs mcs_mesh_build_wide first");
    }
    const BatchLayout B = batch_layout(items, n, p->walks_per_row);
    MCS_ARG(workspace != nullptr && workspace_bytes >= B.total, f + ": workspace too small");
    MCS_ARG(((uintptr_t)workspace & 255) == 0, f + ": workspace must be 256-byte aligned");
    char *ws = (char *)workspace;
    b.n = n;
    b.p = *p;
    b.jobs = (WalkJob *)(ws + B.jobs);
    b.offs = (unsigned long long *)(ws + B.offs);
    b.ctrl = (Ctrl *)(ws + B.ctrl);
    b.mjobs = (MeshJob *)(ws + B.mjobs);
    int *ints = (int *)(ws + B.ints);
    b.row0 = ints;
    b.unitA = ints + (n + 1);
    b.unitB = ints + 2 * (n + 1);
    b.tile0 = ints + 3 * (n + 1);
    b.ext_ids = ints + 4 * (n + 1);
    b.keys = (unsigned long long *)(ws + B.keys);
    b.keys_s = (unsigned long long *)(ws + B.keys_s);
    b.sort = ws + B.sort;
    b.sort_bytes = B.sort_bytes;
    b.plans.clear();
    int n_ext = 0;
    for (int i = 0; i < n; i++) n_ext += items[i].domain == MCS_EXTERIOR;
    b.mode = n_ext == 0 ? 0 : (n_ext == n ? 1 : 2);
    for (int i = 0; i < n; i++) {
        const mcs_batch_item &it = items[i];
        b.plans.push_back(make_plan(it.mesh, it.rows, it.out, p, it.domain, it.seed, it.origin_auto, it.origin,
                                    ws + B.item[i], b.ctrl + i, false));
    }
    // unit offsets of the batched kernels
    b.h_row0.assign(1, 0);
    b.h_unitA.assign(1, 0);
    b.h_unitB.assign(1, 0);
    b.h_tile0.assign(1, 0);
    b.h_ext.clear();
    b.max_rows = 1;
    b.any_lambda = false;
    b.any_lambda32 = false;
    for (int i = 0; i < n; i++) {
        const Plan &pl = b.plans[i];
        const int R = pl.rows.n_rows, ostride = (R + 255) / 256;
        b.h_row0.push_back(b.h_row0.back() + R);
        b.h_unitA.push_back(b.h_unitA.back() +
                            (pl.ext ? (pl.origin_auto ? (R + ostride - 1) / ostride : 0) : R));
        const int nt = (R + 31) / 32;
        b.h_tile0.push_back(b.h_tile0.back() + nt * nt);
        if (pl.ext) {
            b.h_ext.push_back(i);
            b.h_unitB.push_back(b.h_unitB.back() + R);
        }
        b.max_rows = std::max(b.max_rows, R);
        b.any_lambda = b.any_lambda || pl.out.Lambda != nullptr;
        b.any_lambda32 = b.any_lambda32 || (pl.out.Lambda != nullptr && pl.out.Lambda32 != nullptr);
    }
    return MCS_OK;
}

static MeshJob make_mesh_job(const Plan &pl) {
    MeshJob J;
    memset(&J, 0, sizeof J);
    J.m = pl.m->dev();
    J.pos = pl.rows.pos;
    J.nrm = pl.rows.nrm;
    J.area = pl.rows.area;
    J.V = pl.m->V;
    J.ball = pl.ball();
    J.ctrl = pl.ctrl;
    J.order = pl.order();
    J.exits = pl.exits();
    J.H0 = pl.H0();
    J.cf = pl.cf();
    J.hbin = pl.out.hist_bin;
    J.hcnt = pl.out.hist_cnt;
    J.hnnz = pl.out.hist_nnz;
    J.Lambda = pl.out.Lambda;
    J.Lambda32 = pl.out.Lambda32;
    J.omega = pl.out.omega;
    J.fr = pl.fr;
    for (int k = 0; k < 3; k++) {
        J.lo[k] = pl.m->lo[k];
        J.inv[k] = 1.0 / (pl.m->hi[k] - pl.m->lo[k]);
        J.origin[k] = pl.origin[k];
    }
    const bool kill = pl.ext && pl.killing > 0;
    J.inv_n0 = kill ? 1.0 / (double)pl.killing : 0.0;
    J.kill = kill;
    J.R = pl.rows.n_rows;
    J.W = pl.W;
    J.cap = std::min(pl.W, pl.rows.n_rows);
    J.nv = pl.m->nv;
    J.ext = pl.ext;
    J.origin_auto = pl.origin_auto;
    J.ostride = (pl.rows.n_rows + 255) / 256;
    return J;
}

static mcs_status store_int_array(const std::vector<int> &v, int *d, cudaStream_t st) {
    for (size_t base = 0; base < v.size(); base += kIntChunk) {
        IntChunk c;
        c.count = (int)std::min<size_t>(kIntChunk, v.size() - base);
        c.base = (int)base;
        for (int i = 0; i < c.count; i++) c.v[i] = v[base + i];
        note_launch();
        k_store_ints<<<1, 256, 0, st>>>(c, d);
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

// the batch's row setup in a fixed number of launches: job table, row
// schedule (one segmented sort), interior tangent balls, exterior frames,
// exterior tangent balls, column factors
static mcs_status enqueue_batch_setup(const Batch &b, int row_order, cudaStream_t st) {
    MCS_CUDA(cudaMemsetAsync(b.ctrl, 0, sizeof(Ctrl) * (b.n + 1), st));
    for (int base = 0; base < b.n; base += kMeshChunk) {
        MeshChunk c;
        c.count = std::min(kMeshChunk, b.n - base);
        c.base = base;
        for (int i = 0; i < c.count; i++) c.j[i] = make_mesh_job(b.plans[base + i]);
        note_launch();
        k_store_mesh_jobs<<<1, 64, 0, st>>>(c, b.mjobs);
    }
    mcs_status s;
    if ((s = store_int_array(b.h_row0, b.row0, st)) != MCS_OK) return s;
    if ((s = store_int_array(b.h_unitA, b.unitA, st)) != MCS_OK) return s;
    if ((s = store_int_array(b.h_unitB, b.unitB, st)) != MCS_OK) return s;
    if ((s = store_int_array(b.h_tile0, b.tile0, st)) != MCS_OK) return s;
    if (!b.h_ext.empty() && (s = store_int_array(b.h_ext, b.ext_ids, st)) != MCS_OK) return s;
    const int rows = b.h_row0.back(), tb = 256;
    const bool identity = row_order & 1;
    note_launch();
    k_b_rows<<<(rows + tb - 1) / tb, tb, 0, st>>>(b.mjobs, b.row0, b.n, identity, b.keys);
    if (!identity) {
        size_t sb = b.sort_bytes;
        MCS_CUDA(cub::DeviceSegmentedRadixSort::SortKeys(b.sort, sb, b.keys, b.keys_s, rows, b.n, b.row0, b.row0 + 1,
                                                         0, 62, st));
        note_launch();
        k_b_order<<<(rows + tb - 1) / tb, tb, 0, st>>>(b.mjobs, b.row0, b.n, b.keys_s);
    }
    const int ua = b.h_unitA.back(), ub = b.h_unitB.back(), ne = (int)b.h_ext.size();
    if (ua > 0) {
        note_launch();
        k_b_tangent_int<<<(ua + kTanWarps - 1) / kTanWarps, 32 * kTanWarps, 0, st>>>(b.mjobs, b.unitA, b.n);
    }
    if (ne > 0) {
        note_launch();
        k_b_frame<<<b.n, kFrameThreads, 0, st>>>(b.mjobs);
        note_launch();
        k_b_tangent_ext<<<(ub + kTanWarps - 1) / kTanWarps, 32 * kTanWarps, 0, st>>>(b.mjobs, b.unitB, ne,
                                                                                    b.ext_ids);
        note_launch();
        k_b_colfactor<<<(rows + tb - 1) / tb, tb, 0, st>>>(b.mjobs, b.row0, b.n);
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

// histograms, row normalisation, symmetrisation and diagonals of every mesh
static mcs_status enqueue_batch_finish(const Batch &b, cudaStream_t st) {
    const int rows = b.h_row0.back();
    if (b.any_lambda) {
        note_launch();
        k_b_fill_zero<<<dim3(64, b.n), 256, 0, st>>>(b.mjobs);
    }
    note_launch();
    k_b_histogram<<<rows, kHistThreads, hist_smem(b.max_rows), st>>>(b.mjobs, b.row0, b.n);
    if (b.any_lambda) {
        note_launch();
        k_b_symmetrize<<<b.h_tile0.back(), dim3(32, 8), 0, st>>>(b.mjobs, b.tile0, b.n);
        note_launch();
        k_b_diagonal<<<(rows * 32 + 255) / 256, 256, 0, st>>>(b.mjobs, b.row0, b.n);
        if (b.any_lambda32) {
            note_launch();
            k_b_to_f32<<<dim3(64, b.n), 256, 0, st>>>(b.mjobs);
        }
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

// queue order of the jobs: as given, or by descending walk count (bit 2 of queue_order)
static std::vector<int> job_order(const Batch &b) {
    std::vector<int> ord(b.n);
    for (int i = 0; i < b.n; i++) ord[i] = i;
    if (b.p.queue_order & 2)
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
            const unsigned long long wx = b.plans[x].walks() + b.plans[x].killing;
            const unsigned long long wy = b.plans[y].walks() + b.plans[y].killing;
            return wx > wy;
        });
    return ord;
}

// everything a batched estimate launches, in stream order; `ev` (optional,
// 4 events) marks setup | walks | histogram + assembly; `external`: the
// events are recorded by the graph being captured, at each replay
static mcs_status enqueue_batch(const Batch &b, cudaStream_t st, cudaEvent_t *ev, bool external = false) {
    mcs_status s;
    auto mark = [&](int i) {
        if (!ev) return;
        if (external) cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal);
        else cudaEventRecord(ev[i], st);
    };
    mark(0);
    if ((s = enqueue_batch_setup(b, b.p.queue_order, st)) != MCS_OK) return s;
    std::vector<WalkJob> jobs;
    for (int i : job_order(b)) jobs.push_back(make_job(b.plans[i], b.plans[i].walks(), (unsigned long long)b.plans[i].killing));
    if (b.n > 1 && (s = store_jobs(jobs, b.jobs, b.offs, st)) != MCS_OK) return s;
    int tpb = 0, bps = 0;
    if ((s = walk_residency(&b.p, b.mode, b.n > 1, &tpb, &bps)) != MCS_OK) return s;
    mark(1);
    // one mesh: the one-job kernel, counters straight into the mesh's block
    if ((s = launch_walks(b.jobs, b.offs, b.n, b.n > 1 ? nullptr : &jobs[0], b.n > 1 ? b.launch_ctrl() : b.plans[0].ctrl,
                          &b.p, b.mode, tpb, bps, st)) != MCS_OK)
        return s;
    mark(2);
    if ((s = enqueue_batch_finish(b, st)) != MCS_OK) return s;
    mark(3);
    return MCS_OK;
}

static mcs_status batch_hist_prepare(const Batch &b) {
    MCS_CUDA(cudaFuncSetAttribute(k_b_histogram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)hist_smem(b.max_rows)));
    return MCS_OK;
}

// per-mesh and launch statistics of a finished batch (synchronises st)
static mcs_status batch_stats(const Batch &b, mcs_stats *total, mcs_stats *per_item, cudaStream_t st,
                              const char *fn) {
    std::vector<Ctrl> hc(b.n + 1);
    MCS_CUDA(cudaMemcpyAsync(hc.data(), b.ctrl, sizeof(Ctrl) * (b.n + 1), cudaMemcpyDeviceToHost, st));
    MCS_CUDA(cudaStreamSynchronize(st));
    mcs_status worst = MCS_OK;
    // the launch block holds the work counters; the rest is summed over meshes
    Ctrl sum = hc[b.n];
    sum.discarded = 0;
    sum.steps = sum.capped = sum.lost = sum.kill_steps = sum.kill_capped = 0;
    if (b.n == 1) {  // the one-job kernel counted its work in the mesh's block
        sum.nodes = hc[0].nodes;
        sum.tris = hc[0].tris;
    }
    unsigned long long walks = 0;
    std::string msgs;
    int n_bad = 0;
    for (int i = 0; i < b.n; i++) {
        sum.steps += hc[i].steps;
        sum.capped += hc[i].capped;
        sum.lost += hc[i].lost;
        sum.kill_steps += hc[i].kill_steps;
        sum.kill_capped += hc[i].kill_capped;
        const std::string name = std::string(fn) + " item " + std::to_string(i);
        const mcs_status s = read_stats(hc[i], &b.plans[i], b.plans[i].walks(), per_item ? per_item + i : nullptr,
                                        name.c_str());
        if (s < 0) {
            if (n_bad < 3) msgs += (msgs.empty() ? "" : "; ") + get_error();
            n_bad++;
        }
        if (s < 0 && worst >= 0) worst = s;
        else if (s > 0 && worst == MCS_OK) worst = s;
        sum.discarded += hc[i].discarded;
        sum.err |= hc[i].err;
        walks += b.plans[i].walks();
    }
    if (total) {
        read_stats(sum, nullptr, walks, total, fn);
        for (int k = 0; k < 4; k++) total->phase_ms[k] = 0.f;
    }
    if (worst < 0) {
        if (n_bad > 3) msgs += "; ... (" + std::to_string(n_bad) + " meshes reported errors)";
        set_error(msgs);
        return worst;
    }
    return worst;
}

}  // namespace mcs

struct mcs_graph_s {
    mcs::Batch b;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches = 0;  // library kernels per replay
    // params.timing: phase events recorded by every replay (setup | walks | finish)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool timed = false;
    ~mcs_graph_s() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
};

using namespace mcs;

extern "C" {

void mcs_default_params(mcs_params *p) {
    if (!p) return;
    p->eps = 1e-3;
    p->cap_deg = 2.5;
    p->bisect_iters = 10;
    p->kappa = -1.0;
    p->max_steps = 1024;
    p->rho_min_factor = 4.0;
    p->prec = MCS_FP32;
    p->domain = MCS_INTERIOR;
    p->origin_auto = 1;
    p->origin[0] = p->origin[1] = p->origin[2] = 0.0;
    p->killing_walks = 0;
    p->seed = 0;
    p->walks_per_row = 1024;
    p->blocks_per_sm = 0;
    p->threads_per_block = 0;
    p->timing = 0;
    p->count_work = 0;
    p->queue_order = 0;
    p->bvh_layout = 0;
    p->lanes_per_query = 0;
    p->start_mode = 0;
    p->inset = 0.0;
}

size_t mcs_estimate_workspace_size(mcs_mesh m, int n_rows, int walks_per_row, long long killing_walks) {
    (void)m; (void)killing_walks;
    if (n_rows <= 0 || walks_per_row <= 0) return 0;
    return layout(n_rows, walks_per_row, true).total;
}

mcs_status mcs_estimate_dtn(mcs_mesh m, const mcs_rows *rows, const mcs_params *p, const mcs_outputs *out,
                            void *workspace, size_t workspace_bytes, mcs_stats *stats, void *stream_) {
    const std::string f = "mcs_estimate_dtn";
    MCS_ARG(m && rows && p && out, f + ": NULL mesh, rows, params or outputs");
    mcs_status s = check_common(p, f);
    if (s != MCS_OK) return s;
    if ((s = check_mesh_rows(m, rows, out, p->domain, p->walks_per_row, f)) != MCS_OK) return s;
    if ((s = check_start_mode(p, p->domain, out, f)) != MCS_OK) return s;
    MCS_ARG(!use_wide(p) || mcs_mesh_has_wide(m), f + ": bvh_layout 4 needs mcs_mesh_build_wide first");
    const Layout L = layout(rows->n_rows, p->walks_per_row, true);
    MCS_ARG(workspace != nullptr && workspace_bytes >= L.total, f + ": workspace too small");
    MCS_ARG(((uintptr_t)workspace & 255) == 0, f + ": workspace must be 256-byte aligned");
    cudaStream_t st = as_stream(stream_);
    char *ws = (char *)workspace;
    const Plan pl = make_plan(m, *rows, *out, p, p->domain, p->seed, p->origin_auto, p->origin, ws, nullptr, true);

    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    const bool timing = stats && p->timing;
    if (timing)
        for (auto &e : ev) MCS_CUDA(cudaEventCreate(&e));
    auto mark = [&](int i) { if (timing) cudaEventRecord(ev[i], st); };
    auto release = [&]() { if (timing) for (auto &e : ev) cudaEventDestroy(e); };
    NvtxRange range("mcs_estimate_dtn");
    mark(0);
    {
        NvtxRange phase("setup_and_tangent_balls");
        if ((s = enqueue_setup(pl, p->queue_order, st)) != MCS_OK) { release(); return s; }
    }
    const WalkJob job = make_job(pl, pl.walks(), (unsigned long long)pl.killing);
    int tpb = 0, bps = 0;
    const int mode = pl.ext ? 1 : (p->start_mode != 0 ? 3 : 0);
    if ((s = walk_residency(p, mode, false, &tpb, &bps)) != MCS_OK) { release(); return s; }
    if (rows->n_rows <= kHistDenseMaxRows && (s = prepare_histogram(hist_smem(rows->n_rows))) != MCS_OK) {
        release();
        return s;
    }
    mark(1);
    {
        NvtxRange phase("walks");
        if ((s = launch_walks(nullptr, nullptr, 1, &job, pl.ctrl, p, mode, tpb, bps, st)) != MCS_OK) { release(); return s; }
    }
    mark(2);
    {
        NvtxRange phase("histogram");
        if ((s = enqueue_hist(pl, st)) != MCS_OK) { release(); return s; }
    }
    mark(3);
    {
        NvtxRange phase("assembly");
        if ((s = enqueue_assembly(pl, st)) != MCS_OK) { release(); return s; }
    }
    mark(4);
    if (!stats) { release(); return MCS_OK; }
    Ctrl hc;
    cudaError_t e = cudaMemcpyAsync(&hc, pl.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { release(); return cuda_fail(e, "mcs_estimate_dtn: reading the control block"); }
    for (int i = 0; i < 4; i++) {
        stats->phase_ms[i] = 0.f;
        if (timing) cudaEventElapsedTime(&stats->phase_ms[i], ev[i], ev[i + 1]);
    }
    release();
    return read_stats(hc, &pl, pl.walks(), stats, "mcs_estimate_dtn");
}

size_t mcs_estimate_batched_workspace_size(const mcs_batch_item *items, int n, int walks_per_row) {
    if (!items || n <= 0 || walks_per_row <= 0) return 0;
    return batch_layout(items, n, walks_per_row).total;
}

mcs_status mcs_estimate_batched(const mcs_batch_item *items, int n, const mcs_params *p, void *workspace,
                                size_t workspace_bytes, mcs_stats *total, mcs_stats *per_item, void *stream_) {
    NvtxRange range("mcs_estimate_batched");
    Batch b;
    mcs_status s = make_batch(items, n, p, workspace, workspace_bytes, b, "mcs_estimate_batched");
    if (s != MCS_OK) return s;
    cudaStream_t st = as_stream(stream_);
    if ((s = batch_hist_prepare(b)) != MCS_OK) return s;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    const bool timing = total && p->timing;
    if (timing)
        for (auto &e : ev) MCS_CUDA(cudaEventCreate(&e));
    s = enqueue_batch(b, st, timing ? ev : nullptr);
    if (s == MCS_OK && (total || per_item)) {
        s = batch_stats(b, total, per_item, st, "mcs_estimate_batched");
        if (timing)
            for (int i = 0; i < 3; i++) cudaEventElapsedTime(&total->phase_ms[i], ev[i], ev[i + 1]);
    }
    if (timing)
        for (auto &e : ev) cudaEventDestroy(e);
    return s;
}

mcs_status mcs_graph_create(const mcs_batch_item *items, int n, const mcs_params *p, void *workspace,
                            size_t workspace_bytes, mcs_graph *out) {
    MCS_ARG(out != nullptr, "mcs_graph_create: NULL output handle");
    *out = nullptr;
    mcs_graph g = new (std::nothrow) mcs_graph_s;
    if (!g) { set_error("mcs_graph_create: host allocation failed"); return MCS_ERR_OOM; }
    mcs_status s = make_batch(items, n, p, workspace, workspace_bytes, g->b, "mcs_graph_create");
    if (s == MCS_OK) s = batch_hist_prepare(g->b);
    int tpb = 0, bps = 0;
    if (s == MCS_OK) s = walk_residency(p, g->b.mode, n > 1, &tpb, &bps);  // occupancy queried before capture
    if (s != MCS_OK) { delete g; return s; }
    g->timed = p->timing != 0;
    if (g->timed)
        for (auto &ev : g->ev) {
            const cudaError_t ee = cudaEventCreate(&ev);
            if (ee != cudaSuccess) { delete g; return cuda_fail(ee, "mcs_graph_create: cudaEventCreate"); }
        }
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "mcs_graph_create: cudaStreamCreateWithFlags"); }
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        delete g;
        return cuda_fail(e, "mcs_graph_create: cudaStreamBeginCapture");
    }
    const unsigned long long before = g_launches.load();
    s = enqueue_batch(g->b, cs, g->timed ? g->ev : nullptr, true);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    // captured kernels run at each replay, not here
    g->launches = g_launches.load() - before;
    g_launches.fetch_sub(g->launches);
    cudaStreamDestroy(cs);
    if (s != MCS_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        delete g;
        return s != MCS_OK ? s : cuda_fail(e, "mcs_graph_create: cudaStreamEndCapture");
    }
    g->graph = graph;
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete g;
        return cuda_fail(e, "mcs_graph_create: cudaGraphInstantiate");
    }
    *out = g;
    return MCS_OK;
}

mcs_status mcs_graph_launch(mcs_graph g, void *stream) {
    MCS_ARG(g != nullptr, "mcs_graph_launch: NULL graph");
    NvtxRange range("mcs_graph_launch");
    MCS_CUDA(cudaGraphLaunch(g->exec, as_stream(stream)));
    note_launch(g->launches);
    return MCS_OK;
}

mcs_status mcs_graph_stats(mcs_graph g, mcs_stats *total, mcs_stats *per_item, void *stream) {
    MCS_ARG(g != nullptr, "mcs_graph_stats: NULL graph");
    const mcs_status s = batch_stats(g->b, total, per_item, as_stream(stream), "mcs_graph_stats");
    if (total && g->timed)  // the last replay's phases (batch_stats synchronised the stream)
        for (int i = 0; i < 3; i++)
            if (cudaEventElapsedTime(&total->phase_ms[i], g->ev[i], g->ev[i + 1]) != cudaSuccess)
                total->phase_ms[i] = 0.f;
    return s;
}

size_t mcs_graph_nodes(mcs_graph g) {
    if (!g || !g->graph) return 0;
    size_t k = 0;
    if (cudaGraphGetNodes(g->graph, nullptr, &k) != cudaSuccess) return 0;
    return k;
}

void mcs_graph_destroy(mcs_graph g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

mcs_status mcs_autotune_walks(const mcs_batch_item *items, int n, const mcs_params *p, void *workspace,
                              size_t workspace_bytes, double sample_fraction, mcs_params *tuned,
                              mcs_tune_trial *trials, int max_trials, int *n_trials, void *stream_) {
    NvtxRange nvtx_range("mcs_autotune_walks");
    const std::string f = "mcs_autotune_walks";
    MCS_ARG(tuned != nullptr, f + ": NULL tuned params");
    MCS_ARG(sample_fraction > 0.0 && sample_fraction <= 1.0, f + ": sample_fraction must be in (0, 1]");
    MCS_ARG(max_trials >= 0 && (max_trials == 0 || trials != nullptr), f + ": NULL trials");
    Batch b;
    mcs_status s = make_batch(items, n, p, workspace, workspace_bytes, b, f.c_str());
    if (s != MCS_OK) return s;
    cudaStream_t st = as_stream(stream_);
    int count = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MCS_CUDA(cudaEventCreate(&e0));
    MCS_CUDA(cudaEventCreate(&e1));
    auto cleanup = [&]() { cudaEventDestroy(e0); cudaEventDestroy(e1); };
    int cur_rows = -1;
    // the sample holds at least kTuneLaneWalks walks per resident lane of the
    // default launch (the whole batch if it has fewer): a shorter one is
    // dominated by the launch's tail and misranks the layouts (an 8-mesh
    // batch, 4.2M walks, sampled at 1/64: 2 walks per lane; the sample
    // preferred 4-wide nodes, whose full launch took 81 ms against 62 ms)
    constexpr long long kTuneLaneWalks = 32;
    int stride = std::max(1, (int)std::floor(1.0 / sample_fraction));
    {
        int dev = 0, sms = 0, tpb0 = 0, bps0 = 0;
        MCS_CUDA(cudaGetDevice(&dev));
        MCS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        mcs_params d = *p;
        d.threads_per_block = 0;
        d.blocks_per_sm = 0;
        if ((s = walk_residency(&d, b.mode, b.n > 1, &tpb0, &bps0)) != MCS_OK) { cleanup(); return s; }
        long long walks = 0;
        for (const Plan &pl : b.plans) walks += (long long)pl.rows.n_rows * pl.W;
        const long long floor_walks = kTuneLaneWalks * sms * tpb0 * bps0;
        stride = (int)std::max(1LL, std::min((long long)stride, walks / std::max(1LL, floor_walks)));
    }
    // sample: every stride-th row of every mesh (in the candidate's row order), no killing walks
    auto trial = [&](const mcs_params &q, float *ms, int *bps_used) -> mcs_status {
        mcs_status r;
        if ((q.queue_order & 1) != cur_rows) {
            if ((r = enqueue_batch_setup(b, q.queue_order, st)) != MCS_OK) return r;
            cur_rows = q.queue_order & 1;
        }
        Batch bq = b;
        bq.p = q;
        std::vector<WalkJob> jobs;
        for (int i : job_order(bq)) {
            // every stride-th row of the mesh's schedule: a sample spread over the whole mesh
            const Plan &pl = b.plans[i];
            const int R = pl.rows.n_rows;
            const unsigned long long rows = (unsigned long long)((R + stride - 1) / stride);
            WalkJob J = make_job(pl, rows * pl.W, 0);
            J.row_stride = stride;
            jobs.push_back(J);
        }
        if (b.n > 1 && (r = store_jobs(jobs, b.jobs, b.offs, st)) != MCS_OK) return r;
        int tpb = 0, bps = 0;
        if ((r = walk_residency(&q, b.mode, b.n > 1, &tpb, &bps)) != MCS_OK) return r;
        float best = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            MCS_CUDA(cudaMemsetAsync(b.launch_ctrl(), 0, sizeof(Ctrl), st));
            MCS_CUDA(cudaEventRecord(e0, st));
            if ((r = launch_walks(b.jobs, b.offs, b.n, b.n > 1 ? nullptr : &jobs[0], b.launch_ctrl(), &q, b.mode, tpb,
                                  bps, st)) != MCS_OK)
                return r;
            MCS_CUDA(cudaEventRecord(e1, st));
            MCS_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            MCS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            best = std::min(best, ms);
        }
        Ctrl hc;
        MCS_CUDA(cudaMemcpy(&hc, b.launch_ctrl(), sizeof(Ctrl), cudaMemcpyDeviceToHost));
        if (hc.err) {
            set_error(f + ": a device error during a tuning launch");
            return MCS_ERR_DEVICE;
        }
        if (count < max_trials) {
            trials[count].threads_per_block = tpb;
            trials[count].blocks_per_sm = bps;
            trials[count].queue_order = q.queue_order;
            trials[count].bvh_layout = use_wide(&q) ? 4 : 2;
            trials[count].lanes_per_query = trav_of(&q) == 2 ? 4 : 1;
            trials[count].ms = best;
        }
        count++;
        *ms = best;
        *bps_used = bps;
        return MCS_OK;
    };
    // coordinate search, largest effect first: queue order (row schedule and
    // mesh order), BVH node layout, residency (block size x blocks per SM).
    // A candidate replaces the incumbent only when it is faster by more than
    // kTuneMargin: differences below that are run-to-run noise of the sample
    // (measured +-5% between boxes on the 512-mesh batch; with a 2% margin the
    // sample once chose 64 x 16 threads per SM for a 3% gain, and the full
    // launch took 4.36 s against 3.89 s at 128 x 10)
    constexpr float kTuneMargin = 0.95f;
    mcs_params best = *p;
    best.queue_order = 0;
    best.bvh_layout = use_wide(p) ? 4 : 2;  // the library default unless the caller fixed one
    float best_ms = 1e30f;
    best.threads_per_block = 128;
    best.blocks_per_sm = 0;
    bool all_wide = true;
    for (int i = 0; i < n; i++) all_wide = all_wide && mcs_mesh_has_wide(items[i].mesh);
    best.lanes_per_query = trav_of(p) == 2 ? 4 : 1;
    // a batch always dispenses its meshes longest first (bit 1): that cuts
    // the tail of the shared queue, an effect that grows with the walks per
    // mesh and that the sample (1/64 of the walks) does not show -- on the
    // 512-mesh batch the sample preferred the caller's mesh order by 1-5%,
    // while the full launch took 4.10 s in that order against 3.90 s longest
    // first; only the row order within a mesh (bit 0) is tried
    for (int qo : {0, 1, 2, 3}) {
        if ((qo >= 2) != (n > 1)) continue;
        mcs_params q = best;
        q.queue_order = qo;
        float ms = 0.f;
        int used = 0;
        if ((s = trial(q, &ms, &used)) != MCS_OK) { cleanup(); return s; }
        if (ms < best_ms * kTuneMargin || best_ms == 1e30f) {
            best_ms = ms;
            best.queue_order = qo;
            best.blocks_per_sm = used;  // the default residency, stated
        }
    }
    const int layouts[3][2] = {{2, 1}, {4, 1}, {4, 4}};
    for (const auto &lq : layouts) {
        if (p->bvh_layout != 0 && lq[0] != best.bvh_layout) continue;
        if (p->lanes_per_query != 0 && lq[1] != best.lanes_per_query) continue;
        if (lq[0] == 4 && !all_wide) continue;
        if (lq[0] == best.bvh_layout && lq[1] == best.lanes_per_query) continue;  // the incumbent
        mcs_params q = best;
        q.bvh_layout = lq[0];
        q.lanes_per_query = lq[1];
        q.blocks_per_sm = 0;
        float ms = 0.f;
        int used = 0;
        if ((s = trial(q, &ms, &used)) != MCS_OK) { cleanup(); return s; }
        if (ms < best_ms * kTuneMargin) {
            best_ms = ms;
            best.bvh_layout = lq[0];
            best.lanes_per_query = lq[1];
            best.blocks_per_sm = used;
        }
    }
    for (int tpb : {64, 128}) {
        mcs_params q = best;
        q.threads_per_block = tpb;
        q.blocks_per_sm = 0;
        int t = 0, occ = 0;
        if ((s = walk_residency(&q, b.mode, n > 1, &t, &occ)) != MCS_OK) { cleanup(); return s; }
        // only the largest residency of each block size: the full launch is
        // latency-bound and wants every warp it can hold, while the sample's
        // tail (few walks per SM) favours fewer -- on the 512-mesh batch the
        // sample chose 128 x 8 and 64 x 16 over 128 x 10, whose full launches
        // took 4.36 s against 3.89 s
        for (int bps = occ; bps <= occ; bps++) {
            if (tpb == best.threads_per_block && bps == best.blocks_per_sm) continue;  // the incumbent
            q.blocks_per_sm = bps;
            float ms = 0.f;
            int used = 0;
            if ((s = trial(q, &ms, &used)) != MCS_OK) { cleanup(); return s; }
            if (ms < best_ms * kTuneMargin) { best_ms = ms; best.threads_per_block = tpb; best.blocks_per_sm = bps; }
        }
    }
    cleanup();
    *tuned = best;
    if (n_trials) *n_trials = count;
    return MCS_OK;
}

}  // extern "C"
