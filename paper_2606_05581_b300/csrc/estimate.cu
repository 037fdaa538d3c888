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
    int argmax_row;
    int pad;
};

struct Frame {
    double onemk, iw0, eps, rho_min_factor, rmax;
    int bisect_iters;
};

__device__ __forceinline__ double dist64(const DevMesh &m, double x, double y, double z, int *err) {
    Hit<double> h;
    closest<double>(m, x, y, z, -1, h, err);
    return sqrt(h.d2);
}

// ---------------------------------------------------------------- row schedule
__global__ void k_row_keys(const double *pos, int R, double lx, double ly, double lz, double ix, double iy, double iz,
                           unsigned long long *keys) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= R) return;
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
    keys[v] = ((unsigned long long)code << 32) | (unsigned)v;
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

__device__ __forceinline__ double wdist(const DevMesh &m, double x, double y, double z, int *front, int *err) {
    Hit<double> h;
    warp_query<double, kFull>(m, x, y, z, 0.0, h, front, err);
    return sqrt(h.d2);
}
__device__ __forceinline__ bool wclear(const DevMesh &m, double x, double y, double z, double thr, int *front,
                                       int *err) {
    Hit<double> h;
    return !warp_query<double, kBelow>(m, x, y, z, thr, h, front, err);
}

// rows v = i * stride, i = 0, 1, ... (stride 1: every row)
__global__ void __launch_bounds__(32 * kTanWarps) k_tangent_int(DevMesh m, const double *pos, const double *nrm, int R,
                                                                int stride, Frame fr, RowBall *ball, Ctrl *ctrl) {
    __shared__ int fronts[kTanWarps][32];
    const int v = (blockIdx.x * kTanWarps + (threadIdx.x >> 5)) * stride;
    if (v >= R) return;
    int *front = fronts[threadIdx.x >> 5];
    int err = 0;
    const double s0 = pos[3 * v], s1 = pos[3 * v + 1], s2 = pos[3 * v + 2];
    const double n0 = nrm[3 * v], n1 = nrm[3 * v + 1], n2 = nrm[3 * v + 2];
    const bool nz = (n0 != 0.0 || n1 != 0.0 || n2 != 0.0);
    RowBall b;
    b.c[0] = b.c[1] = b.c[2] = 0.0;
    b.n[0] = n0; b.n[1] = n1; b.n[2] = n2;
    b.rho = 0.0; b.r = 0.0; b.kfac = 1.0;
    if (nz) {
        const double rmax = fr.rmax;
        double r;
        if (wclear(m, s0 - rmax * n0, s1 - rmax * n1, s2 - rmax * n2, fr.onemk * rmax, front, &err)) {
            r = rmax;
        } else {
            double lo = 0.0, hi = rmax;
            for (int it = 0; it < fr.bisect_iters; it++) {
                const double mid = 0.5 * (lo + hi);
                if (wclear(m, s0 - mid * n0, s1 - mid * n1, s2 - mid * n2, fr.onemk * mid, front, &err)) lo = mid;
                else hi = mid;
            }
            r = lo;
        }
        b.c[0] = s0 - r * n0; b.c[1] = s1 - r * n1; b.c[2] = s2 - r * n2;
        b.rho = wdist(m, b.c[0], b.c[1], b.c[2], front, &err);
        b.r = r;
    }
    b.valid = nz && (b.rho >= fr.rho_min_factor * fr.eps);
    b.M = b.valid ? (fr.iw0 - 1.0) / (2.0 * b.rho) : 0.0;
    b.pad = 0;
    if ((threadIdx.x & 31) == 0) {
        ball[v] = b;
        if (err) atomicOr(&ctrl->err, err);
    }
}

// largest empty radius over rows 0, stride, 2 stride, ..., lowest row on ties
// -> inversion centre (any interior point serves; Sec. 4.3)
__global__ void k_origin_argmax(const RowBall *ball, int R, int stride, Ctrl *ctrl) {
    __shared__ double sv[1024];
    __shared__ int si[1024];
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
        ctrl->argmax_row = v;
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
__global__ void k_set_origin(Ctrl *ctrl, double x, double y, double z) {
    ctrl->origin[0] = x; ctrl->origin[1] = y; ctrl->origin[2] = z;
}

// Kelvin-inverted AABB of the vertices (radius clamp) and the radius of the
// empty ball at the inverted origin, 1 / max |v - o|
__global__ void k_ext_frame(const double *V, int nv, Ctrl *ctrl) {
    __shared__ double sm[7][256];
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
}

// exterior tangent ball: the inverted ball B(c~, r) (not containing 0) is the
// image of the primal ball with centre c~/(|c~|^2 - r^2) and radius
// r/(|c~|^2 - r^2); the accepted ball is replaced by the image of the primal
// empty ball B(C, dist(C))
__device__ bool inv_ball_ok(const DevMesh &m, const double st[3], const double nt[3], double r, const double o[3],
                            double onemk, int *front, int *err) {
    const double ct0 = st[0] - r * nt[0], ct1 = st[1] - r * nt[1], ct2 = st[2] - r * nt[2];
    const double cc = ct0 * ct0 + ct1 * ct1 + ct2 * ct2;
    const double den = cc - r * r;
    // clear of the inversion centre by a margin that keeps the primal image
    // ball (centre ~ 1/den) within FP64 resolution
    if (!(den > 1e-6 * cc)) return false;
    const double inv = 1.0 / den;
    const double C0 = ct0 * inv, C1 = ct1 * inv, C2 = ct2 * inv;
    const double Rp = r * inv;
    return wclear(m, C0 + o[0], C1 + o[1], C2 + o[2], onemk * Rp, front, err);
}

__global__ void __launch_bounds__(32 * kTanWarps) k_tangent_ext(DevMesh m, const double *pos, const double *nrm, int R,
                                                                Frame fr, RowBall *ball, Ctrl *ctrl) {
    __shared__ int fronts[kTanWarps][32];
    const int v = blockIdx.x * kTanWarps + (threadIdx.x >> 5);
    if (v >= R) return;
    int *front = fronts[threadIdx.x >> 5];
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
        if (inv_ball_ok(m, st, nt, rmax, o, fr.onemk, front, &err)) {
            r = rmax;
        } else {
            double lo = 0.0, hi = rmax;
            for (int it = 0; it < fr.bisect_iters; it++) {
                const double mid = 0.5 * (lo + hi);
                if (inv_ball_ok(m, st, nt, mid, o, fr.onemk, front, &err)) lo = mid;
                else hi = mid;
            }
            r = lo;
        }
        b.r = r;
        if (r > 0.0) {
            const double ct0 = st[0] - r * nt[0], ct1 = st[1] - r * nt[1], ct2 = st[2] - r * nt[2];
            const double cc = ct0 * ct0 + ct1 * ct1 + ct2 * ct2;
            const double den = cc - r * r;
            if (den > 1e-6 * cc) {
                const double invd = 1.0 / den;
                const double C0 = ct0 * invd, C1 = ct1 * invd, C2 = ct2 * invd;
                const double D = wdist(m, C0 + o[0], C1 + o[1], C2 + o[2], front, &err);
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

// ---------------------------------------------------------------- walks
struct WalkArgs {
    DevMesh m;
    const RowBall *ball;
    const int32_t *order;
    const int32_t *tri2bin;
    int32_t *exits;        // R x W, by sorted row position
    int32_t *exit_tri;     // optional, R x W by canonical row
    int32_t *H0;           // killing histogram
    Ctrl *ctrl;
    unsigned long long total;
    int R, W;
    uint32_t k0, k1;
    double eps, iw0;
    float eps2f;
    int max_steps;
    int killing;
};

__device__ __forceinline__ int exit_bin(const WalkArgs &a, int f, double b0, double b1, double b2) {
    if (a.tri2bin) return a.tri2bin[f];
    const int i0 = a.m.F[3 * f], i1 = a.m.F[3 * f + 1], i2 = a.m.F[3 * f + 2];
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
    unsigned long long wi;  // queue index
    int k;                  // next step number
    int prev;               // previous closest slot
    int v;                  // canonical row (-1: killing walk)
};

template <typename T, bool EXT, bool COUNT>
__global__ void __launch_bounds__(128, 6) k_walks(WalkArgs a) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const uint32_t k0 = a.k0, k1 = a.killing ? (a.k1 ^ kKillKeyXor) : a.k1;
    const double o64[3] = {EXT ? a.ctrl->origin[0] : 0.0, EXT ? a.ctrl->origin[1] : 0.0,
                           EXT ? a.ctrl->origin[2] : 0.0};
    const double r0max64 = EXT ? a.ctrl->rho0max : 0.0;
    const T oT[3] = {(T)o64[0], (T)o64[1], (T)o64[2]};
    const T r0maxT = (T)r0max64;
    const T epsT = sizeof(T) == 8 ? (T)a.eps : (T)a.eps2f;  // FP32: re-check below 2 eps
    unsigned long long *queue = a.killing ? &a.ctrl->kqueue : &a.ctrl->queue;
    WalkState<T> s;
    s.x = V3<T>{(T)0, (T)0, (T)0};
    s.g = 0; s.wi = 0; s.k = 1; s.prev = -1; s.v = -1;
    bool active = false, more = true;
    long long n_steps = 0, n_capped = 0, n_lost = 0;
    int err = 0;
    Work work{0ull, 0ull};

    auto finish = [&](int bin, int f, bool capped, bool lost) {
        n_capped += capped;
        n_lost += lost;
        if (bin >= a.R) { err |= kErrBin; bin = -1; }
        if (a.killing) {
            if (bin >= 0) atomicAdd(&a.H0[bin], 1);
        } else {
            const int rp = (int)(s.wi / (unsigned long long)a.W), j = (int)(s.wi % (unsigned long long)a.W);
            a.exits[(size_t)rp * a.W + j] = bin;
            if (a.exit_tri) a.exit_tri[(size_t)s.v * a.W + j] = f;
        }
        active = false;
    };

    while (true) {
        const bool need = !active && more;
        const unsigned nm = __ballot_sync(FULL, need);
        if (nm) {
            const int leader = __ffs(nm) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(queue, (unsigned long long)__popc(nm));
            base = __shfl_sync(FULL, base, leader);
            if (need) {
                const unsigned long long wi = base + __popc(nm & ((1u << lane) - 1u));
                if (wi >= a.total) {
                    more = false;
                } else if (a.killing) {
                    s.wi = wi; s.g = wi; s.v = -1; s.k = 1; s.prev = -1;
                    s.x = V3<T>{(T)0, (T)0, (T)0};
                    active = true;
                } else {
                    const int rp = (int)(wi / (unsigned long long)a.W), j = (int)(wi % (unsigned long long)a.W);
                    const int v = a.order[rp];
                    const RowBall &b = a.ball[v];
                    s.wi = wi;
                    s.v = v;
                    if (!b.valid) {
                        a.exits[(size_t)rp * a.W + j] = -1;
                        if (a.exit_tri) a.exit_tri[(size_t)v * a.W + j] = -1;
                    } else {
                        s.g = (unsigned long long)v * (unsigned long long)a.W + (unsigned long long)j;
                        const unsigned long long gp = s.g - (unsigned long long)(j & 1);
                        s.x = start_point<T>(k0, k1, gp, j & 1, (T)a.iw0, V3<T>{(T)b.c[0], (T)b.c[1], (T)b.c[2]},
                                             (T)b.rho, V3<T>{(T)b.n[0], (T)b.n[1], (T)b.n[2]});
                        s.k = 1;
                        s.prev = -1;
                        active = true;
                    }
                }
            }
        }
        if (!__any_sync(FULL, active || more)) break;
        if (!active) continue;

        // ---- one walk-on-spheres step
        T step;
        if (!EXT) {
            Hit<T> h;
            closest<T, COUNT>(a.m, s.x.x, s.x.y, s.x.z, s.prev, h, &err, &work);
            n_steps++;
            if (h.slot < 0 || h.id < 0 || h.id >= a.m.nf) {
                err |= kErrNoHit;
                record_nohit(a.ctrl, 1, a.killing, s.g, s.k, (double)s.x.x, (double)s.x.y, (double)s.x.z);
                finish(-1, -1, true, true);
                continue;
            }
            const T d = rsq<T>(h.d2);
            if (d < epsT || s.k == a.max_steps) {
                if (sizeof(T) == 8) {
                    finish(exit_bin(a, h.id, (double)h.b0, (double)h.b1, (double)h.b2), h.id, !(d < epsT), false);
                    continue;
                }
                double b[3];
                const double d64 = sqrt(recheck64(a.m, h.slot, (double)s.x.x, (double)s.x.y, (double)s.x.z, b));
                if (d64 < a.eps || s.k == a.max_steps) {
                    finish(exit_bin(a, h.id, b[0], b[1], b[2]), h.id, !(d64 < a.eps), false);
                    continue;
                }
            }
            s.prev = h.slot;
            step = d;
        } else {
            const T r2 = s.x.x * s.x.x + s.x.y * s.x.y + s.x.z * s.x.z;
            if (r2 == (T)0) {
                if (s.k == a.max_steps) { finish(-1, -1, true, true); continue; }
                step = r0maxT;
            } else {
                const T inv = (T)1 / r2;
                const T xp0 = s.x.x * inv, xp1 = s.x.y * inv, xp2 = s.x.z * inv;
                Hit<T> h;
                closest<T, COUNT>(a.m, xp0 + oT[0], xp1 + oT[1], xp2 + oT[2], s.prev, h, &err, &work);
                n_steps++;
                if (h.slot < 0 || h.id < 0 || h.id >= a.m.nf) {
                    err |= kErrNoHit;
                    record_nohit(a.ctrl, 2, a.killing, s.g, s.k, (double)s.x.x, (double)s.x.y, (double)s.x.z);
                    finish(-1, -1, true, true);
                    continue;
                }
                const T d = rsq<T>(h.d2);
                const T nx = rsq<T>(xp0 * xp0 + xp1 * xp1 + xp2 * xp2);
                const T ri = d / (nx * (nx + d));
                const T r0 = r0maxT - rsq<T>(r2);
                const T rho = ri > r0 ? ri : r0;
                if (rho < epsT || s.k == a.max_steps) {
                    if (sizeof(T) == 8) {
                        finish(exit_bin(a, h.id, (double)h.b0, (double)h.b1, (double)h.b2), h.id, !(rho < epsT), false);
                        continue;
                    }
                    const double xd0 = (double)s.x.x, xd1 = (double)s.x.y, xd2 = (double)s.x.z;
                    const double r2d = xd0 * xd0 + xd1 * xd1 + xd2 * xd2;
                    const double invd = 1.0 / r2d;
                    const double xpd0 = xd0 * invd, xpd1 = xd1 * invd, xpd2 = xd2 * invd;
                    double b[3];
                    const double dd = sqrt(recheck64(a.m, h.slot, xpd0 + o64[0], xpd1 + o64[1], xpd2 + o64[2], b));
                    const double nxd = sqrt(xpd0 * xpd0 + xpd1 * xpd1 + xpd2 * xpd2);
                    const double rid = dd / (nxd * (nxd + dd));
                    const double r0d = r0max64 - sqrt(r2d);
                    const double rhod = rid > r0d ? rid : r0d;
                    if (rhod < a.eps || s.k == a.max_steps) {
                        finish(exit_bin(a, h.id, b[0], b[1], b[2]), h.id, !(rhod < a.eps), false);
                        continue;
                    }
                }
                s.prev = h.slot;
                step = rho;
            }
        }
        const V3<T> u = direction<T>(k0, k1, s.g, (uint32_t)s.k);
        s.x.x = s.x.x + step * u.x;
        s.x.y = s.x.y + step * u.y;
        s.x.z = s.x.z + step * u.z;
        s.k++;
    }
    // per-warp reduction of the counters
    for (int off = 16; off > 0; off >>= 1) {
        n_steps += __shfl_down_sync(FULL, n_steps, off);
        n_capped += __shfl_down_sync(FULL, n_capped, off);
        n_lost += __shfl_down_sync(FULL, n_lost, off);
        err |= __shfl_down_sync(FULL, err, off);
        if (COUNT) {
            work.nodes += __shfl_down_sync(FULL, work.nodes, off);
            work.tris += __shfl_down_sync(FULL, work.tris, off);
        }
    }
    if (lane == 0) {
        if (COUNT) {
            atomicAdd(&a.ctrl->nodes, work.nodes);
            atomicAdd(&a.ctrl->tris, work.tris);
        }
        if (a.killing) {
            atomicAdd(&a.ctrl->kill_steps, (unsigned long long)n_steps);
            atomicAdd(&a.ctrl->kill_capped, (unsigned long long)n_capped);
            atomicAdd(&a.ctrl->kill_lost, (unsigned long long)n_lost);
        } else {
            atomicAdd(&a.ctrl->steps, (unsigned long long)n_steps);
            atomicAdd(&a.ctrl->capped, (unsigned long long)n_capped);
            atomicAdd(&a.ctrl->lost, (unsigned long long)n_lost);
        }
        if (err) atomicOr(&a.ctrl->err, err);
    }
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
__global__ void __launch_bounds__(kHistThreads) k_histogram(const int32_t *exits, const int32_t *order,
                                                           const RowBall *ball, const double *area, const double *cf,
                                                           int R, int W, int cap, int32_t *hbin, int32_t *hcnt,
                                                           int32_t *hnnz, double *Lambda, double *omega_out,
                                                           Ctrl *ctrl) {
    extern __shared__ int hist[];
    typedef cub::BlockScan<int, kHistThreads> Scan;
    __shared__ typename Scan::TempStorage scan_tmp;
    const int rp = blockIdx.x;
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

// Lambda <- -(D + D^T)/2 off the diagonal, by 32 x 32 tile pairs (I <= J)
__global__ void k_symmetrize(double *L, int R) {
    __shared__ double A[32][33], B[32][33];
    const int I = blockIdx.y, J = blockIdx.x;
    if (I > J) return;
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

// Laplacian diagonal: Lambda_vv = sum_{u != v} Wsym_vu (+ killing 4 pi cf_v H0_v / N0)
__global__ void k_diagonal(double *L, int R, const double *cf, const int32_t *H0, double inv_n0) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= R) return;
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

// ---------------------------------------------------------------- workspace
struct Layout {
    size_t ball, keys, keys_s, order, exits, H0, cf, ctrl, sort, total;
    size_t sort_bytes;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static Layout layout(int R, int W) {
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
    L.ctrl = take(sizeof(Ctrl));
    size_t sb = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, sb, (unsigned long long *)nullptr, (unsigned long long *)nullptr, R, 0, 62);
    L.sort_bytes = sb;
    L.sort = take(sb);
    L.total = o;
    return L;
}

}  // namespace mcs

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
}

size_t mcs_estimate_workspace_size(mcs_mesh m, int n_rows, int walks_per_row, long long killing_walks) {
    (void)m; (void)killing_walks;
    if (n_rows <= 0 || walks_per_row <= 0) return 0;
    return layout(n_rows, walks_per_row).total;
}

mcs_status mcs_estimate_dtn(mcs_mesh m, const mcs_rows *rows, const mcs_params *p, const mcs_outputs *out,
                            void *workspace, size_t workspace_bytes, mcs_stats *stats, void *stream_) {
    MCS_ARG(m && rows && p && out, "mcs_estimate_dtn: NULL mesh, rows, params or outputs");
    const int R = rows->n_rows, W = p->walks_per_row;
    MCS_ARG(R > 0, "mcs_estimate_dtn: n_rows must be positive");
    MCS_ARG(rows->pos && rows->nrm && rows->area, "mcs_estimate_dtn: NULL row arrays");
    MCS_ARG(rows->tri2bin != nullptr || R == m->nv, "mcs_estimate_dtn: vertex rows need n_rows == nv");
    MCS_ARG(W > 0 && W % 2 == 0, "mcs_estimate_dtn: walks_per_row must be a positive even number");
    MCS_ARG((long long)R * W < (1LL << 40), "mcs_estimate_dtn: too many walks");
    MCS_ARG(p->eps > 0.0 && std::isfinite(p->eps), "mcs_estimate_dtn: eps must be positive");
    MCS_ARG(p->cap_deg > 0.0 && p->cap_deg < 180.0, "mcs_estimate_dtn: cap_deg must be in (0, 180)");
    MCS_ARG(p->bisect_iters >= 0 && p->bisect_iters <= 60, "mcs_estimate_dtn: bisect_iters out of range");
    MCS_ARG(p->max_steps >= 2, "mcs_estimate_dtn: max_steps must be >= 2");
    MCS_ARG(p->prec == MCS_FP32 || p->prec == MCS_FP64, "mcs_estimate_dtn: prec must be 32 or 64");
    MCS_ARG(p->domain == MCS_INTERIOR || p->domain == MCS_EXTERIOR, "mcs_estimate_dtn: bad domain");
    MCS_ARG(p->killing_walks >= 0, "mcs_estimate_dtn: killing_walks < 0");
    MCS_ARG(out->hist_bin && out->hist_cnt && out->hist_nnz, "mcs_estimate_dtn: NULL histogram outputs");
    MCS_ARG((size_t)R * sizeof(int) <= 200 * 1024, "mcs_estimate_dtn: more than 51200 rows per estimate");
    const Layout L = layout(R, W);
    MCS_ARG(workspace != nullptr && workspace_bytes >= L.total, "mcs_estimate_dtn: workspace too small");
    MCS_ARG(((uintptr_t)workspace & 255) == 0, "mcs_estimate_dtn: workspace must be 256-byte aligned");
    const bool ext = p->domain == MCS_EXTERIOR;
    const double kappa = p->kappa >= 0.0 ? p->kappa : (rows->tri2bin ? 1e-6 : 0.05);
    MCS_ARG(kappa < 1.0, "mcs_estimate_dtn: kappa must be < 1");

    cudaStream_t st = as_stream(stream_);
    char *ws = (char *)workspace;
    RowBall *ball = (RowBall *)(ws + L.ball);
    unsigned long long *keys = (unsigned long long *)(ws + L.keys), *keys_s = (unsigned long long *)(ws + L.keys_s);
    int32_t *order = (int32_t *)(ws + L.order);
    int32_t *exits = (int32_t *)(ws + L.exits);
    int32_t *H0 = out->H0 ? out->H0 : (int32_t *)(ws + L.H0);
    double *cf = ext ? (double *)(ws + L.cf) : nullptr;
    Ctrl *ctrl = (Ctrl *)(ws + L.ctrl);
    const DevMesh dm = m->dev();

    Frame fr;
    fr.onemk = 1.0 - kappa;
    fr.iw0 = 1.0 / sin(p->cap_deg * (M_PI / 360.0));
    fr.eps = p->eps;
    fr.rho_min_factor = p->rho_min_factor;
    fr.rmax = m->rmax;
    fr.bisect_iters = p->bisect_iters;

    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    const bool timing = stats && p->timing;
    if (timing)
        for (auto &e : ev) MCS_CUDA(cudaEventCreate(&e));
    auto mark = [&](int i) { if (timing) cudaEventRecord(ev[i], st); };
    mark(0);
    MCS_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st));
    MCS_CUDA(cudaMemsetAsync(H0, 0, sizeof(int32_t) * R, st));
    const int tb = 128, gr = (R + tb - 1) / tb;
    // Z-order row schedule
    double inv[3];
    for (int k = 0; k < 3; k++) inv[k] = 1.0 / (m->hi[k] - m->lo[k]);
    k_row_keys<<<gr, tb, 0, st>>>(rows->pos, R, m->lo[0], m->lo[1], m->lo[2], inv[0], inv[1], inv[2], keys);
    size_t sb = L.sort_bytes;
    MCS_CUDA(cub::DeviceRadixSort::SortKeys(ws + L.sort, sb, keys, keys_s, R, 0, 62, st));
    k_order_from_keys<<<gr, tb, 0, st>>>(keys_s, R, order);
    // tangent balls
    if (ext) {
        if (p->origin_auto) {
            const int ostride = (R + 255) / 256, nsub = (R + ostride - 1) / ostride;
            k_tangent_int<<<(nsub + kTanWarps - 1) / kTanWarps, 32 * kTanWarps, 0, st>>>(dm, rows->pos, rows->nrm, R,
                                                                                        ostride, fr, ball, ctrl);
            k_origin_argmax<<<1, 1024, 0, st>>>(ball, R, ostride, ctrl);
        } else {
            k_set_origin<<<1, 1, 0, st>>>(ctrl, p->origin[0], p->origin[1], p->origin[2]);
        }
        k_ext_frame<<<1, 256, 0, st>>>(m->V, m->nv, ctrl);
        k_tangent_ext<<<(R + kTanWarps - 1) / kTanWarps, 32 * kTanWarps, 0, st>>>(dm, rows->pos, rows->nrm, R, fr,
                                                                                 ball, ctrl);
        k_colfactor<<<gr, tb, 0, st>>>(rows->pos, R, ctrl, cf);
    } else {
        k_tangent_int<<<(R + kTanWarps - 1) / kTanWarps, 32 * kTanWarps, 0, st>>>(dm, rows->pos, rows->nrm, R, 1, fr,
                                                                                 ball, ctrl);
    }
    MCS_CUDA(cudaGetLastError());
    // walks
    WalkArgs a;
    a.m = dm;
    a.ball = ball;
    a.order = order;
    a.tri2bin = rows->tri2bin;
    a.exits = exits;
    a.exit_tri = out->exit_tri;
    a.H0 = H0;
    a.ctrl = ctrl;
    a.total = (unsigned long long)R * (unsigned long long)W;
    a.R = R;
    a.W = W;
    a.k0 = (uint32_t)p->seed;
    a.k1 = (uint32_t)(p->seed >> 32);
    a.eps = p->eps;
    a.iw0 = fr.iw0;
    a.eps2f = (float)(2.0 * p->eps);
    a.max_steps = p->max_steps;
    a.killing = 0;
    void (*kern)(WalkArgs) = nullptr;
    if (p->count_work) {
        if (p->prec == MCS_FP64) kern = ext ? k_walks<double, true, true> : k_walks<double, false, true>;
        else kern = ext ? k_walks<float, true, true> : k_walks<float, false, true>;
    } else {
        if (p->prec == MCS_FP64) kern = ext ? k_walks<double, true, false> : k_walks<double, false, false>;
        else kern = ext ? k_walks<float, true, false> : k_walks<float, false, false>;
    }
    const int tpb = 128;
    int occ = 0;
    MCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, tpb, 0));
    const int bps = p->blocks_per_sm > 0 ? p->blocks_per_sm : std::max(1, occ);
    const int grid = num_sms() * bps;
    mark(1);
    kern<<<grid, tpb, 0, st>>>(a);
    if (ext && p->killing_walks > 0) {
        a.killing = 1;
        a.total = (unsigned long long)p->killing_walks;
        kern<<<grid, tpb, 0, st>>>(a);
    }
    MCS_CUDA(cudaGetLastError());
    // histogram, row normalisation, assembly
    mark(2);
    if (out->Lambda) {
        const size_t nn = (size_t)R * R;
        k_fill_zero<<<num_sms() * 8, 256, 0, st>>>(out->Lambda, nn);
    }
    const size_t smem = sizeof(int) * (size_t)R;
    MCS_CUDA(cudaFuncSetAttribute(k_histogram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 1024)));
    k_histogram<<<R, kHistThreads, smem, st>>>(exits, order, ball, rows->area, cf, R, W, std::min(W, R), out->hist_bin,
                                             out->hist_cnt, out->hist_nnz, out->Lambda, out->omega, ctrl);
    mark(3);
    if (out->Lambda) {
        const int nt = (R + 31) / 32;
        k_symmetrize<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(out->Lambda, R);
        const bool kill = ext && p->killing_walks > 0;
        k_diagonal<<<(R * 32 + 255) / 256, 256, 0, st>>>(out->Lambda, R, cf, kill ? H0 : nullptr,
                                                        kill ? 1.0 / (double)p->killing_walks : 0.0);
    }
    mark(4);
    MCS_CUDA(cudaGetLastError());
    if (!stats) return MCS_OK;
    Ctrl hc;
    MCS_CUDA(cudaMemcpyAsync(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    MCS_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < 4; i++) {
        stats->phase_ms[i] = 0.f;
        if (timing) cudaEventElapsedTime(&stats->phase_ms[i], ev[i], ev[i + 1]);
    }
    if (timing)
        for (auto &e : ev) cudaEventDestroy(e);
    stats->nodes_visited = (long long)hc.nodes;
    stats->tris_tested = (long long)hc.tris;
    stats->walks = (long long)R * W;
    stats->steps = (long long)hc.steps;
    stats->capped = (long long)hc.capped;
    stats->lost = (long long)hc.lost;
    stats->discarded_rows = hc.discarded;
    stats->killing_steps = (long long)hc.kill_steps;
    stats->killing_capped = (long long)hc.kill_capped;
    for (int k = 0; k < 3; k++) stats->origin[k] = ext ? hc.origin[k] : 0.0;
    stats->rmax = ext ? hc.rmax_ext : m->rmax;
    stats->device_error = hc.err;
    if (hc.err & kErrNoOrigin) {
        set_error("mcs_estimate_dtn: no interior tangent ball to place the inversion centre");
        return MCS_ERR_NO_INTERIOR_POINT;
    }
    if (hc.err & kErrNoHit) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "mcs_estimate_dtn: a walk query found no triangle (kind %d, killing %d, walk %llu, step %d, "
                 "x~ = (%.9g, %.9g, %.9g)); walk retired as lost",
                 hc.diag_kind, hc.diag_killing, hc.diag_walk, hc.diag_step, hc.diag_p[0], hc.diag_p[1], hc.diag_p[2]);
        set_error(buf);
        return MCS_ERR_DEVICE;
    }
    if (hc.err) {
        set_error(hc.err & kErrBin ? "mcs_estimate_dtn: tri2bin maps a triangle outside [0, n_rows)"
                                   : "mcs_estimate_dtn: BVH traversal stack or iteration bound exceeded");
        return MCS_ERR_DEVICE;
    }
    return (hc.capped || hc.kill_capped) ? MCS_WARN_CAPPED : MCS_OK;
}

}  // extern "C"
