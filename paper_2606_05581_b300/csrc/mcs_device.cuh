// mcs_device.cuh -- device-side building blocks of the DtN estimator:
// Philox-4x32-10, exact uniforms, samplers, point-triangle closest point,
// BVH layout and closest-point traversal.
//
// Every floating-point expression that decides a walk (sampler, step,
// closest point, tangent ball) is written in a fixed operation order and the
// library is compiled with -fmad=false, IEEE division and square root, so
// FP64 (and FP32) walks are reproducible operation for operation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mcs {

constexpr uint32_t kTagRadial = 0xFFFFFFFFu;
constexpr uint32_t kKillKeyXor = 0x4B494C4Cu;
constexpr int kMaxReject = 32;
constexpr int kStackDepth = 64;

// device status word bits
constexpr int kErrStack = 1;       // traversal stack full (a far child was dropped)
constexpr int kErrNoOrigin = 2;    // exterior: no interior tangent ball for the inversion centre
constexpr int kErrTree = 4;        // traversal / refit exceeded its iteration bound
constexpr int kErrBin = 8;         // an exit bin outside [0, n_rows)
constexpr int kErrNoHit = 64;      // a walk query found no triangle (non-finite point); walk retired as lost

// --------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products, key bumped by the Weyl constants after each.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// uniforms on (0,1): (2k+1) 2^-53 from 52 bits, (2k+1) 2^-24 from 23 bits
__device__ __forceinline__ double uni64(uint32_t hi, uint32_t lo) {
    const unsigned long long b = ((((unsigned long long)hi) << 32) | lo) >> 12;
    return (double)b * (1.0 / 4503599627370496.0) + (1.0 / 9007199254740992.0);
}
__device__ __forceinline__ float uni32(uint32_t x) {
    return (float)(x >> 9) * (1.0f / 8388608.0f) + (1.0f / 16777216.0f);
}

template <typename T> struct Uni;
template <> struct Uni<double> {
    // signed pair (a, b) in (-1,1)^2 from one Philox block
    __device__ static void pair(uint4 x, double &a, double &b) {
        a = 2.0 * uni64(x.x, x.y) - 1.0;
        b = 2.0 * uni64(x.z, x.w) - 1.0;
    }
    __device__ static double one(uint4 x) { return uni64(x.x, x.y); }
};
template <> struct Uni<float> {
    __device__ static void pair(uint4 x, float &a, float &b) {
        a = 2.0f * uni32(x.x) - 1.0f;
        b = 2.0f * uni32(x.z) - 1.0f;
    }
    __device__ static float one(uint4 x) { return uni32(x.x); }
};

template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ double rsq<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float rsq<float>(float x) { return sqrtf(x); }

template <typename T> struct V3 { T x, y, z; };

// uniform direction on S^2, Marsaglia (1972): (a,b) uniform in the square,
// accept a^2+b^2 < 1, u = (2a sqrt(1-s), 2b sqrt(1-s), 1-2s)
template <typename T>
__device__ __forceinline__ V3<T> direction(uint32_t k0, uint32_t k1, unsigned long long g, uint32_t step) {
    for (uint32_t t = 0; t < (uint32_t)kMaxReject; t++) {
        const uint4 x = philox(make_uint4((uint32_t)g, (uint32_t)(g >> 32), step, t), k0, k1);
        T a, b;
        Uni<T>::pair(x, a, b);
        const T s = a * a + b * b;
        if (s < (T)1) {
            const T h = rsq<T>((T)1 - s);
            return V3<T>{(T)2 * a * h, (T)2 * b * h, (T)1 - (T)2 * s};
        }
    }
    return V3<T>{(T)0, (T)0, (T)1};
}

// orthonormal basis of a unit n (Duff et al., JCGT 6(1) 2017)
template <typename T>
__device__ __forceinline__ void onb(V3<T> n, V3<T> &e1, V3<T> &e2) {
    const T sg = copysign((T)1, n.z);
    const T a = (T)-1 / (sg + n.z);
    const T b = n.x * n.y * a;
    e1 = V3<T>{(T)1 + sg * n.x * n.x * a, sg * b, -(sg * n.x)};
    e2 = V3<T>{b, sg + n.y * n.y * a, -n.y};
}

// Start point of walk pair gp on the empty ball B(c, rho), pole c + rho n:
// w = sin(theta/2) drawn with density ~1/w^2 on [w0, 1] (the ball jump
// kernel outside the cap), azimuth uniform, odd partner at phi + pi.
template <typename T>
__device__ __forceinline__ V3<T> start_point(uint32_t k0, uint32_t k1, unsigned long long gp, int odd, T iw0,
                                             V3<T> c, T rho, V3<T> n, int mode = 0, double iw0d = 0.0,
                                             double *q = nullptr) {
    const uint4 xr = philox(make_uint4((uint32_t)gp, (uint32_t)(gp >> 32), 0u, kTagRadial), k0, k1);
    const T u = Uni<T>::one(xr);
    T w, cth;
    if (mode == 0) {
        // w = sin(theta/2) with pdf ~ 1/w^2 on [w0, 1]: J^B importance sampling
        const T iw = iw0 - u * (iw0 - (T)1);
        w = (T)1 / iw;
        cth = (T)1 - (T)2 * (w * w);
        if (q) *q = 1.0;
    } else {
        // cos(theta) uniform on [-1, cos(theta0)] (mode 1) or [-1, 1] (mode 2);
        // mode 1 walks carry q = |dB outside the cap| J^B(p, z) / M
        const T w0 = (T)1 / iw0;
        const T c0 = mode == 1 ? (T)1 - (T)2 * (w0 * w0) : (T)1;
        cth = c0 - u * (c0 + (T)1);
        w = rsq<T>(((T)1 - cth) * (T)0.5);
        if (q) {
            const double wd = (double)w, w0d = 1.0 / iw0d;
            *q = mode == 1 ? (1.0 - w0d * w0d) / (2.0 * (wd * wd * wd) * (iw0d - 1.0)) : 1.0;
        }
    }
    const T sth = ((T)2 * w) * rsq<T>((T)1 - w * w);
    T cph = (T)1, sph = (T)0;
    for (uint32_t t = 0; t < (uint32_t)kMaxReject; t++) {
        const uint4 x = philox(make_uint4((uint32_t)gp, (uint32_t)(gp >> 32), 0u, t), k0, k1);
        T a, b;
        Uni<T>::pair(x, a, b);
        const T s = a * a + b * b;
        if (s < (T)1) {
            const T r = rsq<T>(s);
            cph = a / r;
            sph = b / r;
            break;
        }
    }
    if (odd) { cph = -cph; sph = -sph; }
    V3<T> e1, e2;
    onb<T>(n, e1, e2);
    V3<T> z;
    z.x = c.x + rho * (cth * n.x + sth * (cph * e1.x + sph * e2.x));
    z.y = c.y + rho * (cth * n.y + sth * (cph * e1.y + sph * e2.y));
    z.z = c.z + rho * (cth * n.z + sth * (cph * e1.z + sph * e2.z));
    return z;
}

// --------------------------------------------------------------------------
// point-triangle closest point on (a, ab, ac): Voronoi-region tests on dot
// products (Ericson, Real-Time Collision Detection, Sec. 5.1.5), with
// bp = ap - ab, cp = ap - ac; zero-length edge regions take parameter 0; a
// zero normal, or a failed interior test, falls back to the nearest edge.
// Returns |p - q|^2 and the barycentrics of q.
// --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T dot3(T a0, T a1, T a2, T b0, T b1, T b2) { return a0 * b0 + a1 * b1 + a2 * b2; }

template <typename T>
__device__ __forceinline__ T seg_closest(T o0, T o1, T o2, T e0, T e1, T e2, T tnum, T &t) {
    const T L = e0 * e0 + e1 * e1 + e2 * e2;
    T tt = L > (T)0 ? tnum / L : (T)0;
    if (!(tt > (T)0)) tt = (T)0;
    if (tt > (T)1) tt = (T)1;
    const T d0 = o0 - tt * e0, d1 = o1 - tt * e1, d2 = o2 - tt * e2;
    t = tt;
    return d0 * d0 + d1 * d1 + d2 * d2;
}

template <typename T>
__device__ __noinline__ T tri_degenerate(T ap0, T ap1, T ap2, T ab0, T ab1, T ab2, T ac0, T ac1, T ac2, T *bary) {
    const T bp0 = ap0 - ab0, bp1 = ap1 - ab1, bp2 = ap2 - ab2;
    const T bc0 = ac0 - ab0, bc1 = ac1 - ab1, bc2 = ac2 - ab2;
    const T d1 = ab0 * ap0 + ab1 * ap1 + ab2 * ap2;
    const T d2 = ac0 * ap0 + ac1 * ap1 + ac2 * ap2;
    T t;
    T best = seg_closest<T>(ap0, ap1, ap2, ab0, ab1, ab2, d1, t);
    bary[0] = (T)1 - t; bary[1] = t; bary[2] = (T)0;
    T cur = seg_closest<T>(ap0, ap1, ap2, ac0, ac1, ac2, d2, t);
    if (cur < best) { best = cur; bary[0] = (T)1 - t; bary[1] = (T)0; bary[2] = t; }
    const T dbc = bc0 * bp0 + bc1 * bp1 + bc2 * bp2;
    cur = seg_closest<T>(bp0, bp1, bp2, bc0, bc1, bc2, dbc, t);
    if (cur < best) { best = cur; bary[0] = (T)0; bary[1] = (T)1 - t; bary[2] = t; }
    return best;
}

// the Voronoi-region tests of a triangle with a nonzero normal (ap = p - a)
template <typename T>
__device__ __forceinline__ T tri_regions(T ap0, T ap1, T ap2, T ab0, T ab1, T ab2, T ac0, T ac1, T ac2, T *bary) {
    const T d1 = ab0 * ap0 + ab1 * ap1 + ab2 * ap2;
    const T d2 = ac0 * ap0 + ac1 * ap1 + ac2 * ap2;
    if (d1 <= (T)0 && d2 <= (T)0) {
        bary[0] = (T)1; bary[1] = (T)0; bary[2] = (T)0;
        return ap0 * ap0 + ap1 * ap1 + ap2 * ap2;
    }
    const T bp0 = ap0 - ab0, bp1 = ap1 - ab1, bp2 = ap2 - ab2;
    const T d3 = ab0 * bp0 + ab1 * bp1 + ab2 * bp2;
    const T d4 = ac0 * bp0 + ac1 * bp1 + ac2 * bp2;
    if (d3 >= (T)0 && d4 <= d3) {
        bary[0] = (T)0; bary[1] = (T)1; bary[2] = (T)0;
        return bp0 * bp0 + bp1 * bp1 + bp2 * bp2;
    }
    const T vc = d1 * d4 - d3 * d2;
    if (vc <= (T)0 && d1 >= (T)0 && d3 <= (T)0) {
        const T den = d1 - d3;
        const T v = den > (T)0 ? d1 / den : (T)0;
        const T q0 = ap0 - v * ab0, q1 = ap1 - v * ab1, q2 = ap2 - v * ab2;
        bary[0] = (T)1 - v; bary[1] = v; bary[2] = (T)0;
        return q0 * q0 + q1 * q1 + q2 * q2;
    }
    const T cp0 = ap0 - ac0, cp1 = ap1 - ac1, cp2 = ap2 - ac2;
    const T d5 = ab0 * cp0 + ab1 * cp1 + ab2 * cp2;
    const T d6 = ac0 * cp0 + ac1 * cp1 + ac2 * cp2;
    if (d6 >= (T)0 && d5 <= d6) {
        bary[0] = (T)0; bary[1] = (T)0; bary[2] = (T)1;
        return cp0 * cp0 + cp1 * cp1 + cp2 * cp2;
    }
    const T vb = d5 * d2 - d1 * d6;
    if (vb <= (T)0 && d2 >= (T)0 && d6 <= (T)0) {
        const T den = d2 - d6;
        const T w = den > (T)0 ? d2 / den : (T)0;
        const T q0 = ap0 - w * ac0, q1 = ap1 - w * ac1, q2 = ap2 - w * ac2;
        bary[0] = (T)1 - w; bary[1] = (T)0; bary[2] = w;
        return q0 * q0 + q1 * q1 + q2 * q2;
    }
    const T va = d3 * d6 - d5 * d4;
    const T e43 = d4 - d3, e56 = d5 - d6;
    if (va <= (T)0 && e43 >= (T)0 && e56 >= (T)0) {
        const T den = e43 + e56;
        const T w = den > (T)0 ? e43 / den : (T)0;
        const T bc0 = ac0 - ab0, bc1 = ac1 - ab1, bc2 = ac2 - ab2;
        const T q0 = bp0 - w * bc0, q1 = bp1 - w * bc1, q2 = bp2 - w * bc2;
        bary[0] = (T)0; bary[1] = (T)1 - w; bary[2] = w;
        return q0 * q0 + q1 * q1 + q2 * q2;
    }
    const T den = (va + vb) + vc;
    if (den > (T)0) {
        const T inv = (T)1 / den;
        const T v = vb * inv, w = vc * inv;
        const T q0 = (ap0 - v * ab0) - w * ac0;
        const T q1 = (ap1 - v * ab1) - w * ac1;
        const T q2 = (ap2 - v * ab2) - w * ac2;
        bary[0] = ((T)1 - v) - w; bary[1] = v; bary[2] = w;
        return q0 * q0 + q1 * q1 + q2 * q2;
    }
    return tri_degenerate<T>(ap0, ap1, ap2, ab0, ab1, ab2, ac0, ac1, ac2, bary);
}

// a zero normal (n = ab x ac, every component exactly 0 in T) marks a
// degenerate triangle, whose closest point is on its nearest edge
template <typename T>
__device__ __forceinline__ bool tri_zero_normal(T ab0, T ab1, T ab2, T ac0, T ac1, T ac2) {
    const T n0 = ab1 * ac2 - ab2 * ac1;
    const T n1 = ab2 * ac0 - ab0 * ac2;
    const T n2 = ab0 * ac1 - ab1 * ac0;
    return n0 == (T)0 && n1 == (T)0 && n2 == (T)0;
}

template <typename T>
__device__ __forceinline__ T tri_closest(T p0, T p1, T p2, T a0, T a1, T a2, T ab0, T ab1, T ab2, T ac0, T ac1, T ac2,
                                         T *bary) {
    const T ap0 = p0 - a0, ap1 = p1 - a1, ap2 = p2 - a2;
    if (tri_zero_normal<T>(ab0, ab1, ab2, ac0, ac1, ac2))
        return tri_degenerate<T>(ap0, ap1, ap2, ab0, ab1, ab2, ac0, ac1, ac2, bary);
    return tri_regions<T>(ap0, ap1, ap2, ab0, ab1, ab2, ac0, ac1, ac2, bary);
}

// --------------------------------------------------------------------------
// mesh on the device
// --------------------------------------------------------------------------
// binary BVH node: both children's boxes (float, rounded outward) + children
// (>= 0 internal node, < 0 leaf: ~k = triangle slot in BVH order)
struct __align__(16) Node {
    float4 a;  // lo0.x lo0.y lo0.z hi0.x
    float4 b;  // hi0.y hi0.z lo1.x lo1.y
    float4 c;  // lo1.z hi1.x hi1.y hi1.z
    int4 d;    // child0 child1 - -
};
// 4-wide node: the binary tree collapsed two levels at a time (the nodes
// at even depth keep their grandchildren), one 128-byte line per node.
// Child boxes in SoA order; child k >= 0 internal 4-wide node, < 0 leaf
// (~slot), kNoChild unused (its box is empty: lo = +inf, hi = -inf)
constexpr int kNoChild = 0x7FFFFFFF;
struct __align__(128) Node4 {
    float4 lox, loy, loz, hix, hiy, hiz;
    int4 child;
    int4 pad;
};
// triangle slot in BVH order, FP32: (a, id) (ab, zero-normal flag) (ac, -);
// the flag (an int in ab.w) is tri_zero_normal of the float ab, ac
struct __align__(16) Tri32 {
    float4 a;
    float4 ab;
    float4 ac;
};
// triangle slot in BVH order, FP64
struct __align__(16) Tri64 {
    double a[3], ab[3], ac[3];
    int id, pad;
};

struct DevMesh {
    const double *V;       // nv x 3
    const int32_t *F;      // nf x 3
    const Node *nodes;     // nf - 1 internal nodes (root 0); none when nf == 1
    const Node4 *nodes4;   // the same tree, 4-wide (root 0); none when nf == 1
    const Tri32 *t32;      // nf slots
    const Tri64 *t64;      // nf slots
    int nv, nf;
    float scale;           // max |coordinate| of the mesh, for the pruning slack
};

template <typename T> struct Hit {
    T d2;
    int id;    // original triangle id
    int slot;  // BVH slot
    T b0, b1, b2;
};

template <typename T> struct Slot;
template <> struct Slot<float> {
    __device__ static float test(const DevMesh &m, int s, float px, float py, float pz, float *b, int &id) {
        const Tri32 t = m.t32[s];
        id = __float_as_int(t.a.w);
        // tri_closest with the normal test taken from the slot's flag
        const float ap0 = px - t.a.x, ap1 = py - t.a.y, ap2 = pz - t.a.z;
        if (__float_as_int(t.ab.w) != 0)
            return tri_degenerate<float>(ap0, ap1, ap2, t.ab.x, t.ab.y, t.ab.z, t.ac.x, t.ac.y, t.ac.z, b);
        return tri_regions<float>(ap0, ap1, ap2, t.ab.x, t.ab.y, t.ab.z, t.ac.x, t.ac.y, t.ac.z, b);
    }
};
template <> struct Slot<double> {
    __device__ static double test(const DevMesh &m, int s, double px, double py, double pz, double *b, int &id) {
        const Tri64 &t = m.t64[s];
        id = t.id;
        return tri_closest<double>(px, py, pz, t.a[0], t.a[1], t.a[2], t.ab[0], t.ab[1], t.ab[2], t.ac[0], t.ac[1],
                                   t.ac[2], b);
    }
};

// relative pruning slack: a node is skipped only when its box is farther
// than the best distance plus tau = rel * (scale + |p|_inf), which bounds
// the rounding of the box and triangle distance computations, so the
// traversal returns exactly the brute-force argmin of (d^2, id)
template <typename T> __device__ __forceinline__ T prune_rel();
template <> __device__ __forceinline__ float prune_rel<float>() { return 6.103515625e-05f; }        // 2^-14
template <> __device__ __forceinline__ double prune_rel<double>() { return 1.4551915228366852e-11; } // 2^-36

template <typename T>
__device__ __forceinline__ T box_d2(T px, T py, T pz, float lx, float ly, float lz, float hx, float hy, float hz) {
    const T dx = fmax(fmax((T)lx - px, (T)0), px - (T)hx);
    const T dy = fmax(fmax((T)ly - py, (T)0), py - (T)hy);
    const T dz = fmax(fmax((T)lz - pz, (T)0), pz - (T)hz);
    return dx * dx + dy * dy + dz * dz;
}

template <typename T> __device__ __forceinline__ float store_down(T x);
template <> __device__ __forceinline__ float store_down<float>(float x) { return x; }
template <> __device__ __forceinline__ float store_down<double>(double x) { return __double2float_rd(x); }

// optional work counters of a traversal
struct Work {
    unsigned long long nodes, tris;
};

// closest triangle by traversal of the binary BVH (nearest child first,
// explicit stack); guess >= 0 is a slot tested first to tighten the bound
template <typename T, bool COUNT = false>
__device__ void closest(const DevMesh &m, T px, T py, T pz, int guess, Hit<T> &best, int *err, Work *work = nullptr) {
    best.d2 = (T)INFINITY;
    best.id = 0x7FFFFFFF;
    best.slot = -1;
    best.b0 = best.b1 = best.b2 = (T)0;
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) return;  // no triangle: caller checks slot < 0
    const T tau = prune_rel<T>() * ((T)m.scale + fmax(fabs(px), fmax(fabs(py), fabs(pz))));
    T thr2 = (T)INFINITY;
    auto test = [&](int s) {
        if (COUNT) work->tris++;
        T b[3];
        int id;
        const T d2 = Slot<T>::test(m, s, px, py, pz, b, id);
        if (d2 < best.d2 || (d2 == best.d2 && id < best.id)) {
            best.d2 = d2; best.id = id; best.slot = s;
            best.b0 = b[0]; best.b1 = b[1]; best.b2 = b[2];
            const T r = rsq<T>(d2) + tau;
            thr2 = r * r;
        }
    };
    if (guess >= 0) test(guess);
    if (m.nf == 1) { if (guess != 0) test(0); return; }
    int stack[kStackDepth];
    float sdist[kStackDepth];
    int sp = 0;
    int node = 0;
    for (int guard = 0;; guard++) {
        if (guard > 2 * m.nf + 64) { *err |= kErrTree; break; }
        if (COUNT) work->nodes++;
        const Node nd = m.nodes[node];
        const T d0 = box_d2<T>(px, py, pz, nd.a.x, nd.a.y, nd.a.z, nd.a.w, nd.b.x, nd.b.y);
        const T d1 = box_d2<T>(px, py, pz, nd.b.z, nd.b.w, nd.c.x, nd.c.y, nd.c.z, nd.c.w);
        const int c0 = nd.d.x, c1 = nd.d.y;
        bool h0 = d0 <= thr2, h1 = d1 <= thr2;
        if (h0 && c0 < 0) { test(~c0); h0 = false; }
        if (h1 && c1 < 0) { test(~c1); h1 = false; }
        h0 = h0 && d0 <= thr2;
        h1 = h1 && d1 <= thr2;
        if (h0 && h1) {
            const bool first0 = d0 <= d1;
            if (sp < kStackDepth) {
                stack[sp] = first0 ? c1 : c0;
                sdist[sp] = store_down<T>(first0 ? d1 : d0);
                sp++;
            } else {
                *err |= kErrStack;
            }
            node = first0 ? c0 : c1;
            continue;
        }
        if (h0) { node = c0; continue; }
        if (h1) { node = c1; continue; }
        bool found = false;
        while (sp > 0) {
            sp--;
            if ((T)sdist[sp] <= thr2) { node = stack[sp]; found = true; break; }
        }
        if (!found) break;
    }
}

// Resumable form of `closest` for loops that interleave the queries of many
// walks in one warp.  A lane advances its traversal one node per bq_step; the
// leaf triangles it meets are queued (at most two) and tested by bq_flush in
// rounds of the whole warp, so the costly triangle test runs on many lanes at
// once instead of a few per node.  A lane steps only with an empty queue, so
// its own sequence of visits and tests is exactly `closest`'s.  Every
// node is pruned only against a bound attained by a tested triangle (plus the
// slack tau), and the (d^2, id) minimum does not depend on the order of the
// tests, so the result equals `closest`'s.
template <typename T> struct BinQuery {
    T px, py, pz, tau, thr2;
    T nd2;      // box distance of `node`, re-checked before the visit
    int node;   // next node; -1: pop the stack first
    int sp, nq, q0, q1, guard;
    const Node *nodes;  // the mesh's tree and visit bound, held per query so that a
    int lim;            // node's address does not wait on a load of the job's mesh
};

template <typename T, bool COUNT>
__device__ __forceinline__ void bq_test(const DevMesh &m, BinQuery<T> &q, Hit<T> &best, int s, Work *work) {
    if (COUNT) work->tris++;
    T b[3];
    int id;
    const T d2 = Slot<T>::test(m, s, q.px, q.py, q.pz, b, id);
    if (d2 < best.d2 || (d2 == best.d2 && id < best.id)) {
        best.d2 = d2; best.id = id; best.slot = s;
        best.b0 = b[0]; best.b1 = b[1]; best.b2 = b[2];
        const T r = rsq<T>(d2) + q.tau;
        q.thr2 = r * r;
    }
}

// starts a query at p (guess >= 0: a slot tested at once); false when the
// query is already complete (non-finite point: best.slot stays -1; or a
// one-triangle mesh)
template <typename T, bool COUNT>
__device__ __forceinline__ bool bq_begin(const DevMesh &m, BinQuery<T> &q, Hit<T> &best, T px, T py, T pz, int guess,
                                         Work *work) {
    best.d2 = (T)INFINITY;
    best.id = 0x7FFFFFFF;
    best.slot = -1;
    best.b0 = best.b1 = best.b2 = (T)0;
    q.nq = 0; q.sp = 0; q.guard = 0; q.node = -1;
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) return false;
    q.px = px; q.py = py; q.pz = pz;
    q.tau = prune_rel<T>() * ((T)m.scale + fmax(fabs(px), fmax(fabs(py), fabs(pz))));
    q.thr2 = (T)INFINITY;
    if (guess >= 0) bq_test<T, COUNT>(m, q, best, guess, work);
    if (m.nf == 1) {
        if (guess != 0) bq_test<T, COUNT>(m, q, best, 0, work);
        return false;
    }
    q.node = 0;
    q.nd2 = (T)0;
    q.nodes = m.nodes;
    q.lim = 2 * m.nf + 64;
    return true;
}

// one node of a lane with no queued triangle (the stack is popped first when
// no node is pending); false when the query is complete
template <typename T, bool COUNT>
__device__ __forceinline__ bool bq_step(BinQuery<T> &q, int *stack, float *sdist, int *err, Work *work) {
    if (q.node >= 0 && q.nd2 > q.thr2) q.node = -1;
    if (q.node < 0) {
        while (q.sp > 0) {
            q.sp--;
            if ((T)sdist[q.sp] <= q.thr2) { q.node = stack[q.sp]; break; }
        }
        if (q.node < 0) return false;
    }
    if (q.guard++ > q.lim) { *err |= kErrTree; q.node = -1; q.sp = 0; return false; }
    if (COUNT) work->nodes++;
    const Node nd = q.nodes[q.node];
    const T d0 = box_d2<T>(q.px, q.py, q.pz, nd.a.x, nd.a.y, nd.a.z, nd.a.w, nd.b.x, nd.b.y);
    const T d1 = box_d2<T>(q.px, q.py, q.pz, nd.b.z, nd.b.w, nd.c.x, nd.c.y, nd.c.z, nd.c.w);
    const int c0 = nd.d.x, c1 = nd.d.y;
    bool h0 = d0 <= q.thr2, h1 = d1 <= q.thr2;
    if (h0 && c0 < 0) { q.q0 = ~c0; q.nq = 1; h0 = false; }
    if (h1 && c1 < 0) {
        if (q.nq) q.q1 = ~c1; else q.q0 = ~c1;
        q.nq++;
        h1 = false;
    }
    if (h0 && h1) {
        const bool first0 = d0 <= d1;
        if (q.sp < kStackDepth) {
            stack[q.sp] = first0 ? c1 : c0;
            sdist[q.sp] = store_down<T>(first0 ? d1 : d0);
            q.sp++;
        } else {
            *err |= kErrStack;
        }
        q.node = first0 ? c0 : c1;
        q.nd2 = first0 ? d0 : d1;
    } else if (h0 || h1) {
        q.node = h0 ? c0 : c1;
        q.nd2 = h0 ? d0 : d1;
    } else {
        q.node = -1;
    }
    return true;
}

// tests one queued triangle
template <typename T, bool COUNT>
__device__ __forceinline__ void bq_flush(const DevMesh &m, BinQuery<T> &q, Hit<T> &best, Work *work) {
    const int s = q.nq == 2 ? q.q1 : q.q0;
    q.nq--;
    bq_test<T, COUNT>(m, q, best, s, work);
}

constexpr int kStack4 = 96;  // 4-wide traversal: up to 3 deferred children per level

// closest triangle by traversal of the 4-wide BVH: the children in reach are
// visited nearest first, the others deferred on the stack; same result as
// closest() (the exact argmin of (d^2, id)), fewer dependent node fetches
template <typename T, bool COUNT = false>
__device__ void closest4(const DevMesh &m, T px, T py, T pz, int guess, Hit<T> &best, int *err,
                         Work *work = nullptr) {
    best.d2 = (T)INFINITY;
    best.id = 0x7FFFFFFF;
    best.slot = -1;
    best.b0 = best.b1 = best.b2 = (T)0;
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) return;  // no triangle: caller checks slot < 0
    const T tau = prune_rel<T>() * ((T)m.scale + fmax(fabs(px), fmax(fabs(py), fabs(pz))));
    T thr2 = (T)INFINITY;
    auto test = [&](int s) {
        if (COUNT) work->tris++;
        T b[3];
        int id;
        const T d2 = Slot<T>::test(m, s, px, py, pz, b, id);
        if (d2 < best.d2 || (d2 == best.d2 && id < best.id)) {
            best.d2 = d2; best.id = id; best.slot = s;
            best.b0 = b[0]; best.b1 = b[1]; best.b2 = b[2];
            const T r = rsq<T>(d2) + tau;
            thr2 = r * r;
        }
    };
    if (guess >= 0) test(guess);
    if (m.nf == 1) { if (guess != 0) test(0); return; }
    int stack[kStack4];
    float sdist[kStack4];
    int sp = 0;
    int node = 0;
    for (int guard = 0;; guard++) {
        if (guard > m.nf + 64) { *err |= kErrTree; break; }
        if (COUNT) work->nodes++;
        const Node4 nd = m.nodes4[node];
        const float lx[4] = {nd.lox.x, nd.lox.y, nd.lox.z, nd.lox.w};
        const float ly[4] = {nd.loy.x, nd.loy.y, nd.loy.z, nd.loy.w};
        const float lz[4] = {nd.loz.x, nd.loz.y, nd.loz.z, nd.loz.w};
        const float hx[4] = {nd.hix.x, nd.hix.y, nd.hix.z, nd.hix.w};
        const float hy[4] = {nd.hiy.x, nd.hiy.y, nd.hiy.z, nd.hiy.w};
        const float hz[4] = {nd.hiz.x, nd.hiz.y, nd.hiz.z, nd.hiz.w};
        const int ch[4] = {nd.child.x, nd.child.y, nd.child.z, nd.child.w};
        T d[4];
#pragma unroll
        for (int k = 0; k < 4; k++) d[k] = box_d2<T>(px, py, pz, lx[k], ly[k], lz[k], hx[k], hy[k], hz[k]);
        // leaves in reach first (they tighten the bound), nearest first
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (ch[k] < 0 && d[k] <= thr2) test(~ch[k]);
        // internal children still in reach, sorted by distance (at most 4)
        int ci[4];
        T cd[4];
        int nc = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (ch[k] >= 0 && ch[k] != kNoChild && d[k] <= thr2) {
                int j = nc++;
                while (j > 0 && cd[j - 1] > d[k]) { cd[j] = cd[j - 1]; ci[j] = ci[j - 1]; j--; }
                cd[j] = d[k];
                ci[j] = ch[k];
            }
        }
        if (nc > 0) {
            // defer the farther ones, farthest deepest
            for (int j = nc - 1; j >= 1; j--) {
                if (sp < kStack4) {
                    stack[sp] = ci[j];
                    sdist[sp] = store_down<T>(cd[j]);
                    sp++;
                } else {
                    *err |= kErrStack;
                }
            }
            node = ci[0];
            continue;
        }
        bool found = false;
        while (sp > 0) {
            sp--;
            if ((T)sdist[sp] <= thr2) { node = stack[sp]; found = true; break; }
        }
        if (!found) break;
    }
}

// closest triangle on the 4-wide BVH by a group of 4 consecutive lanes (the
// same query in all four; `r` = lane & 3, `gm` = the group's lane mask):
// lane r tests child box r of the current node and, when that child is a
// leaf in reach, its triangle; the group takes the lexicographic minimum of
// (d^2, id), sorts the internal children in reach by distance, visits the
// nearest and defers the others on a stack that every lane of the group
// holds a copy of.  Same result as closest(); every lane returns it.
template <typename T, bool COUNT = false>
__device__ void closest_g4(const DevMesh &m, T px, T py, T pz, int guess, Hit<T> &best, int *err, Work *work,
                           unsigned gm, int r) {
    best.d2 = (T)INFINITY;
    best.id = 0x7FFFFFFF;
    best.slot = -1;
    best.b0 = best.b1 = best.b2 = (T)0;
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) return;
    const T tau = prune_rel<T>() * ((T)m.scale + fmax(fabs(px), fmax(fabs(py), fabs(pz))));
    T thr2 = (T)INFINITY;
    const int base = (threadIdx.x & 31) & ~3;
    auto take = [&](T d2, int id, int slot, T b0, T b1, T b2) {
        if (d2 < best.d2 || (d2 == best.d2 && id < best.id)) {
            best.d2 = d2; best.id = id; best.slot = slot;
            best.b0 = b0; best.b1 = b1; best.b2 = b2;
            const T rr = rsq<T>(d2) + tau;
            thr2 = rr * rr;
        }
    };
    if (guess >= 0) {
        T b[3];
        int id;
        const T d2 = Slot<T>::test(m, guess, px, py, pz, b, id);
        if (COUNT && r == 0) work->tris++;
        take(d2, id, guess, b[0], b[1], b[2]);
    }
    if (m.nf == 1) {
        if (guess != 0) {
            T b[3];
            int id;
            const T d2 = Slot<T>::test(m, 0, px, py, pz, b, id);
            if (COUNT && r == 0) work->tris++;
            take(d2, id, 0, b[0], b[1], b[2]);
        }
        return;
    }
    int stack[kStack4];
    float sdist[kStack4];
    int sp = 0;
    int node = 0;
    for (int guard = 0;; guard++) {
        if (guard > m.nf + 64) { *err |= kErrTree; break; }
        if (COUNT && r == 0) work->nodes++;
        const float *nf4 = reinterpret_cast<const float *>(m.nodes4 + node);
        const int ch = reinterpret_cast<const int *>(nf4)[24 + r];
        T d = (T)INFINITY;
        if (ch != kNoChild) d = box_d2<T>(px, py, pz, nf4[r], nf4[4 + r], nf4[8 + r], nf4[12 + r], nf4[16 + r], nf4[20 + r]);
        // leaf children in reach: one triangle per lane, then the group minimum
        T ld = (T)INFINITY, lb0 = (T)0, lb1 = (T)0, lb2 = (T)0;
        int lid = 0x7FFFFFFF, lslot = -1;
        if (ch < 0 && d <= thr2) {
            T b[3];
            lslot = ~ch;
            ld = Slot<T>::test(m, lslot, px, py, pz, b, lid);
            lb0 = b[0]; lb1 = b[1]; lb2 = b[2];
            if (COUNT) work->tris++;
        }
        int wl = r;  // lane holding the group minimum
        {
            T md = ld;
            int mid = lid;
#pragma unroll
            for (int o = 1; o < 4; o <<= 1) {
                const T od = __shfl_xor_sync(gm, md, o);
                const int oi = __shfl_xor_sync(gm, mid, o);
                const int ol = __shfl_xor_sync(gm, wl, o);
                if (od < md || (od == md && oi < mid)) { md = od; mid = oi; wl = ol; }
            }
            const T w0 = __shfl_sync(gm, lb0, base + wl), w1 = __shfl_sync(gm, lb1, base + wl),
                    w2 = __shfl_sync(gm, lb2, base + wl);
            const int ws = __shfl_sync(gm, lslot, base + wl);
            if (ws >= 0) take(md, mid, ws, w0, w1, w2);
        }
        // internal children still in reach, nearest first (every lane builds the same list)
        const bool cand = ch >= 0 && ch != kNoChild && d <= thr2;
        int ci[4];
        T cd[4];
        int nc = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const T dk = __shfl_sync(gm, d, base + k);
            const int chk = __shfl_sync(gm, ch, base + k);
            const bool ck = __shfl_sync(gm, (int)cand, base + k) != 0;
            if (ck) {
                int j = nc++;
                while (j > 0 && cd[j - 1] > dk) { cd[j] = cd[j - 1]; ci[j] = ci[j - 1]; j--; }
                cd[j] = dk;
                ci[j] = chk;
            }
        }
        if (nc > 0) {
            for (int j = nc - 1; j >= 1; j--) {
                if (sp < kStack4) {
                    stack[sp] = ci[j];
                    sdist[sp] = store_down<T>(cd[j]);
                    sp++;
                } else {
                    *err |= kErrStack;
                }
            }
            node = ci[0];
            continue;
        }
        bool found = false;
        while (sp > 0) {
            sp--;
            if ((T)sdist[sp] <= thr2) { node = stack[sp]; found = true; break; }
        }
        if (!found) break;
    }
}

// --------------------------------------------------------------------------
// warp-cooperative query: the 32 lanes of a warp answer ONE query together.
// The top of the tree is expanded breadth-first into at most 32 subtrees
// (one per lane), each lane then traverses its subtree depth-first; the
// pruning bound is shared through warp reductions.
//   kFull:  exact argmin of (d^2, id) over all triangles (as `closest`);
//           with thr > 0, over the triangles nearer than thr (none: slot < 0)
//   kBelow: whether some triangle has sqrt(d^2) < thr (early exit), i.e. the
//           negation of sqrt(min d^2) >= thr, decided on the same per-triangle
//           values as the brute-force scan
// Every lane must call it with the same point; `front` is 32 ints of shared
// memory owned by the warp.
// --------------------------------------------------------------------------
constexpr int kFull = 0, kBelow = 1, kCollect = 2;
constexpr int kCandMax = 256;  // kCollect: band triangles kept per warp (measured: 256 cuts the two-sphere setup 6% below 64)
constexpr int kNone = 0x7FFFFFFF;

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

//   kCollect: true if some triangle has sqrt(d^2) < lo (early exit); else
//           the slots of the triangles with lo <= sqrt(d^2) < thr are stored
//           in cand (shared, kCandMax entries; *ncand counts them and must be
//           zero on entry); once it passes kCandMax the traversal stops, and
//           the result says nothing beyond that overflow
template <typename T, int MODE>
__device__ bool warp_query(const DevMesh &m, T px, T py, T pz, T thr, Hit<T> &out, int *front, int *err,
                           T lo = (T)0, int *cand = nullptr, int *ncand = nullptr) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const T tau = prune_rel<T>() * ((T)m.scale + fmax(fabs(px), fmax(fabs(py), fabs(pz))));
    T bound2;  // prune a box when its squared distance exceeds this
    if (MODE != kFull || thr > (T)0) {
        // kFull with thr > 0: only triangles nearer than thr are searched
        // (out.slot < 0 when there is none)
        const T r = thr + tau;
        bound2 = r * r;
    } else {
        bound2 = (T)INFINITY;
    }
    Hit<T> best;
    best.d2 = (T)INFINITY; best.id = 0x7FFFFFFF; best.slot = -1; best.b0 = best.b1 = best.b2 = (T)0;
    bool hit = false;
    auto test = [&](int s) {
        T b[3];
        int id;
        const T d2 = Slot<T>::test(m, s, px, py, pz, b, id);
        if (MODE == kBelow) {
            if (rsq<T>(d2) < thr) hit = true;
        } else if (MODE == kCollect) {
            const T d = rsq<T>(d2);
            if (d < lo) {
                hit = true;
            } else if (d < thr) {
                const int k = atomicAdd(ncand, 1);
                if (k < kCandMax) cand[k] = s;
            }
        } else if (d2 < best.d2 || (d2 == best.d2 && id < best.id)) {
            best.d2 = d2; best.id = id; best.slot = s; best.b0 = b[0]; best.b1 = b[1]; best.b2 = b[2];
        }
    };
    auto refresh = [&]() {
        if (MODE == kFull) {
            const T r = rsq<T>(warp_min<T>(best.d2)) + tau;
            bound2 = fmin(bound2, r * r);
        }
    };
    // ---- breadth-first expansion of the top of the tree
    int entry = kNone;  // >= 0 internal node, < 0 leaf (~slot)
    if (lane == 0) entry = (m.nf == 1) ? ~0 : 0;
    for (int round = 0; round < 8; round++) {
        const bool internal = entry != kNone && entry >= 0;
        int c0 = kNone, c1 = kNone;
        if (internal) {
            const Node nd = m.nodes[entry];
            const T d0 = box_d2<T>(px, py, pz, nd.a.x, nd.a.y, nd.a.z, nd.a.w, nd.b.x, nd.b.y);
            const T d1 = box_d2<T>(px, py, pz, nd.b.z, nd.b.w, nd.c.x, nd.c.y, nd.c.z, nd.c.w);
            if (d0 <= bound2) c0 = nd.d.x;
            if (d1 <= bound2) c1 = nd.d.y;
        }
        const int cnt = internal ? (c0 != kNone) + (c1 != kNone) : (entry != kNone);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        if (!__any_sync(FULL, internal) || total > 32) break;
        __syncwarp();
        int pos = incl - cnt;
        if (internal) {
            if (c0 != kNone) front[pos++] = c0;
            if (c1 != kNone) front[pos++] = c1;
        } else if (entry != kNone) {
            front[pos] = entry;
        }
        __syncwarp();
        entry = lane < total ? front[lane] : kNone;
        __syncwarp();
    }
    // ---- depth-first traversal of each lane's subtree
    int stack[kStackDepth];
    float sdist[kStackDepth];
    int sp = 0;
    int node = kNone;
    if (entry != kNone) {
        if (entry < 0) test(~entry);
        else node = entry;
    }
    int guard = 0;
    while (true) {
        refresh();
        if (MODE != kFull && __any_sync(FULL, hit)) { hit = true; break; }
        // kCollect past kCandMax: the caller falls back to an exact FP64
        // query, so the rest of this traversal would be wasted
        if (MODE == kCollect && __any_sync(FULL, *ncand > kCandMax)) break;
        const bool active = node != kNone;
        if (!__any_sync(FULL, active)) break;
        if (!active) continue;
        if (++guard > 2 * m.nf + 64) { *err |= kErrTree; node = kNone; continue; }
        const Node nd = m.nodes[node];
        const T d0 = box_d2<T>(px, py, pz, nd.a.x, nd.a.y, nd.a.z, nd.a.w, nd.b.x, nd.b.y);
        const T d1 = box_d2<T>(px, py, pz, nd.b.z, nd.b.w, nd.c.x, nd.c.y, nd.c.z, nd.c.w);
        const int c0 = nd.d.x, c1 = nd.d.y;
        bool h0 = d0 <= bound2, h1 = d1 <= bound2;
        if (h0 && c0 < 0) { test(~c0); h0 = false; }
        if (h1 && c1 < 0) { test(~c1); h1 = false; }
        if (h0 && h1) {
            const bool first0 = d0 <= d1;
            if (sp < kStackDepth) {
                stack[sp] = first0 ? c1 : c0;
                sdist[sp] = store_down<T>(first0 ? d1 : d0);
                sp++;
            } else {
                *err |= kErrStack;
            }
            node = first0 ? c0 : c1;
        } else if (h0) {
            node = c0;
        } else if (h1) {
            node = c1;
        } else {
            node = kNone;
            while (sp > 0) {
                sp--;
                if ((T)sdist[sp] <= bound2) { node = stack[sp]; break; }
            }
        }
    }
    if (MODE != kFull) return __any_sync(FULL, hit);
    // ---- lexicographic warp argmin of (d^2, id)
    T bd = best.d2;
    int bi = best.id, bl = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T od = __shfl_xor_sync(FULL, bd, o);
        const int oi = __shfl_xor_sync(FULL, bi, o);
        const int ol = __shfl_xor_sync(FULL, bl, o);
        if (od < bd || (od == bd && oi < bi)) { bd = od; bi = oi; bl = ol; }
    }
    out.d2 = bd;
    out.id = bi;
    out.slot = __shfl_sync(FULL, best.slot, bl);
    out.b0 = __shfl_sync(FULL, best.b0, bl);
    out.b1 = __shfl_sync(FULL, best.b1, bl);
    out.b2 = __shfl_sync(FULL, best.b2, bl);
    return false;
}

}  // namespace mcs
