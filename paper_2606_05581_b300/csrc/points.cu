// points.cu -- the point-based Galerkin basis (Sec. 4.4 "Point-based Galerkin
// basis"; appendix "Point-based k-NN Interpolator").
//
// The function space lives on a point set P sampled on the surface (the
// farthest-point sample rows serve as the blue-noise points).  Three pieces:
//   * a k-nearest-point query over P: a uniform grid built on the device
//     (bounding box, cell keys, one radix sort, cell ranges), searched in
//     growing shells of cells until the k-th best squared distance is below
//     the distance to every unvisited cell.  Squared distances are FP64,
//     ((dx dx + dy dy) + dz dz) with d = q - p, ties by the smaller point
//     index, so the neighbour lists are exact and reproducible;
//   * the bilateral interpolator: w_i proportional to
//     exp(-|q - x_i|^2 / (2 sigma^2)) exp(-(1 - <n_q, n_i>) / tau_n) over the
//     k nearest points, normalised (evaluated as exp(-(a_i - min a)) with a
//     the summed exponents: the same ratios, and never all zero);
//   * the point-cloud Laplacian: each point's k nearest other points are
//     projected onto its tangent plane and its Voronoi cell among them is cut
//     out of a box by the bisector half-planes; the weight of neighbour j is
//     |cell edge on the (i, j) bisector| / |u_j| (the cotangent weight of the
//     local Delaunay triangulation), and the dense symmetric Laplacian takes
//     L_ij = -(w_ij + w_ji) / 2, L_ii = -sum_j L_ij.
// The Galerkin matrix over P accumulates, per walk, w (b_s - b_t)(b_s - b_t)^T
// with b_s the interpolator at the row point p_r (normal n_r), b_t the
// interpolator at the exit point (normal of the exit face) and
// w = omega_r / (2 W) (times |t - o| for exterior walks), FP64 atomics.
// Everything here is FP64 and bounded: no kernel waits on another.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>

#include "mcs_internal.h"

namespace mcs {
namespace points {

constexpr int kMaxK = 32;       // neighbours per query (interpolator and Laplacian)
constexpr int kMaxPoly = 4 + kMaxK;

struct Grid {
    double lo[3];
    double h, inv_h;
    int g[3];
    int n;
};

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
static size_t max_cells(int n) { return 2 * (size_t)n + 64; }

struct Layout {
    size_t hdr, keys, keys_s, ids, Ps, begin, end, sidx, sw, sort, total;
    size_t sort_bytes;
};

static Layout layout(int n) {
    Layout l;
    size_t o = 0;
    l.hdr = o; o += 256;
    l.keys = o; o += a256((size_t)n * 8);
    l.keys_s = o; o += a256((size_t)n * 8);
    l.ids = o; o += a256((size_t)n * 4);
    l.Ps = o; o += a256((size_t)n * 24);
    l.begin = o; o += a256(max_cells(n) * 4);
    l.end = o; o += a256(max_cells(n) * 4);
    l.sidx = o; o += a256((size_t)n * kMaxK * 4);
    l.sw = o; o += a256((size_t)n * kMaxK * 8);
    l.sort_bytes = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, l.sort_bytes, (unsigned long long *)nullptr,
                                   (unsigned long long *)nullptr, n, 0, 64);
    l.sort = o; o += a256(l.sort_bytes);
    l.total = o;
    return l;
}

// bounding box (one block) and the grid: the finest h (in steps of 0.9 from
// the largest extent) whose cell count stays within max_cells
__global__ void k_grid(const double *P, int n, long long cap, Grid *G) {
    __shared__ double mn[3][256], mx[3][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int a = 0; a < 3; a++) {
            lo[a] = fmin(lo[a], P[3 * i + a]);
            hi[a] = fmax(hi[a], P[3 * i + a]);
        }
    for (int a = 0; a < 3; a++) { mn[a][threadIdx.x] = lo[a]; mx[a][threadIdx.x] = hi[a]; }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int a = 0; a < 3; a++) {
                mn[a][threadIdx.x] = fmin(mn[a][threadIdx.x], mn[a][threadIdx.x + s]);
                mx[a][threadIdx.x] = fmax(mx[a][threadIdx.x], mx[a][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x) return;
    double ext[3], big = 0.0;
    for (int a = 0; a < 3; a++) {
        ext[a] = mx[a][0] - mn[a][0];
        big = fmax(big, ext[a]);
        G->lo[a] = mn[a][0];
    }
    double h = big > 0.0 ? big : 1.0;
    for (int it = 0; it < 400; it++) {
        const double hn = 0.9 * h;
        double cells = 1.0;
        for (int a = 0; a < 3; a++) cells *= floor(ext[a] / hn) + 1.0;
        if (cells > (double)cap) break;
        h = hn;
    }
    G->h = h;
    G->inv_h = 1.0 / h;
    for (int a = 0; a < 3; a++) G->g[a] = (int)(floor(ext[a] / h) + 1.0);
    G->n = n;
}

__device__ __forceinline__ int cell_coord(double x, double lo, double inv_h, int g) {
    const double f = floor((x - lo) * inv_h);
    return f < 0.0 ? 0 : (f > (double)(g - 1) ? g - 1 : (int)f);
}

__global__ void k_keys(const double *P, int n, const Grid *G, unsigned long long *keys) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Grid g = *G;
    const int cx = cell_coord(P[3 * i], g.lo[0], g.inv_h, g.g[0]);
    const int cy = cell_coord(P[3 * i + 1], g.lo[1], g.inv_h, g.g[1]);
    const int cz = cell_coord(P[3 * i + 2], g.lo[2], g.inv_h, g.g[2]);
    const unsigned long long c = ((unsigned long long)cz * g.g[1] + cy) * g.g[0] + cx;
    keys[i] = (c << 32) | (unsigned)i;
}

__global__ void k_cells(const unsigned long long *ks, const double *P, int n, int *ids, double *Ps, int *begin,
                        int *end) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long c = ks[i] >> 32;
    const int id = (int)(ks[i] & 0xffffffffull);
    ids[i] = id;
    Ps[3 * i] = P[3 * id];
    Ps[3 * i + 1] = P[3 * id + 1];
    Ps[3 * i + 2] = P[3 * id + 2];
    if (i == 0 || (ks[i - 1] >> 32) != c) begin[c] = i;
    if (i == n - 1 || (ks[i + 1] >> 32) != c) end[c] = i + 1;
}

struct GridView {
    Grid g;
    const int *begin, *end, *ids;
    const double *Ps;
};

// (d2, index) order; squared distances are never negative, so their bit
// patterns order like the values and the comparison stays off the FP64 pipe
__device__ __forceinline__ bool before(double a, int ia, double b, int ib) {
    const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
    return x < y || (x == y && ia < ib);
}

// the k nearest points of q (skipping point `skip`), ascending (d2, index);
// returns how many were found (k unless the set is smaller)
__device__ int knn_query(const GridView &V, double qx, double qy, double qz, int k, int skip, double *bd, int *bi) {
    const Grid &g = V.g;
    const int c[3] = {cell_coord(qx, g.lo[0], g.inv_h, g.g[0]), cell_coord(qy, g.lo[1], g.inv_h, g.g[1]),
                      cell_coord(qz, g.lo[2], g.inv_h, g.g[2])};
    const double q[3] = {qx, qy, qz};
    int cnt = 0;
    const int smax = max(g.g[0], max(g.g[1], g.g[2]));
    for (int s = 0; s <= smax; s++) {
        const int z0 = max(c[2] - s, 0), z1 = min(c[2] + s, g.g[2] - 1);
        const int y0 = max(c[1] - s, 0), y1 = min(c[1] + s, g.g[1] - 1);
        for (int z = z0; z <= z1; z++)
            for (int y = y0; y <= y1; y++) {
                const bool face = abs(z - c[2]) == s || abs(y - c[1]) == s;
                const int step = (face || s == 0) ? 1 : 2 * s;
                const int xa = face ? max(c[0] - s, 0) : c[0] - s;
                const int xb = face ? min(c[0] + s, g.g[0] - 1) : c[0] + s;
                for (int x = xa; x <= xb; x += step) {
                    if (x < 0 || x >= g.g[0]) continue;
                    const size_t cell = ((size_t)z * g.g[1] + y) * g.g[0] + x;
                    for (int j = V.begin[cell]; j < V.end[cell]; j++) {
                        const int pid = V.ids[j];
                        if (pid == skip) continue;
                        const double dx = qx - V.Ps[3 * j], dy = qy - V.Ps[3 * j + 1], dz = qz - V.Ps[3 * j + 2];
                        const double d2 = dx * dx + dy * dy + dz * dz;
                        if (cnt < k || before(d2, pid, bd[k - 1], bi[k - 1])) {
                            int p = cnt < k ? cnt++ : k - 1;
                            while (p > 0 && before(d2, pid, bd[p - 1], bi[p - 1])) {
                                bd[p] = bd[p - 1];
                                bi[p] = bi[p - 1];
                                p--;
                            }
                            bd[p] = d2;
                            bi[p] = pid;
                        }
                    }
                }
            }
        // distance from q to the cells not yet visited (infinite where the
        // visited block already reaches the grid's edge)
        double b = INFINITY;
        for (int a = 0; a < 3; a++) {
            if (c[a] - s > 0) b = fmin(b, q[a] - (g.lo[a] + (c[a] - s) * g.h));
            if (c[a] + s + 1 < g.g[a]) b = fmin(b, g.lo[a] + (c[a] + s + 1) * g.h - q[a]);
        }
        if (b == INFINITY) break;
        const double bs = b - 1e-7 * g.h;  // margin for the rounding of the cell assignment
        if (cnt >= k && bs > 0.0 && bd[k - 1] < bs * bs) break;
    }
    return cnt;
}

// bilateral weights of the k neighbours (normalised; see the file comment)
__device__ void bilateral(const double *NP, double nx, double ny, double nz, int k, double sigma, double tau,
                          const double *bd, const int *bi, double *w) {
    double amin = INFINITY;
    const double is = 1.0 / (2.0 * sigma * sigma), it = 1.0 / tau;  // reciprocals: FP64 divisions are costly here
    for (int i = 0; i < k; i++) {
        const double *m = NP + 3 * bi[i];
        const double dot = nx * m[0] + ny * m[1] + nz * m[2];
        w[i] = bd[i] * is + (1.0 - dot) * it;
        amin = fmin(amin, w[i]);
    }
    double sum = 0.0;
    for (int i = 0; i < k; i++) {
        w[i] = exp(-(w[i] - amin));
        sum += w[i];
    }
    const double inv = 1.0 / sum;
    for (int i = 0; i < k; i++) w[i] *= inv;
}

__global__ void k_knn(GridView V, const double *NP, const double *Q, const double *NQ, int nq, int k, double sigma,
                      double tau, int exclude_self, int32_t *idx, double *w, double *d2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double bd[kMaxK];
    int bi[kMaxK];
    knn_query(V, Q[3 * q], Q[3 * q + 1], Q[3 * q + 2], k, exclude_self ? q : -1, bd, bi);
    for (int i = 0; i < k; i++) {
        if (idx) idx[(size_t)q * k + i] = bi[i];
        if (d2) d2[(size_t)q * k + i] = bd[i];
    }
    if (w) {
        double ww[kMaxK];
        bilateral(NP, NQ[3 * q], NQ[3 * q + 1], NQ[3 * q + 2], k, sigma, tau, bd, bi, ww);
        for (int i = 0; i < k; i++) w[(size_t)q * k + i] = ww[i];
    }
}

// one point per thread: tangent frame, projected neighbours, Voronoi cell of
// the origin by successive half-plane cuts of a box (vertex + tag of the edge
// leaving it; tag -1 = box), then the per-neighbour dual/primal weights
__global__ void k_local_cells(GridView V, const double *P, const double *NP, int n, int k, int32_t *nbr,
                              double *nbr_w, double *area) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double bd[kMaxK];
    int bi[kMaxK];
    knn_query(V, P[3 * i], P[3 * i + 1], P[3 * i + 2], k, i, bd, bi);
    const double nn[3] = {NP[3 * i], NP[3 * i + 1], NP[3 * i + 2]};
    const double an[3] = {fabs(nn[0]), fabs(nn[1]), fabs(nn[2])};
    const int ax = (an[0] <= an[1] && an[0] <= an[2]) ? 0 : (an[1] <= an[2] ? 1 : 2);
    const double av[3] = {ax == 0 ? 1.0 : 0.0, ax == 1 ? 1.0 : 0.0, ax == 2 ? 1.0 : 0.0};
    double e1[3] = {nn[1] * av[2] - nn[2] * av[1], nn[2] * av[0] - nn[0] * av[2], nn[0] * av[1] - nn[1] * av[0]};
    const double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int a = 0; a < 3; a++) e1[a] /= l1;
    const double e2[3] = {nn[1] * e1[2] - nn[2] * e1[1], nn[2] * e1[0] - nn[0] * e1[2],
                          nn[0] * e1[1] - nn[1] * e1[0]};
    double ux[kMaxK], uy[kMaxK];
    double R = 0.0;
    for (int j = 0; j < k; j++) {
        const double d0 = P[3 * bi[j]] - P[3 * i], d1 = P[3 * bi[j] + 1] - P[3 * i + 1],
                     d2 = P[3 * bi[j] + 2] - P[3 * i + 2];
        ux[j] = d0 * e1[0] + d1 * e1[1] + d2 * e1[2];
        uy[j] = d0 * e2[0] + d1 * e2[1] + d2 * e2[2];
        R = fmax(R, sqrt(ux[j] * ux[j] + uy[j] * uy[j]));
    }
    R *= 2.0;
    double px[kMaxPoly], py[kMaxPoly], ox[kMaxPoly], oy[kMaxPoly];
    int pt[kMaxPoly], ot[kMaxPoly];
    int m = 4;
    px[0] = -R; py[0] = -R; px[1] = R; py[1] = -R; px[2] = R; py[2] = R; px[3] = -R; py[3] = R;
    pt[0] = pt[1] = pt[2] = pt[3] = -1;
    for (int j = 0; j < k && m > 0; j++) {
        const double a = ux[j], b = uy[j];
        const double c = 0.5 * (a * a + b * b);
        if (c == 0.0) continue;
        int mo = 0;
        for (int v = 0; v < m; v++) {
            const int w = v + 1 == m ? 0 : v + 1;
            const double fp = px[v] * a + py[v] * b - c;
            const double fq = px[w] * a + py[w] * b - c;
            if (fp <= 0.0) {
                if (mo < kMaxPoly) { ox[mo] = px[v]; oy[mo] = py[v]; ot[mo] = pt[v]; mo++; }
                if (fq > 0.0) {
                    const double s = fp / (fp - fq);
                    if (mo < kMaxPoly) { ox[mo] = px[v] + s * (px[w] - px[v]); oy[mo] = py[v] + s * (py[w] - py[v]); ot[mo] = j; mo++; }
                }
            } else if (fq <= 0.0) {
                const double s = fp / (fp - fq);
                if (mo < kMaxPoly) { ox[mo] = px[v] + s * (px[w] - px[v]); oy[mo] = py[v] + s * (py[w] - py[v]); ot[mo] = pt[v]; mo++; }
            }
        }
        m = mo;
        for (int v = 0; v < m; v++) { px[v] = ox[v]; py[v] = oy[v]; pt[v] = ot[v]; }
    }
    double lens[kMaxK];
    for (int j = 0; j < k; j++) lens[j] = 0.0;
    double A = 0.0;
    for (int v = 0; v < m; v++) {
        const int w = v + 1 == m ? 0 : v + 1;
        A += px[v] * py[w] - px[w] * py[v];
        if (pt[v] >= 0) lens[pt[v]] += hypot(px[w] - px[v], py[w] - py[v]);
    }
    if (area) area[i] = 0.5 * A;
    for (int j = 0; j < k; j++) {
        const double r = sqrt(ux[j] * ux[j] + uy[j] * uy[j]);
        nbr[(size_t)i * k + j] = bi[j];
        nbr_w[(size_t)i * k + j] = r > 0.0 ? lens[j] / r : 0.0;
    }
}

__global__ void k_laplacian_offdiag(const int32_t *nbr, const double *nbr_w, int n, int k, double *L) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * k) return;
    const int i = (int)(e / k), j = nbr[e];
    const double x = 0.5 * nbr_w[e];
    if (x == 0.0) return;
    atomicAdd(&L[(size_t)i * n + j], -x);
    atomicAdd(&L[(size_t)j * n + i], -x);
}

// L_ii = -sum_{j != i} L_ij: one warp per row
__global__ void k_laplacian_diag(int n, double *L) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= n) return;
    const double *r = L + (size_t)row * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32)
        if (j != row) s += r[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) L[(size_t)row * n + row] = -s;
}

// per walk: exit point and face normal, its k neighbours and weights, and
// w (b_s - b_t)(b_s - b_t)^T into the dense point-set matrix
__global__ void k_point_assemble(GridView V, const double *Vm, const int32_t *F, const double *NP, int n, int W,
                                 const double *omega, const int32_t *exit_tri, const double *exit_bary, int exterior,
                                 double o0, double o1, double o2, int k, double sigma, double tau,
                                 const int32_t *sidx, const double *sw, double *L) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * W) return;
    const int r = (int)(e / W);
    const int t = exit_tri[e];
    if (t < 0) return;
    double w = 0.5 * omega[r] / (double)W;
    if (!(w != 0.0)) return;
    const double *bt = exit_bary + 3 * e;
    const int tv[3] = {F[3 * t], F[3 * t + 1], F[3 * t + 2]};
    double p[3];
    for (int a = 0; a < 3; a++)
        p[a] = bt[0] * Vm[3 * tv[0] + a] + bt[1] * Vm[3 * tv[1] + a] + bt[2] * Vm[3 * tv[2] + a];
    if (exterior) {
        const double d0 = p[0] - o0, d1 = p[1] - o1, d2 = p[2] - o2;
        w *= sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    const double u0 = Vm[3 * tv[1]] - Vm[3 * tv[0]], u1 = Vm[3 * tv[1] + 1] - Vm[3 * tv[0] + 1],
                 u2 = Vm[3 * tv[1] + 2] - Vm[3 * tv[0] + 2];
    const double v0 = Vm[3 * tv[2]] - Vm[3 * tv[0]], v1 = Vm[3 * tv[2] + 1] - Vm[3 * tv[0] + 1],
                 v2 = Vm[3 * tv[2] + 2] - Vm[3 * tv[0] + 2];
    double fn[3] = {u1 * v2 - u2 * v1, u2 * v0 - u0 * v2, u0 * v1 - u1 * v0};
    const double fl = sqrt(fn[0] * fn[0] + fn[1] * fn[1] + fn[2] * fn[2]);
    const double ifl = fl > 0.0 ? 1.0 / fl : 0.0;
    for (int a = 0; a < 3; a++) fn[a] *= ifl;
    double bd[kMaxK], tw[kMaxK];
    int bi[kMaxK];
    knn_query(V, p[0], p[1], p[2], k, -1, bd, bi);
    bilateral(NP, fn[0], fn[1], fn[2], k, sigma, tau, bd, bi, tw);
    const int32_t *si = sidx + (size_t)r * k;
    const double *sv = sw + (size_t)r * k;
    // the upper triangle only (k_mirror copies it down): pair (a, b), a < b,
    // adds w d_a d_b at (min, max) of its two points, twice on the diagonal
    // when both entries name the same point
    for (int a = 0; a < 2 * k; a++) {
        const int ia = a < k ? si[a] : bi[a - k];
        const double wa = w * (a < k ? sv[a] : -tw[a - k]);
        atomicAdd(&L[(size_t)ia * n + ia], wa * (a < k ? sv[a] : -tw[a - k]));
        for (int b = a + 1; b < 2 * k; b++) {
            const int ib = b < k ? si[b] : bi[b - k];
            const double x = wa * (b < k ? sv[b] : -tw[b - k]);
            if (ia == ib) atomicAdd(&L[(size_t)ia * n + ia], 2.0 * x);
            else atomicAdd(&L[(size_t)min(ia, ib) * n + max(ia, ib)], x);
        }
    }
}

// lower triangle = upper triangle (32 x 32 tiles through shared memory)
__global__ void k_mirror(int n, double *L) {
    __shared__ double t[32][33];
    const int bx = blockIdx.x, by = blockIdx.y;
    if (bx < by) return;  // tile (by, bx) in the upper part feeds tile (bx, by)
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int i = by * 32 + r, j = bx * 32 + tx;
        t[r][tx] = (i < n && j < n) ? L[(size_t)i * n + j] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = bx * 32 + r, j = by * 32 + tx;  // lower element (i, j) = upper (j, i)
        if (i < n && j < n && i > j) L[(size_t)i * n + j] = t[tx][r];
    }
}

// killing walks (exterior): 4 pi |p_r - o| H0_r / N0 b_s b_s^T at their bin row
__global__ void k_point_killing(const double *P, int n, const int32_t *H0, double n_kill, double o0, double o1,
                                double o2, int k, const int32_t *sidx, const double *sw, double *L) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n || H0[r] == 0) return;
    const double d0 = P[3 * r] - o0, d1 = P[3 * r + 1] - o1, d2 = P[3 * r + 2] - o2;
    const double x = 12.566370614359172 * sqrt(d0 * d0 + d1 * d1 + d2 * d2) * H0[r] / n_kill;
    const int32_t *si = sidx + (size_t)r * k;
    const double *sv = sw + (size_t)r * k;
    for (int a = 0; a < k; a++) {
        atomicAdd(&L[(size_t)si[a] * n + si[a]], x * sv[a] * sv[a]);
        for (int b = a + 1; b < k; b++)  // distinct points: one neighbour list
            atomicAdd(&L[(size_t)min(si[a], si[b]) * n + max(si[a], si[b])], x * sv[a] * sv[b]);
    }
}

// build the grid of P in the workspace; returns the view the queries use
static mcs_status build_grid(const double *P, int n, char *w, const Layout &l, cudaStream_t st, GridView *view) {
    Grid *G = (Grid *)(w + l.hdr);
    unsigned long long *keys = (unsigned long long *)(w + l.keys), *keys_s = (unsigned long long *)(w + l.keys_s);
    int *ids = (int *)(w + l.ids), *begin = (int *)(w + l.begin), *end = (int *)(w + l.end);
    double *Ps = (double *)(w + l.Ps);
    note_launch();
    k_grid<<<1, 256, 0, st>>>(P, n, (long long)max_cells(n), G);
    note_launch();
    k_keys<<<(n + 255) / 256, 256, 0, st>>>(P, n, G, keys);
    size_t sb = l.sort_bytes;
    MCS_CUDA(cub::DeviceRadixSort::SortKeys(w + l.sort, sb, keys, keys_s, n, 0, 64, st));
    MCS_CUDA(cudaMemsetAsync(begin, 0, max_cells(n) * 4, st));
    MCS_CUDA(cudaMemsetAsync(end, 0, max_cells(n) * 4, st));
    note_launch();
    k_cells<<<(n + 255) / 256, 256, 0, st>>>(keys_s, P, n, ids, Ps, begin, end);
    Grid h;
    MCS_CUDA(cudaMemcpyAsync(&h, G, sizeof(Grid), cudaMemcpyDeviceToHost, st));
    MCS_CUDA(cudaStreamSynchronize(st));
    view->g = h;
    view->begin = begin;
    view->end = end;
    view->ids = ids;
    view->Ps = Ps;
    return MCS_OK;
}

}  // namespace points
}  // namespace mcs

using namespace mcs;
using namespace mcs::points;

extern "C" {

size_t mcs_points_workspace_size(int n_points) {
    if (n_points < 1) return 0;
    return layout(n_points).total;
}

#define PT_WS(fn)                                                                                   \
    const Layout l = layout(n_points);                                                              \
    MCS_ARG(workspace && workspace_bytes >= l.total, fn ": workspace too small");                   \
    MCS_ARG(((uintptr_t)workspace & 255) == 0, fn ": workspace must be 256-byte aligned");          \
    char *wsb = (char *)workspace;                                                                  \
    cudaStream_t st = as_stream(stream);                                                            \
    GridView view;                                                                                  \
    {                                                                                               \
        const mcs_status gs = build_grid(P, n_points, wsb, l, st, &view);                             \
        if (gs != MCS_OK) return gs;                                                                \
    }

mcs_status mcs_point_knn(const double *P, const double *NP, int n_points, const double *Q, const double *NQ,
                         int n_queries, int k, double sigma, double tau_n, int exclude_self, int32_t *idx, double *w,
                         double *d2, void *workspace, size_t workspace_bytes, void *stream) {
    MCS_ARG(n_points >= 1 && n_queries >= 0, "mcs_point_knn: need n_points >= 1");
    MCS_ARG(P && (n_queries == 0 || (Q && (idx || w || d2))), "mcs_point_knn: NULL argument");
    MCS_ARG(k >= 1 && k <= kMaxK && k <= n_points - (exclude_self ? 1 : 0), "mcs_point_knn: need 1 <= k <= 32 and k <= the candidates");
    MCS_ARG(!exclude_self || n_queries == n_points, "mcs_point_knn: exclude_self needs the points as the queries");
    MCS_ARG(!w || (NP && NQ && sigma > 0.0 && tau_n > 0.0), "mcs_point_knn: weights need both normals and sigma, tau_n > 0");
    if (n_queries == 0) return MCS_OK;
    PT_WS("mcs_point_knn")
    note_launch();
    k_knn<<<(n_queries + 127) / 128, 128, 0, st>>>(view, NP, Q, NQ, n_queries, k, sigma, tau_n, exclude_self, idx, w,
                                                   d2);
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

mcs_status mcs_point_laplacian(const double *P, const double *NP, int n_points, int k_nbr, double *L,
                               double *cell_area, int32_t *nbr, double *nbr_w, void *workspace,
                               size_t workspace_bytes, void *stream) {
    MCS_ARG(P && NP && L && nbr && nbr_w, "mcs_point_laplacian: NULL argument");
    MCS_ARG(k_nbr >= 3 && k_nbr <= kMaxK && k_nbr <= n_points - 1, "mcs_point_laplacian: need 3 <= k_nbr <= 32, k_nbr < n_points");
    PT_WS("mcs_point_laplacian")
    note_launch();
    k_local_cells<<<(n_points + 127) / 128, 128, 0, st>>>(view, P, NP, n_points, k_nbr, nbr, nbr_w, cell_area);
    MCS_CUDA(cudaMemsetAsync(L, 0, sizeof(double) * (size_t)n_points * n_points, st));
    note_launch();
    k_laplacian_offdiag<<<(unsigned)(((size_t)n_points * k_nbr + 255) / 256), 256, 0, st>>>(nbr, nbr_w, n_points,
                                                                                            k_nbr, L);
    note_launch();
    k_laplacian_diag<<<(n_points + 7) / 8, 256, 0, st>>>(n_points, L);
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

mcs_status mcs_point_galerkin_lambda(mcs_mesh m, const double *P, const double *NP, int n_points,
                                     const double *omega, const int32_t *exit_tri, const double *exit_bary,
                                     int walks_per_row, int exterior, const double *origin, const int32_t *H0,
                                     long long killing_walks, int k, double sigma, double tau_n, double *Lambda_P,
                                     void *workspace, size_t workspace_bytes, void *stream) {
    MCS_ARG(m && P && NP && omega && exit_tri && exit_bary && Lambda_P, "mcs_point_galerkin_lambda: NULL argument");
    MCS_ARG(n_points >= 1 && walks_per_row >= 1, "mcs_point_galerkin_lambda: need n_points, walks_per_row >= 1");
    MCS_ARG(k >= 1 && k <= kMaxK && k <= n_points, "mcs_point_galerkin_lambda: need 1 <= k <= min(32, n_points)");
    MCS_ARG(sigma > 0.0 && tau_n > 0.0, "mcs_point_galerkin_lambda: need sigma, tau_n > 0");
    MCS_ARG(!exterior || origin, "mcs_point_galerkin_lambda: exterior needs the inversion centre");
    PT_WS("mcs_point_galerkin_lambda")
    int32_t *sidx = (int32_t *)(wsb + l.sidx);
    double *sw = (double *)(wsb + l.sw);
    note_launch();
    k_knn<<<(n_points + 127) / 128, 128, 0, st>>>(view, NP, P, NP, n_points, k, sigma, tau_n, 0, sidx, sw, nullptr);
    const double o0 = exterior ? origin[0] : 0.0, o1 = exterior ? origin[1] : 0.0, o2 = exterior ? origin[2] : 0.0;
    MCS_CUDA(cudaMemsetAsync(Lambda_P, 0, sizeof(double) * (size_t)n_points * n_points, st));
    const size_t nw = (size_t)n_points * walks_per_row;
    note_launch();
    k_point_assemble<<<(unsigned)((nw + 127) / 128), 128, 0, st>>>(view, m->V, m->F, NP, n_points, walks_per_row,
                                                                    omega, exit_tri, exit_bary, exterior, o0, o1, o2,
                                                                    k, sigma, tau_n, sidx, sw, Lambda_P);
    if (exterior && H0 && killing_walks > 0) {
        note_launch();
        k_point_killing<<<(n_points + 127) / 128, 128, 0, st>>>(P, n_points, H0, (double)killing_walks, o0, o1, o2,
                                                                k, sidx, sw, Lambda_P);
    }
    note_launch();
    const unsigned nt = (unsigned)((n_points + 31) / 32);
    k_mirror<<<dim3(nt, nt), 256, 0, st>>>(n_points, Lambda_P);
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

}  // extern "C"
