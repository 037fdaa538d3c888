// galerkin.cu -- the Galerkin (K x K) DtN estimator with barycentric basis
// evaluation, and the cotangent Laplacian whose low modes are its default
// basis (Sec. 4.4 "Mesh-based Galerkin basis"; boxed estimators Eq.
// main-estimator and Eq. main-exterior-estimator).
//
// The boxed estimators accumulate  w d(s,t) d(s,t)^T  with d(s,t) = b(s) - b(t),
// b the K basis functions evaluated by barycentric interpolation, and w the
// walk's weight: omega_v / (2 W) (omega_v = A_v M_v, times |s~|^3 for
// exterior rows; the 1/2 is the boxed estimators' own) and, for exterior
// walks, the factor 1/|t~| = |t - o| at the hit point t itself.  With Phi the n x K nodal values of the basis and e_s, beta_t
// the nodal (hat-function) coefficients of the row point and of the exit
// point, d = Phi^T (e_s - beta_t), so the estimate is
//   S = Phi^T Lambda_bary Phi,   Lambda_bary = sum_walks w (e_s - beta_t)(e_s - beta_t)^T,
// an n x n matrix on the mesh's vertices: the full P1 (hat-basis) Galerkin
// stiffness.  The nodal Lambda of the histogram path is exactly the special
// case of one-hot beta at the largest barycentric.  Killing walks (exterior) enter
// lumped at their bin vertex: 4 pi |t - o| / N0 on the diagonal (their exit
// barycentrics are not recorded).
//
// Lambda_bary is assembled with FP64 atomics (summation order varies with
// scheduling: the result is reproducible to rounding, not bitwise);
// Lambda_bary Phi runs on the tensor cores (the split tf32 product of
// eig.cu, FP32-level accuracy); the rest is FP64.  The K x K eigenproblem
// (Phi M-orthonormal, so S c = lambda c) is a cyclic Jacobi in FP64 on one SM.
#include <algorithm>
#include <cmath>
#include <string>

#include "mcs_internal.h"

namespace mcs {
namespace galerkin {

// dense cotangent Laplacian (FP64): row a gathers, over its incident faces
// in ascending order, (cot gamma)/2 for each edge (a, b) of the face (gamma
// the angle opposite the edge); L[a][b] = -sum, L[a][a] = +sum.  Rows are
// written by one thread each (deterministic; symmetric because both ends of an
// edge see the same faces in the same order).
__global__ void k_cotan(const double *V, const int32_t *F, const int32_t *inc_f, const int32_t *vstart, int nv,
                        double *L) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nv) return;
    double *row = L + (size_t)a * nv;
    double diag = 0.0;
    for (int e = vstart[a]; e < vstart[a + 1]; e++) {
        const int f = inc_f[e];
        const int v[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
        for (int i = 0; i < 3; i++) {
            // edge (v[i], v[i+1]) opposite corner v[i+2]
            const int p = v[i], q = v[(i + 1) % 3], c = v[(i + 2) % 3];
            if (p != a && q != a) continue;
            const int b = p == a ? q : p;
            if (b == a) continue;
            const double u0 = V[3 * p] - V[3 * c], u1 = V[3 * p + 1] - V[3 * c + 1], u2 = V[3 * p + 2] - V[3 * c + 2];
            const double w0 = V[3 * q] - V[3 * c], w1 = V[3 * q + 1] - V[3 * c + 1], w2 = V[3 * q + 2] - V[3 * c + 2];
            const double dot = u0 * w0 + u1 * w1 + u2 * w2;
            const double x0 = u1 * w2 - u2 * w1, x1 = u2 * w0 - u0 * w2, x2 = u0 * w1 - u1 * w0;
            const double cr = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
            if (!(cr > 0.0)) continue;  // degenerate face: no contribution
            const double wgt = 0.5 * dot / cr;
            row[b] -= wgt;
            diag += wgt;
        }
    }
    row[a] += diag;
}

// Lambda_bary += w (e_s - beta_t)(e_s - beta_t)^T for every recorded walk
// (form 0), or the naive estimator's (Alg. 1) symmetrised
// w [e_s (e_s - beta_t)^T + (e_s - beta_t) e_s^T] / 2 with w = omega_v / W
// (form 1).  walk_w (optional) multiplies each walk's weight.  Row point
// basis: vertex rows e_v; sample rows the centroid of their face (1/3 on each
// of its vertices).
__global__ void k_assemble(const double *V, const int32_t *F, int nv, int n_rows, int W, const int32_t *row_face,
                           const double *omega, const int32_t *exit_tri, const double *exit_bary,
                           const double *walk_w, int form, int exterior, double o0, double o1, double o2, double *L) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n_rows * W) return;
    const int v = (int)(e / W);
    const int t = exit_tri[e];
    if (t < 0) return;
    double w = (form == 0 ? 0.5 : 1.0) * omega[v] / (double)W;
    if (walk_w) w *= walk_w[e];
    if (!(w != 0.0)) return;
    const double *bt = exit_bary + 3 * e;
    const int tv[3] = {F[3 * t], F[3 * t + 1], F[3 * t + 2]};
    if (exterior) {
        double p[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) p[k] += bt[i] * V[3 * tv[i] + k];
        const double d0 = p[0] - o0, d1 = p[1] - o1, d2 = p[2] - o2;
        w *= sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    // sparse d: up to 3 row-point entries and 3 exit entries
    int idx[6];
    double val[6], sv[6];  // d's entries and its row-point part e_s
    int nz = 0;
    if (row_face) {
        const int f = row_face[v];
        for (int i = 0; i < 3; i++) { idx[nz] = F[3 * f + i]; val[nz] = sv[nz] = 1.0 / 3.0; nz++; }
    } else {
        idx[nz] = v; val[nz] = sv[nz] = 1.0; nz++;
    }
    for (int i = 0; i < 3; i++) { idx[nz] = tv[i]; val[nz] = -bt[i]; sv[nz] = 0.0; nz++; }
    for (int i = 0; i < nz; i++)
        for (int j = 0; j < nz; j++) {
            const double x = form == 0 ? w * val[i] * val[j] : w * (0.5 * (sv[i] * val[j] + val[i] * sv[j]));
            if (x != 0.0) atomicAdd(&L[(size_t)idx[i] * nv + idx[j]], x);
        }
}

// lumped killing term: L[u][u] += 4 pi |p_u - o| H0[u] / N0 on the bin vertex u
// (vertex rows; sample rows spread it over the row face's vertices)
__global__ void k_killing(const double *V, const int32_t *F, int nv, int n_rows, const int32_t *row_face,
                          const int32_t *H0, double n_kill, double o0, double o1, double o2, double *L) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_rows || H0[u] == 0) return;
    const double four_pi = 12.566370614359172;
    if (!row_face) {
        const double d0 = V[3 * u] - o0, d1 = V[3 * u + 1] - o1, d2 = V[3 * u + 2] - o2;
        atomicAdd(&L[(size_t)u * nv + u], four_pi * sqrt(d0 * d0 + d1 * d1 + d2 * d2) * H0[u] / n_kill);
        return;
    }
    const int f = row_face[u];
    double c[3];
    for (int k = 0; k < 3; k++) c[k] = (V[3 * F[3 * f] + k] + V[3 * F[3 * f + 1] + k] + V[3 * F[3 * f + 2] + k]) / 3.0;
    const double d0 = c[0] - o0, d1 = c[1] - o1, d2 = c[2] - o2;
    const double x = four_pi * sqrt(d0 * d0 + d1 * d1 + d2 * d2) * H0[u] / n_kill / 9.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) atomicAdd(&L[(size_t)F[3 * f + i] * nv + F[3 * f + j]], x);
}

// Xt = Phi^T (K x n), the tensor-core product's operand layout
__global__ void k_transpose(const double *Phi, int n, int K, double *Xt) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * K) return;
    const int x = (int)(e / K), j = (int)(e % K);
    Xt[(size_t)j * n + x] = Phi[e];
}

// S[a][b] = sum_x Zt[a][x] Phi[x][b], then symmetrised: one block per
// (a, b) pair with a <= b, a fixed-order block reduction
__global__ void k_project_S(const double *Zt, const double *Phi, int n, int K, double *S) {
    __shared__ double red[256];
    const int a = blockIdx.x, b = blockIdx.y;
    if (a > b) return;
    double s1 = 0.0, s2 = 0.0;
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        s1 += Zt[(size_t)a * n + x] * Phi[(size_t)x * K + b];
        s2 += Zt[(size_t)b * n + x] * Phi[(size_t)x * K + a];
    }
    red[threadIdx.x] = 0.5 * (s1 + s2);
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        S[(size_t)a * K + b] = red[0];
        S[(size_t)b * K + a] = red[0];
    }
}

// cyclic Jacobi on a K x K symmetric matrix in FP64, one block: A (rows
// padded to K + 1) in shared memory, the rotations accumulated transposed in
// C (Qt[p][row], so a rotation of columns p, q touches contiguous rows of
// Qt), transposed back at the end.  Eigenvalues ascending into ev (K), eigenvectors in the
// columns of C in the same order.  Stops when the off-diagonal mass is below
// 1e-24 of the total (off-diagonal norm 1e-12 relative: eigenvalue errors of
// order its square over the gaps) or after max_sweeps.
// (the rotations' multiply-adds are explicit fma(): this kernel is bound by
// one SM's FP64 rate)
constexpr int kJacThreads = 256;
__global__ void __launch_bounds__(kJacThreads) k_jacobi64(const double *S, int K, int max_sweeps, double *ev,
                                                          double *C) {
    extern __shared__ double sm[];
    const int ld = K + 1;
    double *A = sm, *Q = C;
    __shared__ double dg[160];
    __shared__ double cs[96], sn[96];
    __shared__ int pp[96], qq[96];
    __shared__ double red_o[kJacThreads / 32], red_t[kJacThreads / 32];
    __shared__ int stop;
    __shared__ int order[160];
    const int Ke = K + (K & 1);  // an odd K gets a dummy index K in the pairing
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int r = e / K, c = e % K;
        A[r * ld + c] = 0.5 * (S[(size_t)r * K + c] + S[(size_t)c * K + r]);
        Q[(size_t)c * K + r] = r == c ? 1.0 : 0.0;
    }
    __syncthreads();
    const int half = Ke / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int sweep = 0; sweep < max_sweeps; sweep++) {
        double o = 0.0, t = 0.0;
        for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
            const int r = e / K, c = e % K;
            const double v = A[r * ld + c] * A[r * ld + c];
            t += v;
            if (r != c) o += v;
        }
        for (int of = 16; of > 0; of >>= 1) {
            o += __shfl_xor_sync(0xFFFFFFFFu, o, of);
            t += __shfl_xor_sync(0xFFFFFFFFu, t, of);
        }
        if (lane == 0) { red_o[warp] = o; red_t[warp] = t; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double so = 0.0, st = 0.0;
            for (int w = 0; w < kJacThreads / 32; w++) { so += red_o[w]; st += red_t[w]; }
            stop = !(so > 1e-24 * st);
        }
        __syncthreads();
        if (stop) break;
        for (int r = 0; r < Ke - 1; r++) {
            // round-robin pairs (p, q) of indices 0..Ke-1; index K (odd K) is idle
            if (threadIdx.x < half) {
                const int i = threadIdx.x;
                int p, q;
                if (i == 0) { p = Ke - 1; q = r; }
                else { p = (r + i) % (Ke - 1); q = (r - i + (Ke - 1)) % (Ke - 1); }
                if (p > q) { const int tt = p; p = q; q = tt; }
                double c = 1.0, s = 0.0;
                if (q < K) {
                    const double apq = A[p * ld + q];
                    if (apq != 0.0) {
                        const double tau = (A[q * ld + q] - A[p * ld + p]) / (2.0 * apq);
                        const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = tt * c;
                    }
                }
                pp[i] = p; qq[i] = q < K ? q : p; cs[i] = c; sn[i] = q < K ? s : 0.0;
            }
            __syncthreads();
            // columns p, q of A and Q
            // one warp per pair, lanes over rows (no index division)
            for (int i = warp; i < half; i += kJacThreads / 32) {
                const int p = pp[i], q = qq[i];
                if (p == q) continue;
                const double c = cs[i], s = sn[i];
                for (int row = lane; row < K; row += 32) {
                    const double ap = A[row * ld + p], aq = A[row * ld + q];
                    A[row * ld + p] = fma(c, ap, -s * aq);
                    A[row * ld + q] = fma(s, ap, c * aq);
                    const double qp = Q[(size_t)p * K + row], qv = Q[(size_t)q * K + row];
                    Q[(size_t)p * K + row] = fma(c, qp, -s * qv);
                    Q[(size_t)q * K + row] = fma(s, qp, c * qv);
                }
            }
            __syncthreads();
            // rows p, q of A
            for (int i = warp; i < half; i += kJacThreads / 32) {
                const int p = pp[i], q = qq[i];
                if (p == q) continue;
                const double c = cs[i], s = sn[i];
                for (int col = lane; col < K; col += 32) {
                    const double ap = A[p * ld + col], aq = A[q * ld + col];
                    A[p * ld + col] = fma(c, ap, -s * aq);
                    A[q * ld + col] = fma(s, ap, c * aq);
                }
            }
            __syncthreads();
        }
    }
    // ascending order of the diagonal (ties by index), by one thread; then C's
    // columns are permuted through shared memory (A's space, no longer needed)
    for (int i = threadIdx.x; i < K; i += blockDim.x) dg[i] = A[i * ld + i];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < K; i++) order[i] = i;
        for (int i = 1; i < K; i++) {
            const int x = order[i];
            const double vx = dg[x];
            int j = i - 1;
            while (j >= 0 && dg[order[j]] > vx) { order[j + 1] = order[j]; j--; }
            order[j + 1] = x;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) A[e] = Q[e];
    __syncthreads();
    for (int i = threadIdx.x; i < K; i += blockDim.x) ev[i] = dg[order[i]];
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int r = e / K, c = e % K;
        C[(size_t)r * K + c] = A[(size_t)order[c] * K + r];  // A holds Qt here
    }
}

// Psi = Phi C[:, :k] (n x k)
__global__ void k_combine_modes(const double *Phi, const double *C, int n, int K, int k, double *Psi) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * k) return;
    const int x = (int)(e / k), j = (int)(e % k);
    double s = 0.0;
    for (int i = 0; i < K; i++) s += Phi[(size_t)x * K + i] * C[(size_t)i * K + j];
    Psi[e] = s;
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
struct Layout {
    size_t L, Xt, Zt, tc, total;
};
static Layout layout(int nv, int K, bool own_L) {
    Layout l;
    size_t o = 0;
    l.L = o;
    if (own_L) o += a256((size_t)nv * nv * sizeof(double));
    l.Xt = o; o += a256((size_t)K * nv * sizeof(double));
    l.Zt = o; o += a256((size_t)K * nv * sizeof(double));
    l.tc = o; o += a256(mcs_tc_symm_product_workspace_size(nv, K));
    l.total = o;
    return l;
}

}  // namespace galerkin
}  // namespace mcs

using namespace mcs;
using namespace mcs::galerkin;

extern "C" {

mcs_status mcs_cotan_laplacian(mcs_mesh m, double *L, void *stream) {
    MCS_ARG(m && L, "mcs_cotan_laplacian: NULL argument");
    cudaStream_t st = as_stream(stream);
    const int nv = m->nv;
    MCS_CUDA(cudaMemsetAsync(L, 0, sizeof(double) * (size_t)nv * nv, st));
    note_launch();
    k_cotan<<<(nv + 127) / 128, 128, 0, st>>>(m->V, m->F, m->inc_f, m->vstart, nv, L);
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

size_t mcs_galerkin_workspace_size(mcs_mesh m, int K, int own_lambda) {
    if (!m || K < 16 || K > 160 || (K % 16)) return 0;
    return layout(m->nv, K, own_lambda != 0).total;
}

mcs_status mcs_galerkin_dtn(mcs_mesh m, const mcs_rows *rows, const int32_t *row_face, const double *omega,
                            const int32_t *exit_tri, const double *exit_bary, const double *walk_w, int form,
                            int walks_per_row, int exterior,
                            const double *origin, const int32_t *H0, long long killing_walks, const double *Phi,
                            int K, double *S, double *Lambda_bary, void *workspace, size_t workspace_bytes,
                            void *stream) {
    MCS_ARG(m && rows && omega && exit_tri && exit_bary && Phi && S, "mcs_galerkin_dtn: NULL argument");
    MCS_ARG(K >= 16 && K <= 160 && K % 16 == 0, "mcs_galerkin_dtn: K must be a multiple of 16 in [16, 160]");
    MCS_ARG(walks_per_row >= 1 && rows->n_rows >= 1, "mcs_galerkin_dtn: need walks_per_row, n_rows >= 1");
    MCS_ARG(row_face || rows->n_rows == m->nv, "mcs_galerkin_dtn: vertex rows need n_rows == nv (else pass row_face)");
    MCS_ARG(!exterior || origin, "mcs_galerkin_dtn: exterior needs the inversion centre");
    MCS_ARG(form == 0 || (form == 1 && !exterior), "mcs_galerkin_dtn: form 0 (jump), or 1 (naive, interior)");
    MCS_ARG(m->nv >= 16, "mcs_galerkin_dtn: need nv >= 16");
    const Layout l = layout(m->nv, K, Lambda_bary == nullptr);
    MCS_ARG(workspace && workspace_bytes >= l.total, "mcs_galerkin_dtn: workspace too small");
    MCS_ARG(((uintptr_t)workspace & 255) == 0, "mcs_galerkin_dtn: workspace must be 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    char *w = (char *)workspace;
    const int nv = m->nv, R = rows->n_rows;
    double *L = Lambda_bary ? Lambda_bary : (double *)(w + l.L);
    const double o0 = exterior ? origin[0] : 0.0, o1 = exterior ? origin[1] : 0.0, o2 = exterior ? origin[2] : 0.0;
    MCS_CUDA(cudaMemsetAsync(L, 0, sizeof(double) * (size_t)nv * nv, st));
    const size_t nw = (size_t)R * walks_per_row;
    note_launch();
    k_assemble<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(m->V, m->F, nv, R, walks_per_row, row_face, omega,
                                                               exit_tri, exit_bary, walk_w, form, exterior, o0, o1,
                                                               o2, L);
    if (exterior && H0 && killing_walks > 0) {
        note_launch();
        k_killing<<<(R + 255) / 256, 256, 0, st>>>(m->V, m->F, nv, R, row_face, H0, (double)killing_walks, o0, o1,
                                                   o2, L);
    }
    double *Xt = (double *)(w + l.Xt), *Zt = (double *)(w + l.Zt);
    note_launch();
    k_transpose<<<(unsigned)(((size_t)nv * K + 255) / 256), 256, 0, st>>>(Phi, nv, K, Xt);
    mcs_status s = mcs_tc_symm_product(L, Xt, nv, K, Zt, w + l.tc, mcs_tc_symm_product_workspace_size(nv, K), stream);
    if (s != MCS_OK) return s;
    note_launch();
    k_project_S<<<dim3(K, K), 256, 0, st>>>(Zt, Phi, nv, K, S);
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

size_t mcs_galerkin_project_workspace_size(int n, int K) {
    if (n < 16 || K < 16 || K > 160 || (K % 16)) return 0;
    return layout(n, K, false).total;
}

mcs_status mcs_galerkin_project(const double *Lambda, const double *Phi, int n, int K, double *S, void *workspace,
                                size_t workspace_bytes, void *stream) {
    MCS_ARG(Lambda && Phi && S, "mcs_galerkin_project: NULL argument");
    MCS_ARG(K >= 16 && K <= 160 && K % 16 == 0, "mcs_galerkin_project: K must be a multiple of 16 in [16, 160]");
    MCS_ARG(n >= 16, "mcs_galerkin_project: need n >= 16");
    const Layout l = layout(n, K, false);
    MCS_ARG(workspace && workspace_bytes >= l.total, "mcs_galerkin_project: workspace too small");
    MCS_ARG(((uintptr_t)workspace & 255) == 0, "mcs_galerkin_project: workspace must be 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    char *w = (char *)workspace;
    double *Xt = (double *)(w + l.Xt), *Zt = (double *)(w + l.Zt);
    note_launch();
    k_transpose<<<(unsigned)(((size_t)n * K + 255) / 256), 256, 0, st>>>(Phi, n, K, Xt);
    mcs_status s = mcs_tc_symm_product(Lambda, Xt, n, K, Zt, w + l.tc, mcs_tc_symm_product_workspace_size(n, K), stream);
    if (s != MCS_OK) return s;
    note_launch();
    k_project_S<<<dim3(K, K), 256, 0, st>>>(Zt, Phi, n, K, S);
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

mcs_status mcs_galerkin_modes(const double *S, int K, int k, const double *Phi, int n, double *evals, double *coeffs,
                              double *psi, void *stream) {
    MCS_ARG(S && evals, "mcs_galerkin_modes: NULL argument");
    MCS_ARG(K >= 2 && K <= 160 && k >= 1 && k <= K, "mcs_galerkin_modes: need 2 <= K <= 160, 1 <= k <= K");
    MCS_ARG(!psi || (Phi && coeffs && n >= 1), "mcs_galerkin_modes: psi needs Phi, coeffs and n");
    cudaStream_t st = as_stream(stream);
    MCS_ARG(coeffs, "mcs_galerkin_modes: coeffs (K x K) is required");
    double *ev = evals, *C = coeffs;
    const size_t smem = (size_t)K * (K + 1) * sizeof(double);
    MCS_CUDA(cudaFuncSetAttribute(k_jacobi64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    note_launch();
    k_jacobi64<<<1, kJacThreads, smem, st>>>(S, K, 60, ev, C);
    if (psi) {
        note_launch();
        k_combine_modes<<<(unsigned)(((size_t)n * k + 255) / 256), 256, 0, st>>>(Phi, C, n, K, k, psi);
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

}  // extern "C"
