// heat.cu -- Steklov heat and heat kernel signatures from computed eigenpairs.
//
// Steklov heat (Sec. 5, Eq. steklovHeat and Eq. spectralSteklovHeat): the
// heat equation du/dt = -Lambda u solved in the Steklov eigenbasis,
//   u_t = sum_j exp(-lambda_j t) a_j psi_j,   a_j = <u_0, psi_j>_M = psi_j^T M u_0,
// for the interior or the exterior operator alike.  Heat kernel signature
// (Sun et al. 2009, the basis-invariant comparison of Sec. 5, Fig.
// hks_comparison):  HKS(x, t) = sum_j exp(-lambda_j t) psi_j(x)^2.
//
// psi is the row-major n x k block of M-orthonormal eigenvectors that
// mcs_steklov_modes writes.  Everything is FP64, and every sum runs in a
// fixed order (no atomics), so results are bitwise reproducible.  The work is
// a few passes over psi (n k doubles): HBM- or L2-bound, not a tensor-core
// contraction.
#include <algorithm>
#include <string>

#include "mcs_internal.h"

namespace mcs {
namespace heat {

constexpr int kRowsPerChunk = 256;  // projection: rows summed per partial
constexpr int kSub = 32;            // rows staged in shared memory at a time
constexpr int kTile = 32;           // channel tile
constexpr int kMaxK = 128;
constexpr int kHksTimes = 16;       // times per HKS decay table in shared memory
constexpr int kSynRows = 16;        // synthesis tile: rows x channels (32.5 KB of shared memory)
constexpr int kSynTile = 16;

// partial[ch][j][cc] = sum over the chunk's rows x of psi[x][j] m[x] u0[x][cc]
__global__ void __launch_bounds__(256) k_project(const double *psi, const double *mass, const double *u0, int n,
                                                 int k, int c, double *partial) {
    __shared__ double sp[kSub][kMaxK];
    __shared__ double su[kSub][kTile];
    const int ch = blockIdx.x, c0 = blockIdx.y * kTile;
    const int cw = min(kTile, c - c0);
    const int x0 = ch * kRowsPerChunk, x1 = min(n, x0 + kRowsPerChunk);
    // thread t owns entries e = t, t + 256, ... of the k x cw tile
    double acc[(kMaxK * kTile) / 256];
    const int ne = k * cw;
#pragma unroll
    for (int q = 0; q < (kMaxK * kTile) / 256; q++) acc[q] = 0.0;
    for (int xs = x0; xs < x1; xs += kSub) {
        const int nr = min(kSub, x1 - xs);
        for (int e = threadIdx.x; e < nr * k; e += blockDim.x) {
            const int r = e / k, j = e % k;
            sp[r][j] = psi[(size_t)(xs + r) * k + j];
        }
        for (int e = threadIdx.x; e < nr * cw; e += blockDim.x) {
            const int r = e / cw, cc = e % cw;
            su[r][cc] = mass[xs + r] * u0[(size_t)(xs + r) * c + c0 + cc];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < (kMaxK * kTile) / 256; q++) {
            const int e = threadIdx.x + 256 * q;
            if (e < ne) {
                const int j = e / cw, cc = e % cw;
                double s = acc[q];
                for (int r = 0; r < nr; r++) s += sp[r][j] * su[r][cc];
                acc[q] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < (kMaxK * kTile) / 256; q++) {
        const int e = threadIdx.x + 256 * q;
        if (e < ne) {
            const int j = e / cw, cc = e % cw;
            partial[((size_t)ch * k + j) * c + c0 + cc] = acc[q];
        }
    }
}

// a[j][cc] = sum of the chunks' partials, in chunk order
__global__ void k_project_sum(const double *partial, int nch, int k, int c, double *a) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * c) return;
    double s = 0.0;
    for (int ch = 0; ch < nch; ch++) s += partial[(size_t)ch * k * c + e];
    a[e] = s;
}

// b[t][j][cc] = exp(-lambda_j t) a[j][cc]: one exponential per (t, j)
__global__ void k_decay_coeffs(const double *evals, const double *times, const double *a, int k, int c, int nt,
                               double *b) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt * k) return;
    const int t = e / k, j = e % k;
    const double d = exp(-evals[j] * times[t]);
    for (int cc = 0; cc < c; cc++) b[((size_t)t * k + j) * c + cc] = d * a[(size_t)j * c + cc];
}

// out[t][x][cc] = sum_j psi[x][j] b[t][j][cc]
__global__ void __launch_bounds__(256) k_synthesize(const double *psi, const double *b, int n, int k, int c,
                                                    double *out) {
    __shared__ double sp[kSynRows][kMaxK + 1];
    __shared__ double sb[kMaxK][kSynTile];
    const int x0 = blockIdx.x * kSynRows, c0 = blockIdx.y * kSynTile, ti = blockIdx.z;
    const int nr = min(kSynRows, n - x0), cw = min(kSynTile, c - c0);
    const double *bt = b + (size_t)ti * k * c;
    for (int e = threadIdx.x; e < k * cw; e += blockDim.x) {
        const int j = e / cw, cc = e % cw;
        sb[j][cc] = bt[(size_t)j * c + c0 + cc];
    }
    for (int e = threadIdx.x; e < nr * k; e += blockDim.x) {
        const int r = e / k, j = e % k;
        sp[r][j] = psi[(size_t)(x0 + r) * k + j];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * cw; e += blockDim.x) {
        const int r = e / cw, cc = e % cw;
        double s = 0.0;
        for (int j = 0; j < k; j++) s += sp[r][j] * sb[j][cc];
        out[((size_t)ti * n + x0 + r) * c + c0 + cc] = s;
    }
}

// out[t][x] = sum_j exp(-lambda_j t) psi[x][j]^2: one warp per row, the
// decay factors of up to kHksTimes times in shared memory
__global__ void __launch_bounds__(256) k_hks(const double *psi, const double *evals, const double *times, int n,
                                             int k, int nt, int t0, double *out) {
    __shared__ double dec[kHksTimes][kMaxK];
    const int tw = min(kHksTimes, nt - t0);
    for (int e = threadIdx.x; e < tw * k; e += blockDim.x) {
        const int ti = e / k, j = e % k;
        dec[ti][j] = exp(-evals[j] * times[t0 + ti]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int x = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (x >= n) return;
    double sq[kMaxK / 32];
#pragma unroll
    for (int q = 0; q < kMaxK / 32; q++) {
        const int j = lane + 32 * q;
        const double v = j < k ? psi[(size_t)x * k + j] : 0.0;
        sq[q] = v * v;
    }
    for (int ti = 0; ti < tw; ti++) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < kMaxK / 32; q++) {
            const int j = lane + 32 * q;
            if (j < k) s += dec[ti][j] * sq[q];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if (lane == 0) out[(size_t)(t0 + ti) * n + x] = s;
    }
}

// workspace: per-chunk partials, a (k x c), b for up to kHeatTimes times
constexpr int kHeatTimes = 64;  // times per synthesis pass
static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
static size_t heat_ws(int n, int k, int c) {
    const size_t nch = (size_t)(n + kRowsPerChunk - 1) / kRowsPerChunk;
    return a256(nch * k * c * sizeof(double)) + a256((size_t)k * c * sizeof(double)) +
           (size_t)kHeatTimes * k * c * sizeof(double);
}

}  // namespace heat
}  // namespace mcs

using namespace mcs;
using namespace mcs::heat;

extern "C" {

size_t mcs_steklov_heat_workspace_size(int n, int k, int c) {
    if (n <= 0 || k <= 0 || c <= 0) return 0;
    return heat_ws(n, k, c);
}

mcs_status mcs_steklov_heat(const double *evals, const double *evecs, const double *mass, int n, int k,
                            const double *u0, int c, const double *times, int nt, double *out, void *workspace,
                            size_t workspace_bytes, void *stream) {
    MCS_ARG(evals && evecs && mass && u0 && times && out, "mcs_steklov_heat: NULL argument");
    MCS_ARG(n >= 1 && k >= 1 && k <= kMaxK && c >= 1 && nt >= 1, "mcs_steklov_heat: need n, c, nt >= 1, 1 <= k <= 128");
    const size_t need = heat_ws(n, k, c);
    MCS_ARG(workspace && workspace_bytes >= need, "mcs_steklov_heat: workspace too small");
    MCS_ARG(((uintptr_t)workspace & 255) == 0, "mcs_steklov_heat: workspace must be 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    const int nch = (n + kRowsPerChunk - 1) / kRowsPerChunk;
    double *partial = (double *)workspace;
    double *a = (double *)((char *)workspace + a256((size_t)nch * k * c * sizeof(double)));
    double *b = (double *)((char *)a + a256((size_t)k * c * sizeof(double)));
    const int ct = (c + kTile - 1) / kTile;
    note_launch();
    k_project<<<dim3(nch, ct), 256, 0, st>>>(evecs, mass, u0, n, k, c, partial);
    note_launch();
    k_project_sum<<<(k * c + 255) / 256, 256, 0, st>>>(partial, nch, k, c, a);
    // kHeatTimes times per pass: their coefficient tables, then the grid's z
    // dimension carries the times
    for (int t0 = 0; t0 < nt; t0 += kHeatTimes) {
        const int tn = std::min(kHeatTimes, nt - t0);
        note_launch();
        k_decay_coeffs<<<(tn * k + 255) / 256, 256, 0, st>>>(evals, times + t0, a, k, c, tn, b);
        note_launch();
        k_synthesize<<<dim3((n + kSynRows - 1) / kSynRows, (c + kSynTile - 1) / kSynTile, tn), 256, 0, st>>>(
            evecs, b, n, k, c, out + (size_t)t0 * n * c);
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

mcs_status mcs_hks(const double *evals, const double *evecs, int n, int k, const double *times, int nt, double *out,
                   void *stream) {
    MCS_ARG(evals && evecs && times && out, "mcs_hks: NULL argument");
    MCS_ARG(n >= 1 && k >= 1 && k <= kMaxK && nt >= 1, "mcs_hks: need n, nt >= 1, 1 <= k <= 128");
    cudaStream_t st = as_stream(stream);
    const int rows_per_block = 256 / 32;
    for (int t0 = 0; t0 < nt; t0 += kHksTimes) {
        note_launch();
        k_hks<<<(n + rows_per_block - 1) / rows_per_block, 256, 0, st>>>(evecs, evals, times, n, k, nt, t0, out);
    }
    MCS_CUDA(cudaGetLastError());
    return MCS_OK;
}

}  // extern "C"
