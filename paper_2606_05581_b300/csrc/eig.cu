// eig.cu -- Steklov eigenpairs: smallest k eigenpairs of M^-1/2 Lambda M^-1/2
// (Eq. steklov-eigenproblem in Galerkin form Lambda psi = lambda M psi).
//
// Chebyshev-filtered subspace iteration (Zhou & Saad 2007) on a block of
// m = k + guard vectors:
//   filter     Y <- p_d(A) Y by the scaled three-term recurrence; each term is
//              one A*Y product on the tensor cores (tcgen05, kind::tf32) with
//              A and Y split into tf32 high/low parts (hi*hi + hi*lo + lo*hi,
//              FP32-level accuracy), fed by TMA into 128B-swizzled shared
//              memory, accumulated in TMEM, split over K and combined by a
//              deterministic FP32 kernel that also applies the recurrence;
//   orthonorm  CholeskyQR2 in FP64, preceded on the start block by a shifted
//              CholeskyQR (CholeskyQR3); after a filter the first pass turns
//              into the shifted one when it meets a pivot that is not
//              clearly positive, and a third pass follows;
//   Rayleigh-Ritz  H = X^T A X (FP64 Gram of the tensor-core product), its
//              eigenvectors by a parallel cyclic Jacobi in FP32 on one SM, the
//              rotated block re-orthonormalised in FP64 at the next step;
//              Ritz values as FP64 Rayleigh quotients.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mcs_internal.h"

namespace mcs {
namespace eig {

constexpr int BM = 128;          // rows of A per CTA (MMA M)
constexpr int BK = 32;           // K per pipeline stage: 32 fp32 = one 128-byte swizzle row
constexpr int kTcThreads = 128;  // 4 warps: TMA producer, MMA issuer, all four drain TMEM
constexpr int kErrTimeout = 16;  // an mbarrier wait exceeded its time bound
constexpr int kErrChol = 32;     // Cholesky met a non-positive pivot

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// bounded wait: gives up after ~2 s of wall time and sets the error flag
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; it++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 0) {
            const uint64_t t = gtime();
            if (t0 == 0) t0 = t;
            else if (t - t0 > 2000000000ull) {
                atomicOr(err, kErrTimeout);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *tm, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"((uint64_t)tm), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}
// tcgen05 shared-memory descriptor: K-major operand, 128-byte swizzle,
// 8-row core groups 1024 bytes apart (SBO), descriptor version 1
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // SBO
    d |= (uint64_t)1 << 46;             // version
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

struct TcArgs {
    float *part;     // splits x m x n_pad partial products, transposed (column-major in rows)
    int n_pad, m;
    int ktiles, kt_per_split;
    int stages;
    uint32_t idesc;
    uint32_t tmem_cols;
    int *err;
};

// P[split][j][i] = sum_{k in split} A[i][k] * Bt[j][k] with A = Ahi + Alo and
// Bt = Bhi + Blo (tf32 parts); CTA (tile, split) owns rows [128 tile, +128)
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
              const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl, TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[4], empty[4], done;
    __shared__ uint32_t tmem_slot;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * BM;
    const int kt0 = blockIdx.y * a.kt_per_split;
    const int nk = min(a.ktiles, kt0 + a.kt_per_split) - kt0;
    const int m = a.m, S = a.stages;
    const uint32_t A_BYTES = BM * 128, B_BYTES = (uint32_t)m * 128;
    const uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;
    const uint32_t sbase = smem_u32(smem);
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int issued = 0;
        for (int it = 0; it < nk && ok; it++) {
            const int s = it % S, r = it / S;
            if (r > 0 && !mbar_wait(smem_u32(&empty[s]), (r - 1) & 1, a.err)) { ok = false; break; }
            const uint32_t bar = smem_u32(&full[s]);
            mbar_expect_tx(bar, STAGE);
            const uint32_t st = sbase + s * STAGE;
            const int k = (kt0 + it) * BK;
            tma_load_2d(st, &tAh, k, row0, bar);
            tma_load_2d(st + A_BYTES, &tAl, k, row0, bar);
            tma_load_2d(st + 2 * A_BYTES, &tBh, k, 0, bar);
            tma_load_2d(st + 2 * A_BYTES + B_BYTES, &tBl, k, 0, bar);
            issued = it + 1;
        }
        // do not leave with copies in flight: wait (bounded) for the last stages
        for (int it = (issued > S ? issued - S : 0); it < issued; it++)
            mbar_wait(smem_u32(&full[it % S]), (it / S) & 1, a.err);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: 4 K-steps of 8 per stage, three split products each
        for (int it = 0; it < nk; it++) {
            const int s = it % S, r = it / S;
            if (!mbar_wait(smem_u32(&full[s]), r & 1, a.err)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = sbase + s * STAGE;
#pragma unroll
            for (int kk = 0; kk < BK / 8; kk++) {
                const uint64_t ah = sdesc_sw128(st + kk * 32), al = sdesc_sw128(st + A_BYTES + kk * 32);
                const uint64_t bh = sdesc_sw128(st + 2 * A_BYTES + kk * 32);
                const uint64_t bl = sdesc_sw128(st + 2 * A_BYTES + B_BYTES + kk * 32);
                mma_tf32(tmem, ah, bh, a.idesc, (it > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, ah, bl, a.idesc, 1u);
                mma_tf32(tmem, al, bh, a.idesc, 1u);
            }
            mma_commit(smem_u32(&empty[s]));
        }
        mma_commit(smem_u32(&done));
    }
    __syncwarp();
    // drain the accumulator: warp w owns TMEM lanes (rows) 32w .. 32w+31
    const bool got = mbar_wait(smem_u32(&done), 0, a.err);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (got) {
        const int row = row0 + warp * 32 + lane;
        float *P = a.part + (size_t)blockIdx.y * m * a.n_pad;
        for (int c = 0; c < m; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 16; j++) P[(size_t)(c + j) * a.n_pad + row] = v[j];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

// ---------------------------------------------------------------- SIMT kernels
// sinv = M^-1/2 (FP64, once per solve: B300's FP64 divide and square root
// are too slow to repeat per matrix entry)
__global__ void k_inv_sqrt(const double *mass, int n, double *sinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sinv[i] = 1.0 / sqrt(mass[i]);
}

// A = M^-1/2 Lambda M^-1/2 as tf32 high/low parts (zero padded), and the
// absolute row sums of A (Gershgorin bound of its spectrum)
__global__ void k_prep_A(const double *L, const double *sinv, int n, int n_pad, float *Ahi, float *Alo,
                         double *rowabs) {
    const int i = blockIdx.x;
    __shared__ double red[256];
    double acc = 0.0;
    const double si = i < n ? sinv[i] : 0.0;
    for (int j = threadIdx.x; j < n_pad; j += blockDim.x) {
        float h = 0.f, l = 0.f;
        if (i < n && j < n) {
            const double v = L[(size_t)i * n + j] * (si * sinv[j]);
            acc += fabs(v);
            const float f = (float)v;
            h = __uint_as_float(__float_as_uint(f) & 0xFFFFE000u);
            l = f - h;
        }
        Ahi[(size_t)i * n_pad + j] = h;
        Alo[(size_t)i * n_pad + j] = l;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && i < n && rowabs) rowabs[i] = red[0];
}

__global__ void k_max_reduce(const double *x, int n, double *out) {
    __shared__ double red[1024];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, x[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// deterministic start block: Philox uniforms in (-1, 1)
__global__ void k_random_block(double *Xt, int m, int n, int n_pad) {
    const size_t total = (size_t)m * n_pad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n_pad), i = (int)(e % n_pad);
        double v = 0.0;
        if (i < n) {
            const uint4 w = philox(make_uint4((uint32_t)i, (uint32_t)j, 0x5EEDu, 0u), 0x1234567u, 0x89ABCDEu);
            v = 2.0 * uni64(w.x, w.y) - 1.0;
        }
        Xt[e] = v;
    }
}

// FP64 block -> tf32 high/low parts
__global__ void k_split(const double *X, size_t total, float *hi, float *lo) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const float f = (float)X[e];
        const float h = __uint_as_float(__float_as_uint(f) & 0xFFFFE000u);
        hi[e] = h;
        lo[e] = f - h;
    }
}

// out = alpha * (sum of the K-split partials) + beta * Y + gamma * X, for
// rows < n (padding stays zero); written as tf32 parts and/or FP64
__global__ void k_combine(const float *P, int splits, int m, int n, int n_pad, double alpha, double beta,
                          double gamma, const float *Yh, const float *Yl, const float *Xh, const float *Xl,
                          float *Oh, float *Ol, double *O64) {
    const size_t total = (size_t)m * n_pad;
    const size_t stride = (size_t)m * n_pad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n_pad);
        float r = 0.f;
        if (i < n) {
            float s = 0.f;
            for (int q = 0; q < splits; q++) s += P[q * stride + e];
            double v = alpha * (double)s;
            if (Yh) v += beta * ((double)Yh[e] + (double)Yl[e]);
            if (Xh) v += gamma * ((double)Xh[e] + (double)Xl[e]);
            if (O64) O64[e] = v;
            r = (float)v;
        } else if (O64) {
            O64[e] = 0.0;
        }
        if (Oh) {
            const float h = __uint_as_float(__float_as_uint(r) & 0xFFFFE000u);
            Oh[e] = h;
            Ol[e] = r - h;
        }
    }
}

// The FP64 products below (Gram, Cholesky, triangular inverse, block times)
// are bound by B300's FP64 rate, so their multiply-adds are explicit fma()
// (one instruction, one rounding); the library is otherwise built without
// contraction.
// Gp[q][a][b] = sum_{i in chunk q} A[a][i] B[b][i] (FP64): 32 x 32 output
// tiles per block, the n dimension split into gridDim.z chunks.  For
// B = A (upper != 0) only the tiles on and above the diagonal are formed: an
// entry and its mirror are the same products in the same order, so the lower
// tiles would repeat the upper ones bit for bit.
constexpr int kGramChunksMax = 64;
__global__ void k_gram_part(const double *A, const double *B, int m, int n_pad, double *Gp, int upper) {
    __shared__ double sa[32][33], sb[32][33];
    if (upper && blockIdx.y > blockIdx.x) return;
    const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
    const int chunk = (n_pad + gridDim.z - 1) / gridDim.z;
    const int i0 = blockIdx.z * chunk, i1 = min(n_pad, i0 + chunk);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    double acc[4] = {0, 0, 0, 0};
    for (int i = i0; i < i1; i += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int ii = i + tx;
            sa[r][tx] = (a0 + r < m && ii < i1) ? A[(size_t)(a0 + r) * n_pad + ii] : 0.0;
            sb[r][tx] = (b0 + r < m && ii < i1) ? B[(size_t)(b0 + r) * n_pad + ii] : 0.0;
        }
        __syncthreads();
        for (int q = 0; q < 4; q++) {
            const int r = ty + 8 * q;
            double s = 0.0;
            for (int t = 0; t < 32; t++) s = fma(sa[r][t], sb[tx][t], s);
            acc[q] += s;
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; q++) {
        const int r = ty + 8 * q;
        if (a0 + r < m && b0 + tx < m) Gp[((size_t)blockIdx.z * m + a0 + r) * m + b0 + tx] = acc[q];
    }
}
__global__ void k_gram_reduce(const double *Gp, int m, int chunks, double *G, int sym, int upper) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    double s = 0.0;
    if (upper) {
        // (a, b) from the tile on or above the diagonal; exactly symmetric
        const int a = e / m, b = e % m;
        const int src = (a >> 5) <= (b >> 5) ? e : b * m + a;
        for (int q = 0; q < chunks; q++) s += Gp[(size_t)q * m * m + src];
        G[e] = s;
        return;
    }
    for (int q = 0; q < chunks; q++) s += Gp[(size_t)q * m * m + e];
    if (sym) {
        const int a = e / m, b = e % m;
        double t = 0.0;
        for (int q = 0; q < chunks; q++) t += Gp[(size_t)q * m * m + b * m + a];
        s = 0.5 * (s + t);
    }
    G[e] = s;
}

// R^-1 for the upper Cholesky factor R of G (+ shift I, shift = shift_rel *
// trace G), FP64, one block of 1024 threads, S = m x (m + 1) in shared memory.
// B300's FP64 pipe is narrow: each step's elements are spread densely over
// all 1024 threads (full lanes in every FP64 warp instruction), and the FP64
// divides and square roots are done once per pivot.
//  1. right-looking elimination on the upper triangle without square roots:
//     w[a] = S[j][a] / S[j][j], then S[a][b] -= w[a] S[j][b] for j < a <= b
//     (the trailing triangle enumerated from its bottom row up);
//  2. R[j][c] = S[j][c] / sqrt(S[j][j]); R's diagonal is 1 / rs;
//  3. Z = R^-1, right-looking from the bottom row: once row k of Z is final,
//     every row r < k takes acc[r][c] += R[r][k] Z[k][c] (c >= k, Z[k][k] =
//     rs[k]), and row k - 1, whose sum is then complete, becomes
//     Z[k-1][c] = -rs[k-1] acc[k-1][c]; Z's strict upper part lives transposed
//     in S's strict lower triangle.
// mode 0: no shift; 1: shift; 2: no shift first, and on a pivot <= 1e-15 *
// trace a restart with the shift, reported in *shifted.  A pivot that is
// still not positive sets kErrChol and is replaced by 1e-300.
__global__ void __launch_bounds__(1024) k_chol_inv(const double *G, int m, double shift_rel, int mode, double *Rinv,
                                                   int *shifted, int *err) {
    extern __shared__ double S[];  // m x (m + 1)
    __shared__ double w[160], rs[160];
    __shared__ double tr, inv;
    __shared__ int bad;
    const int ld = m + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        double t = 0.0;
        for (int j = lane; j < m; j += 32) t += G[j * m + j];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
        if (lane == 0) tr = t;
    }
    int used_shift = 0;
    for (int attempt = mode == 1 ? 1 : 0; attempt < 2; attempt++) {
        used_shift = attempt;
        __syncthreads();
        const double shift = attempt ? shift_rel * tr : 0.0;
        const double floor_piv = mode == 2 && attempt == 0 ? 1e-15 * tr : 0.0;
        for (int e = tid; e < m * m; e += nt) {
            const int r = e / m, c = e % m;
            S[r * ld + c] = G[e] + (r == c ? shift : 0.0);
        }
        if (tid == 0) {
            bad = 0;
            double d = S[0];
            if (!(d > floor_piv)) {
                if (floor_piv > 0.0) bad = 1;
                else atomicOr(err, kErrChol);
                d = S[0] = 1e-300;
            }
            inv = 1.0 / d;
        }
        __syncthreads();
        for (int j = 0; j < m - 1; j++) {
            for (int a = j + 1 + tid; a < m; a += nt) w[a] = S[j * ld + a] * inv;
            __syncthreads();
            // trailing triangle rows a > j, columns b >= a: element e counts
            // from the bottom row (row m - 1 - s holds s + 1 elements); the
            // thread that updates the next pivot checks it and forms its
            // reciprocal (inv is no longer read in this step)
            const int T = (m - j - 1) * (m - j) / 2;
            for (int e = tid; e < T; e += nt) {
                int s = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                while ((s + 1) * (s + 2) / 2 <= e) s++;
                while (s * (s + 1) / 2 > e) s--;
                const int a = m - 1 - s, b = a + (e - s * (s + 1) / 2);
                double v = fma(-w[a], S[j * ld + b], S[a * ld + b]);
                if (a == j + 1 && b == a) {
                    if (!(v > floor_piv)) {
                        if (floor_piv > 0.0) bad = 1;
                        else atomicOr(err, kErrChol);
                        v = 1e-300;
                    }
                    inv = 1.0 / v;
                }
                S[a * ld + b] = v;
            }
            __syncthreads();
        }
        if (!bad) break;  // uniform: read after the barrier
    }
    if (tid == 0 && shifted) *shifted = used_shift;
    for (int j = tid; j < m; j += nt) rs[j] = 1.0 / sqrt(S[j * ld + j]);
    __syncthreads();
    for (int e = tid; e < m * m; e += nt) {
        const int r = e / m, c = e % m;
        if (c > r) S[r * ld + c] *= rs[r];
        else if (c < r) S[r * ld + c] = 0.0;
    }
    __syncthreads();
    // R's diagonal is 1 / rs; R^-1[k][c] (k < c) lives at S[c][k], its diagonal in rs
    for (int k = m - 1; k >= 1; k--) {
        const int wdt = m - k;  // columns c = k .. m - 1 of rows r = 0 .. k - 1
        const float rw = 1.f / (float)wdt;
        const double zk = rs[k];
        for (int e = tid; e < k * wdt; e += nt) {
            // r = e / wdt exactly: (e + 0.5) / wdt stays at least 0.5 / wdt
            // away from an integer, far beyond the FP32 error for e < 2^14
            const int r = (int)(((float)e + 0.5f) * rw), c = k + (e - r * wdt);
            double v = fma(S[r * ld + k], c == k ? zk : S[c * ld + k], S[c * ld + r]);
            if (r == k - 1) v *= -rs[r];
            S[c * ld + r] = v;
        }
        __syncthreads();
    }
    for (int e = tid; e < m * m; e += nt) {
        const int r = e / m, c = e % m;
        Rinv[e] = c > r ? S[c * ld + r] : c == r ? rs[r] : 0.0;
    }
}

__global__ void k_f32_to_f64(const float *a, int n, double *b) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = (double)a[e];
}

// Out[j][i] = sum_k C[k][j] In[k][i] (FP64): X <- X C for a block stored by
// rows of X^T; eight output rows j per block, C's slice in shared memory.
// For an upper-triangular C (tri != 0) the sum stops at the block's last j:
// the skipped terms are exact zeros.
constexpr int kJG = 8;
__global__ void k_block_times(const double *C, const double *In, int m, int n_pad, double *Out, int tri) {
    extern __shared__ double sc[];  // m x kJG
    const int j0 = blockIdx.y * kJG;
    for (int e = threadIdx.x; e < m * kJG; e += blockDim.x) {
        const int k = e / kJG, jj = e % kJG;
        sc[e] = (j0 + jj < m) ? C[k * m + j0 + jj] : 0.0;
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    double acc[kJG];
#pragma unroll
    for (int jj = 0; jj < kJG; jj++) acc[jj] = 0.0;
    const int kend = tri ? min(m, j0 + kJG) : m;
    for (int k = 0; k < kend; k++) {
        const double x = In[(size_t)k * n_pad + i];
#pragma unroll
        for (int jj = 0; jj < kJG; jj++) acc[jj] = fma(sc[k * kJG + jj], x, acc[jj]);
    }
#pragma unroll
    for (int jj = 0; jj < kJG; jj++)
        if (j0 + jj < m) Out[(size_t)(j0 + jj) * n_pad + i] = acc[jj];
}

// Ritz values theta_j = x_j.z_j / x_j.x_j and residual norms |z_j - theta_j x_j|
__global__ void k_ritz(const double *Xt, const double *Zt, int n_pad, double *theta, double *res) {
    const int j = blockIdx.x;
    __shared__ double r1[256], r2[256], r3[256];
    const double *x = Xt + (size_t)j * n_pad, *z = Zt + (size_t)j * n_pad;
    double xz = 0, xx = 0, zz = 0;
    for (int i = threadIdx.x; i < n_pad; i += blockDim.x) { xz += x[i] * z[i]; xx += x[i] * x[i]; zz += z[i] * z[i]; }
    r1[threadIdx.x] = xz; r2[threadIdx.x] = xx; r3[threadIdx.x] = zz;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) { r1[threadIdx.x] += r1[threadIdx.x + s]; r2[threadIdx.x] += r2[threadIdx.x + s]; r3[threadIdx.x] += r3[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double t = r1[0] / r2[0];
        theta[j] = t;
        res[j] = sqrt(fmax(r3[0] - 2.0 * t * r1[0] + t * t * r2[0], 0.0) / r2[0]);
    }
}

// symmetric eigendecomposition of H (m x m, m even <= 160) by parallel cyclic
// Jacobi (round-robin pair schedule) in FP32, one block; eigenvalues ascending,
// eigenvectors in the columns of Q.  Shared rows are padded to m + 1 floats so
// that column sweeps hit distinct banks.
__global__ void k_jacobi(const double *Hd, int m, float *Q, float *evals, int max_sweeps, int *sweeps_done) {
    extern __shared__ float sj[];
    const int ld = m + 1;
    float *H = sj, *V = sj + m * ld;
    __shared__ float cs[2][80], sn[2][80];  // rotations of the current and the next round
    __shared__ int pp[2][80], qq[2][80];
    __shared__ float red_off[32], red_tot[32];
    __shared__ int stop;
    float prev_off = 0.f;  // thread 0's
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int r = e / m, c = e % m;
        H[r * ld + c] = (float)(0.5 * (Hd[r * m + c] + Hd[c * m + r]));
        V[r * ld + c] = r == c ? 1.f : 0.f;
    }
    __syncthreads();
    const int half = m / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // pair i of round r (round-robin: m - 1 fixed, the others rotate) and its
    // rotation from the current H; c = 1 / sqrt(1 + t^2) by rsqrtf: the
    // rotations need be orthogonal only to FP32 rounding, the block they
    // rotate is re-orthonormalised in FP64 afterwards
    auto rotation = [&](int r, int i, int buf) {
        int p, q;
        if (i == 0) {
            p = m - 1;
            q = r;
        } else {
            p = r + i;
            if (p >= m - 1) p -= m - 1;
            q = r - i;
            if (q < 0) q += m - 1;
        }
        if (p > q) {
            const int tt = p;
            p = q;
            q = tt;
        }
        pp[buf][i] = p;
        qq[buf][i] = q;
        const float apq = H[p * ld + q];
        float c = 1.f, sv = 0.f;
        if (fabsf(apq) > 1e-30f) {
            const float tau = (H[q * ld + q] - H[p * ld + p]) / (2.f * apq);
            const float tt = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + tt * tt);
            sv = tt * c;
        }
        cs[buf][i] = c;
        sn[buf][i] = sv;
    };
    for (int sweep = 0; sweep < max_sweeps; sweep++) {
        float o = 0.f, t = 0.f;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int r = e / m, c = e % m;
            const float v = H[r * ld + c] * H[r * ld + c];
            t += v;
            if (r != c) o += v;
        }
        for (int of = 16; of > 0; of >>= 1) {
            o += __shfl_xor_sync(0xFFFFFFFFu, o, of);
            t += __shfl_xor_sync(0xFFFFFFFFu, t, of);
        }
        if (lane == 0) { red_off[warp] = o; red_tot[warp] = t; }
        __syncthreads();
        if (threadIdx.x == 0) {
            float so = 0.f, st = 0.f;
            for (int w = 0; w < nwarps; w++) { so += red_off[w]; st += red_tot[w]; }
            // converged, or at FP32's rounding floor: a sweep that no longer
            // halves the off-diagonal norm has stopped converging quadratically
            stop = so <= 1e-12f * st || (sweep >= 4 && so > 0.25f * prev_off);
            prev_off = so;
        }
        __syncthreads();
        if (stop) {
            if (threadIdx.x == 0) *sweeps_done += sweep;
            break;
        }
        if (sweep == max_sweeps - 1 && threadIdx.x == 0) *sweeps_done += max_sweeps;
        if (threadIdx.x < half) rotation(0, threadIdx.x, 0);
        __syncthreads();
        for (int r = 0; r < m - 1; r++) {
            const int cur = r & 1;
            // H <- J^T H J by 2 x 2 blocks: block (a, b) holds rows {p_a, q_a}
            // and columns {p_b, q_b}; the column rotation of pair b, then the
            // row rotation of pair a (the order of a column pass followed by
            // a row pass), written to (a, b) and mirrored to (b, a).  One warp
            // per pair a, lanes over b >= a.  Blocks are disjoint.
            for (int a = warp; a < half; a += nwarps) {
                const int pa = pp[cur][a], qa = qq[cur][a];
                const float ca = cs[cur][a], sa = sn[cur][a];
                for (int b = a + lane; b < half; b += 32) {
                    const int pb = pp[cur][b], qb = qq[cur][b];
                    const float cb = cs[cur][b], sb = sn[cur][b];
                    const float b00 = H[pa * ld + pb], b01 = H[pa * ld + qb];
                    const float b10 = H[qa * ld + pb], b11 = H[qa * ld + qb];
                    const float c00 = cb * b00 - sb * b01, c01 = sb * b00 + cb * b01;
                    const float c10 = cb * b10 - sb * b11, c11 = sb * b10 + cb * b11;
                    const float d00 = ca * c00 - sa * c10, d10 = sa * c00 + ca * c10;
                    const float d01 = ca * c01 - sa * c11, d11 = sa * c01 + ca * c11;
                    H[pa * ld + pb] = d00;
                    H[pa * ld + qb] = d01;
                    H[qa * ld + pb] = d10;
                    H[qa * ld + qb] = d11;
                    if (b != a) {
                        H[pb * ld + pa] = d00;
                        H[qb * ld + pa] = d01;
                        H[pb * ld + qa] = d10;
                        H[qb * ld + qa] = d11;
                    }
                }
            }
            __syncthreads();
            // the next round's rotations (from the rotated H) while the
            // others rotate V <- V J, one warp per pair, lanes over rows
            if (r + 1 < m - 1 && threadIdx.x < half) rotation(r + 1, threadIdx.x, cur ^ 1);
            for (int i = warp; i < half; i += nwarps) {
                const int p = pp[cur][i], q = qq[cur][i];
                const float c = cs[cur][i], sv = sn[cur][i];
                for (int row = lane; row < m; row += 32) {
                    const float vp = V[row * ld + p], vq = V[row * ld + q];
                    V[row * ld + p] = c * vp - sv * vq;
                    V[row * ld + q] = sv * vp + c * vq;
                }
            }
            __syncthreads();
        }
    }
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const float d = H[j * ld + j];
        int rank = 0;
        for (int k = 0; k < m; k++) {
            const float e = H[k * ld + k];
            rank += (e < d) || (e == d && k < j);
        }
        evals[rank] = d;
        for (int r = 0; r < m; r++) Q[r * m + rank] = V[r * ld + j];
    }
}

// ---------------------------------------------------------------- sparse product
// A Lambda estimated from walk histograms is mostly zeros when its rows are
// sample points of a large surface (each row only reaches the bins its walks
// exit in).  Then A = M^-1/2 Lambda M^-1/2 is kept in CSR (FP32 values, the
// same rounding of each entry as the dense path's before its tf32 split,
// columns ascending) and each filter term is one fused SIMT kernel reading
// the block vectors by rows (V[i][j], n_pad x m FP32).

// pass 1: nonzeros of row i of A (entries that round to a nonzero float) and
// its absolute row sum (Gershgorin bound); one block per row
__global__ void k_row_stats(const double *L, const double *sinv, int n, long long *cnt, double *rowabs) {
    const int i = blockIdx.x;
    __shared__ double red[256];
    __shared__ int redc[256];
    const double si = sinv[i];
    double acc = 0.0;
    int c = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        // zeros (most of a histogram Lambda) are skipped by an integer test of
        // the bits: they add nothing, and B300's FP64 pipe is narrow
        const double l = L[(size_t)i * n + j];
        if ((__double_as_longlong(l) << 1) == 0) continue;
        const double v = l * (si * sinv[j]);
        acc += fabs(v);
        c += (float)v != 0.f;
    }
    red[threadIdx.x] = acc;
    redc[threadIdx.x] = c;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[threadIdx.x] += red[threadIdx.x + s];
            redc[threadIdx.x] += redc[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rowabs[i] = red[0];
        cnt[i + 1] = redc[0];
    }
}

// in-place inclusive scan of rp[1..n] (rp[0] = 0): one block of 1024 threads,
// each owning a contiguous chunk
__global__ void k_row_scan(long long *rp, int n) {
    __shared__ long long part[1024];
    const int t = threadIdx.x, chunk = (n + 1023) / 1024;
    const int a = 1 + t * chunk, b = min(n + 1, a + chunk);
    long long s = 0;
    for (int i = a; i < b; i++) s += rp[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = t > 0 ? part[t - 1] : 0;
    for (int i = a; i < b; i++) {
        run += rp[i];
        rp[i] = run;
    }
    if (t == 0) rp[0] = 0;
}

// pass 2: row i's nonzeros in ascending column order; one block per row, the
// columns in chunks of 256 compacted by warp ballots
__global__ void k_csr_fill(const double *L, const double *sinv, int n, const long long *rp, float *vals, int *cols) {
    const int i = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int wcount[8];
    const double si = sinv[i];
    long long base = rp[i];
    for (int j0 = 0; j0 < n; j0 += 256) {
        const int j = j0 + threadIdx.x;
        float f = 0.f;
        if (j < n) {
            const double l = L[(size_t)i * n + j];
            if ((__double_as_longlong(l) << 1) != 0) f = (float)(l * (si * sinv[j]));
        }
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, f != 0.f);
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < 8; w++) {
            off += w < warp ? wcount[w] : 0;
            tot += wcount[w];
        }
        if (f != 0.f) {
            const long long e = base + off + __popc(bal & ((1u << lane) - 1u));
            vals[e] = f;
            cols[e] = j;
        }
        base += tot;
        __syncthreads();
    }
}

// FP64 block by rows of X^T (m x n_pad) -> FP32 block by rows of X (n_pad x m)
__global__ void k_to_rows(const double *Xt, int m, int n_pad, float *V) {
    __shared__ float tile[32][33];
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int r = ty; r < 32; r += 8)
        if (j0 + r < m) tile[r][tx] = (float)Xt[(size_t)(j0 + r) * n_pad + i0 + tx];
    __syncthreads();
    for (int r = ty; r < 32; r += 8)
        if (j0 + tx < m) V[(size_t)(i0 + r) * m + j0 + tx] = tile[tx][r];
}

// one filter term on the CSR operator:
//   O = alpha A Y + beta Y + gamma X   (rows < n; padding rows stay zero)
// with Y, X and O by rows (FP32) and, where O64 is given, O also as FP64 by
// rows of O^T.  One warp per row of A and lanes over the block's columns;
// the products accumulate in FP32 with explicit fmaf in ascending column
// order.  A term that continues the recurrence combines in FP32 (its result is
// stored in FP32, and B300's FP64 pipe would bound the kernel); the last term,
// which writes X in FP64, combines in FP64 like the dense path's k_combine.
// A block is
// 32 warps on 32 consecutive rows (one row each, so that short rows still put
// many warps in flight), and the FP64 output leaves through shared memory in
// coalesced rows of O^T.
constexpr int kSpRows = 32;
template <int JW>
__global__ void __launch_bounds__(1024) k_sp_filter(const long long *rp, const int *cols, const float *vals, int n,
                                                    int n_pad, int m, double alpha, double beta, double gamma,
                                                    float alpha_f, float beta_f, float gamma_f, const float *Y,
                                                    const float *X, float *O, double *O64) {
    __shared__ double s64[kSpRows][JW * 32 + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = blockIdx.x * kSpRows;
    {
        const int r = warp;
        const int i = i0 + r;
        float acc[JW];
#pragma unroll
        for (int q = 0; q < JW; q++) acc[q] = 0.f;
        if (i < n) {
            const long long b = rp[i], e = rp[i + 1];
            for (long long c0 = b; c0 < e; c0 += 32) {
                const int cnt = (int)min((long long)32, e - c0);
                int myc = 0;
                float myv = 0.f;
                if (lane < cnt) {
                    myc = cols[c0 + lane];
                    myv = vals[c0 + lane];
                }
                // U nonzeros at a time: all their Y loads issue before the
                // multiply-adds, which keep the ascending column order; slots
                // past the row's end carry weight 0 and read row k = 0
                constexpr int U = JW <= 3 ? 8 : 4;
                for (int t0 = 0; t0 < cnt; t0 += U) {
                    float av[U], yv[U][JW];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int t = t0 + u;
                        const int k = __shfl_sync(0xFFFFFFFFu, myc, t & 31);
                        const float a = __shfl_sync(0xFFFFFFFFu, myv, t & 31);
                        av[u] = t < cnt ? a : 0.f;
                        const float *yr = Y + (size_t)(t < cnt ? k : 0) * m;
#pragma unroll
                        for (int q = 0; q < JW; q++) {
                            const int j = lane + 32 * q;
                            yv[u][q] = j < m ? yr[j] : 0.f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; u++)
#pragma unroll
                        for (int q = 0; q < JW; q++) acc[q] = fmaf(av[u], yv[u][q], acc[q]);
                }
            }
        }
        if (O64) {
#pragma unroll
            for (int q = 0; q < JW; q++) {
                const int j = lane + 32 * q;
                if (j >= m) continue;
                double v = 0.0;
                if (i < n) {
                    v = alpha * (double)acc[q];
                    if (beta != 0.0) v += beta * (double)Y[(size_t)i * m + j];
                    if (gamma != 0.0) v += gamma * (double)X[(size_t)i * m + j];
                }
                if (O) O[(size_t)i * m + j] = (float)v;
                s64[r][j] = v;
            }
        } else {
#pragma unroll
            for (int q = 0; q < JW; q++) {
                const int j = lane + 32 * q;
                if (j >= m) continue;
                float v = 0.f;
                if (i < n) {
                    v = alpha_f * acc[q];
                    if (beta != 0.0) v = fmaf(beta_f, Y[(size_t)i * m + j], v);
                    if (gamma != 0.0) v = fmaf(gamma_f, X[(size_t)i * m + j], v);
                }
                O[(size_t)i * m + j] = v;
            }
        }
    }
    if (!O64) return;
    __syncthreads();
    for (int e = threadIdx.x; e < m * kSpRows; e += blockDim.x) {
        const int j = e / kSpRows, r = e % kSpRows;
        O64[(size_t)j * n_pad + i0 + r] = s64[r][j];
    }
}

__global__ void k_output(const double *Xt, const double *mass, int n, int n_pad, int k, double *evecs) {
    const size_t total = (size_t)n * k;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / k), j = (int)(e % k);
        evecs[e] = Xt[(size_t)j * n_pad + i] / sqrt(mass[i]);
    }
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

static bool make_map(CUtensorMap *tm, const float *ptr, int inner, int rows, int box_rows) {
    auto enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)inner * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)ptr, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Plan {
    int n, k, m, n_pad, splits, ktiles, kt_per_split, stages, smem;
    uint32_t tmem_cols, idesc;
};

static Plan plan_for(int n, int k, int guard) {
    Plan p;
    p.n = n;
    p.k = k;
    p.m = std::min(160, ((k + guard + 15) / 16) * 16);
    p.n_pad = ((n + BM - 1) / BM) * BM;
    p.ktiles = p.n_pad / BK;
    const int tiles = p.n_pad / BM;
    int sp = std::max(1, 148 / tiles);
    sp = std::min(sp, std::max(1, p.ktiles / 4));
    p.kt_per_split = (p.ktiles + sp - 1) / sp;
    p.splits = (p.ktiles + p.kt_per_split - 1) / p.kt_per_split;
    const int stage = 2 * BM * 128 + 2 * p.m * 128;
    p.stages = std::max(2, std::min(4, (220 * 1024) / stage));
    p.smem = p.stages * stage + 1024;
    p.tmem_cols = 32;
    while (p.tmem_cols < (uint32_t)p.m) p.tmem_cols <<= 1;
    // kind::tf32 instruction descriptor: D fp32, A/B tf32, both K-major, N = m, M = 128
    p.idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(p.m >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    return p;
}

struct Ws {
    float *Ahi, *Alo, *P;
    float *vh[4], *vl[4];   // tf32 parts of block vectors (m x n_pad)
    double *Xt, *Zt, *Xt2, *G, *Gp, *Rinv, *Qd, *theta, *res, *rowabs, *bound, *sinv;
    float *Q, *qev;
    int *err, *shifted, *sweeps;
    long long *rp;  // CSR row pointers of the sparse operator (n + 1)
    size_t total;
};

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

static Ws ws_layout(const Plan &p, char *base) {
    Ws w;
    size_t o = 0;
    auto take = [&](size_t b) { char *r = base ? base + o : nullptr; o = a256(o + b); return r; };
    const size_t nn = (size_t)p.n_pad * p.n_pad, mv = (size_t)p.m * p.n_pad;
    w.Ahi = (float *)take(nn * 4);
    w.Alo = (float *)take(nn * 4);
    w.P = (float *)take((size_t)p.splits * mv * 4);
    for (int i = 0; i < 4; i++) { w.vh[i] = (float *)take(mv * 4); w.vl[i] = (float *)take(mv * 4); }
    w.Xt = (double *)take(mv * 8);
    w.Zt = (double *)take(mv * 8);
    w.Xt2 = (double *)take(mv * 8);
    w.G = (double *)take((size_t)p.m * p.m * 8);
    w.Gp = (double *)take((size_t)kGramChunksMax * p.m * p.m * 8);
    w.Rinv = (double *)take((size_t)p.m * p.m * 8);
    w.Qd = (double *)take((size_t)p.m * p.m * 8);
    w.theta = (double *)take(p.m * 8);
    w.res = (double *)take(p.m * 8);
    w.rowabs = (double *)take((size_t)p.n * 8);
    w.sinv = (double *)take((size_t)p.n * 8);
    w.bound = (double *)take(8);
    w.Q = (float *)take((size_t)p.m * p.m * 4);
    w.qev = (float *)take(p.m * 4);
    w.err = (int *)take(4);
    w.shifted = (int *)take(4);
    w.sweeps = (int *)take(4);
    w.rp = (long long *)take((size_t)(p.n + 1) * 8);
    w.total = o;
    return w;
}

struct Ctx {
    Plan p;
    Ws w;
    cudaStream_t st;
    CUtensorMap mAh, mAl, mBh[4], mBl[4];
    bool sparse = false;  // CSR operator: values in Ahi's space, columns in Alo's, vectors by rows in vh[]
};

// P <- A * (block b), the tensor-core product
static cudaError_t tc_product(Ctx &c, int b) {
    TcArgs a;
    a.part = c.w.P;
    a.n_pad = c.p.n_pad;
    a.m = c.p.m;
    a.ktiles = c.p.ktiles;
    a.kt_per_split = c.p.kt_per_split;
    a.stages = c.p.stages;
    a.idesc = c.p.idesc;
    a.tmem_cols = c.p.tmem_cols;
    a.err = c.w.err;
    note_launch();
    k_tc_gemm<<<dim3(c.p.n_pad / BM, c.p.splits), kTcThreads, c.p.smem, c.st>>>(c.mAh, c.mAl, c.mBh[b], c.mBl[b], a);
    return cudaGetLastError();
}

static int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 16); }

// one term O = alpha A Y + beta Y + gamma X on the CSR operator (vectors by rows)
static cudaError_t sp_filter(Ctx &c, double alpha, double beta, double gamma, const float *Y, const float *X, float *O,
                             double *O64) {
    const int m = c.p.m, jw = (m + 31) / 32;
    const dim3 grid(c.p.n_pad / kSpRows);
    const long long *rp = c.w.rp;
    const int *cols = (const int *)c.w.Alo;
    const float *vals = c.w.Ahi;
    note_launch();
#define MCS_SP(JW)                                                                                                    \
    k_sp_filter<JW><<<grid, 32 * kSpRows, 0, c.st>>>(rp, cols, vals, c.p.n, c.p.n_pad, m, alpha, beta, gamma,        \
                                                     (float)alpha, (float)beta, (float)gamma, Y, X, O, O64)
    switch (jw) {
        case 1: MCS_SP(1); break;
        case 2: MCS_SP(2); break;
        case 3: MCS_SP(3); break;
        case 4: MCS_SP(4); break;
        default: MCS_SP(5); break;
    }
#undef MCS_SP
    return cudaGetLastError();
}

// block X (FP64 by rows of X^T) into the product's operand buffer b: tf32
// parts for the dense product, FP32 by rows for the sparse one
static void to_operand(Ctx &c, const double *X, int b) {
    const size_t mv = (size_t)c.p.m * c.p.n_pad;
    note_launch();
    if (c.sparse)
        k_to_rows<<<dim3(c.p.n_pad / 32, (c.p.m + 31) / 32), 256, 0, c.st>>>(X, c.p.m, c.p.n_pad, c.w.vh[b]);
    else
        k_split<<<grid_for(mv), 256, 0, c.st>>>(X, mv, c.w.vh[b], c.w.vl[b]);
}

}  // namespace eig
}  // namespace mcs

using namespace mcs;
using namespace mcs::eig;

extern "C" {

size_t mcs_steklov_workspace_size(int n, int k) {
    if (n <= 0 || k <= 0) return 0;
    const Plan p = plan_for(n, k, 32);
    return ws_layout(p, nullptr).total;
}

mcs_status mcs_steklov_modes(const double *Lambda, const double *mass, int n, int k, double *evals, double *evecs,
                             void *workspace, size_t workspace_bytes, const mcs_eig_params *ep, mcs_eig_stats *stats,
                             void *stream_) {
    NvtxRange nvtx_range("mcs_steklov_modes");
    MCS_ARG(Lambda && mass && evals, "mcs_steklov_modes: NULL Lambda, mass or evals");
    MCS_ARG(n >= 16 && k >= 1 && k <= 128 && k < n / 2, "mcs_steklov_modes: need n >= 16 and 1 <= k <= min(128, n/2 - 1)");
    mcs_eig_params prm;
    mcs_default_eig_params(&prm);
    if (ep) prm = *ep;
    MCS_ARG(prm.degree >= 0 && prm.degree <= 256 && prm.max_iters >= 1 && prm.tol > 0.0 && prm.product >= 0 &&
                prm.product <= 2,
            "mcs_steklov_modes: bad params");
    Ctx c;
    c.p = plan_for(n, k, 32);
    c.st = as_stream(stream_);
    MCS_ARG(c.p.m > k && c.p.m <= 160, "mcs_steklov_modes: block size out of range");
    c.w = ws_layout(c.p, (char *)workspace);
    MCS_ARG(workspace && workspace_bytes >= c.w.total, "mcs_steklov_modes: workspace too small");
    MCS_ARG(((uintptr_t)workspace & 255) == 0, "mcs_steklov_modes: workspace must be 256-byte aligned");
    const Plan &p = c.p;
    const int m = p.m;
    if (!make_map(&c.mAh, c.w.Ahi, p.n_pad, p.n_pad, BM) || !make_map(&c.mAl, c.w.Alo, p.n_pad, p.n_pad, BM)) {
        set_error("mcs_steklov_modes: cuTensorMapEncodeTiled unavailable or failed");
        return MCS_ERR_CUDA;
    }
    for (int b = 0; b < 4; b++)
        if (!make_map(&c.mBh[b], c.w.vh[b], p.n_pad, m, m) || !make_map(&c.mBl[b], c.w.vl[b], p.n_pad, m, m)) {
            set_error("mcs_steklov_modes: tensor map for the block failed");
            return MCS_ERR_CUDA;
        }
    MCS_CUDA(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem));
    const size_t smm = (size_t)m * (m + 1) * sizeof(double);
    MCS_CUDA(cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smm));
    const size_t jsm = 2 * (size_t)m * (m + 1) * sizeof(float);
    MCS_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm));
    cudaStream_t st = c.st;
    const size_t mv = (size_t)m * p.n_pad;
    const int g = grid_for(mv);
    MCS_CUDA(cudaMemsetAsync(c.w.err, 0, sizeof(int), st));
    MCS_CUDA(cudaMemsetAsync(c.w.sweeps, 0, sizeof(int), st));
    // row nonzeros and Gershgorin sums of A, then the operator: CSR when A
    // has at most one nonzero in 32 (or when asked), else the dense tf32 parts
    note_launch();
    k_inv_sqrt<<<(n + 255) / 256, 256, 0, st>>>(mass, n, c.w.sinv);
    note_launch();
    k_row_stats<<<n, 256, 0, st>>>(Lambda, c.w.sinv, n, c.w.rp, c.w.rowabs);
    note_launch();
    k_row_scan<<<1, 1024, 0, st>>>(c.w.rp, n);
    note_launch();
    k_max_reduce<<<1, 1024, 0, st>>>(c.w.rowabs, n, c.w.bound);
    note_launch();
    k_random_block<<<g, 256, 0, st>>>(c.w.Xt, m, n, p.n_pad);
    double bound = 0.0;
    long long nnz = 0;
    MCS_CUDA(cudaMemcpyAsync(&bound, c.w.bound, sizeof(double), cudaMemcpyDeviceToHost, st));
    MCS_CUDA(cudaMemcpyAsync(&nnz, c.w.rp + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
    MCS_CUDA(cudaStreamSynchronize(st));
    c.sparse = prm.product == 2 || (prm.product == 0 && nnz * 32 <= (long long)n * n);
    note_launch();
    if (c.sparse)
        k_csr_fill<<<n, 256, 0, st>>>(Lambda, c.w.sinv, n, c.w.rp, c.w.Ahi, (int *)c.w.Alo);
    else
        k_prep_A<<<p.n_pad, 256, 0, st>>>(Lambda, c.w.sinv, n, p.n_pad, c.w.Ahi, c.w.Alo, nullptr);
    if (!(bound > 0.0)) bound = 1.0;
    const double ub = bound * 1.01;

    // block buffers (m x n_pad FP64, by rows of X^T): X, Z and a spare, rotated by role
    double *X = c.w.Xt, *Z = c.w.Zt, *T = c.w.Xt2;
    // n split so that the active 32 x 32 tiles fill about two blocks per SM
    const int gt = (m + 31) / 32;
    auto gram_chunks = [&](int tiles) {
        const int want = (2 * num_sms() + tiles - 1) / tiles;
        return std::max(1, std::min({kGramChunksMax, p.n_pad / 32, std::max(16, want)}));
    };
    const int gch_full = gram_chunks(gt * gt), gch_upper = gram_chunks(gt * (gt + 1) / 2);
    const dim3 bgrid(p.n_pad / 128, (m + kJG - 1) / kJG);
    const size_t bsm = (size_t)m * kJG * sizeof(double);
    auto gram = [&](const double *A, const double *B, int sym) {
        const int upper = A == B;
        const int ch = upper ? gch_upper : gch_full;
        note_launch();
        k_gram_part<<<dim3(gt, gt, ch), 256, 0, st>>>(A, B, m, p.n_pad, c.w.Gp, upper);
        note_launch();
        k_gram_reduce<<<(m * m + 255) / 256, 256, 0, st>>>(c.w.Gp, m, ch, c.w.G, sym, upper);
    };
    // orthonormalise X: shifted CholeskyQR, then CholeskyQR2 (FP64)
    // one CholeskyQR pass: X <- X R^-1 with R^T R = X^T X (+ shift); mode as k_chol_inv's
    const double shift_rel = 11.0 * ((double)p.n_pad * m + (double)m * (m + 1)) * 1.1102230246251565e-16;
    auto cholqr = [&](int mode) {
        gram(X, X, 1);
        note_launch();
        k_chol_inv<<<1, 1024, smm, st>>>(c.w.G, m, shift_rel, mode, c.w.Rinv, c.w.shifted, c.w.err);
        note_launch();
        k_block_times<<<bgrid, 128, bsm, st>>>(c.w.Rinv, X, m, p.n_pad, T, 1);
        std::swap(X, T);
    };
    // orthonormalise X in FP64: CholeskyQR2, preceded by a shifted pass
    // (CholeskyQR3) always (first = 1) or only when the first pass meets a
    // pivot that is not clearly positive (first = 2: that pass then restarts
    // shifted and a third pass follows)
    auto orth = [&](int first) -> cudaError_t {
        cholqr(first);
        cholqr(0);
        int extra = first == 1;
        if (first == 2) {
            cudaError_t e = cudaMemcpyAsync(&extra, c.w.shifted, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
        }
        if (extra) cholqr(0);
        return cudaGetLastError();
    };
    MCS_CUDA(orth(1));
    std::vector<double> theta(m), res(m);
    double a_cut = ub / 8.0, a_low = 0.0;
    int iters = 0, converged = 0, gemms = 0;
    // filter degree: prm.degree, halved (down to 8) whenever two iterations in
    // a row add no converged pair -- a filter of too high a degree spreads the
    // wanted components over more magnitudes than the FP32-accurate products
    // keep, and the last ones stop converging
    // degree 0: 48 with the dense product, 96 with the sparse one, whose
    // FP32 products (no tf32 truncation) keep the higher degree converging
    // (10,000-row union: 23.2 ms at 48, 21.3 at 64, 19.6 at 96 in 3
    // iterations; the dense two-sphere solve stalls above 48: 24.0 ms at 48,
    // 43 at 64)
    int deg = prm.degree > 0 ? prm.degree : (c.sparse ? 96 : 48), best_conv = -1, stall = 0;
    for (iters = 0; iters < prm.max_iters; iters++) {
        // ---- Chebyshev filter of degree d on [a_cut, ub] applied to X
        to_operand(c, X, 0);
        const double e = 0.5 * (ub - a_cut), cc = 0.5 * (ub + a_cut);
        double sigma = e / (a_low - cc);
        const double tau = 2.0 / sigma;
        int prev = -1, cur = 0;
        for (int d = 1; d <= deg; d++) {
            gemms++;
            int nxt = (cur + 1) % 3;
            if (nxt == prev) nxt = (nxt + 1) % 3;
            const bool last = d == deg;
            if (c.sparse) {
                double alpha, beta, gamma = 0.0;
                if (d == 1) {
                    alpha = sigma / e;
                    beta = -cc * sigma / e;
                } else {
                    const double sig_new = 1.0 / (tau - sigma);
                    alpha = 2.0 * sig_new / e;
                    beta = -2.0 * sig_new * cc / e;
                    gamma = -sigma * sig_new;
                    sigma = sig_new;
                }
                MCS_CUDA(sp_filter(c, alpha, beta, gamma, c.w.vh[cur], d == 1 ? nullptr : c.w.vh[prev],
                                   last ? nullptr : c.w.vh[nxt], last ? X : nullptr));
                prev = cur;
                cur = nxt;
                continue;
            }
            MCS_CUDA(tc_product(c, cur));
            if (d == 1) {
                const double alpha = sigma / e, beta = -cc * sigma / e;
                note_launch();
                k_combine<<<g, 256, 0, st>>>(c.w.P, p.splits, m, n, p.n_pad, alpha, beta, 0.0, c.w.vh[cur],
                                            c.w.vl[cur], nullptr, nullptr, last ? nullptr : c.w.vh[nxt],
                                            last ? nullptr : c.w.vl[nxt], last ? X : nullptr);
            } else {
                const double sig_new = 1.0 / (tau - sigma);
                const double alpha = 2.0 * sig_new / e, beta = -2.0 * sig_new * cc / e, gamma = -sigma * sig_new;
                note_launch();
                k_combine<<<g, 256, 0, st>>>(c.w.P, p.splits, m, n, p.n_pad, alpha, beta, gamma, c.w.vh[cur],
                                            c.w.vl[cur], c.w.vh[prev], c.w.vl[prev], last ? nullptr : c.w.vh[nxt],
                                            last ? nullptr : c.w.vl[nxt], last ? X : nullptr);
                sigma = sig_new;
            }
            prev = cur;
            cur = nxt;
        }
        // a filter that amplifies the lowest eigenvalues by many orders over
        // the top of the block can leave it numerically rank deficient
        // (accurate products keep no noise floor): the unshifted Gram then
        // has pivots that are not positive, and the shifted pass takes over
        MCS_CUDA(orth(2));
        // ---- Rayleigh-Ritz
        to_operand(c, X, 3);
        gemms++;
        if (c.sparse) {
            MCS_CUDA(sp_filter(c, 1.0, 0.0, 0.0, c.w.vh[3], nullptr, nullptr, Z));
        } else {
            MCS_CUDA(tc_product(c, 3));
            note_launch();
            k_combine<<<g, 256, 0, st>>>(c.w.P, p.splits, m, n, p.n_pad, 1.0, 0.0, 0.0, nullptr, nullptr, nullptr,
                                        nullptr, nullptr, nullptr, Z);
        }
        gram(X, Z, 1);
        note_launch();
        k_jacobi<<<1, 1024, jsm, st>>>(c.w.G, m, c.w.Q, c.w.qev, 30, c.w.sweeps);
        note_launch();
        k_f32_to_f64<<<(m * m + 255) / 256, 256, 0, st>>>(c.w.Q, m * m, c.w.Qd);
        note_launch();
        k_block_times<<<bgrid, 128, bsm, st>>>(c.w.Qd, X, m, p.n_pad, T, 0);
        std::swap(X, T);
        note_launch();
        k_block_times<<<bgrid, 128, bsm, st>>>(c.w.Qd, Z, m, p.n_pad, T, 0);
        std::swap(Z, T);
        note_launch();
        k_ritz<<<m, 256, 0, st>>>(X, Z, p.n_pad, c.w.theta, c.w.res);
        MCS_CUDA(cudaGetLastError());
        MCS_CUDA(cudaMemcpyAsync(theta.data(), c.w.theta, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        MCS_CUDA(cudaMemcpyAsync(res.data(), c.w.res, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        MCS_CUDA(cudaStreamSynchronize(st));
        converged = 0;
        while (converged < k && res[converged] <= prm.tol * ub) converged++;
        if (converged >= k) { iters++; break; }
        if (converged > best_conv) {
            best_conv = converged;
            stall = 0;
        } else if (++stall >= 2 && deg > 8) {
            deg = std::max(8, deg / 2);
            stall = 0;
        }
        a_cut = theta[m - 1];
        a_low = std::min(0.0, theta[0]);
    }
    // the last rotation used the FP32 Jacobi vectors: restore FP64 orthonormality
    if (evecs) MCS_CUDA(orth(0));
    int err = 0;
    MCS_CUDA(cudaMemcpyAsync(&err, c.w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MCS_CUDA(cudaMemcpyAsync(evals, c.w.theta, k * sizeof(double), cudaMemcpyDefault, st));
    if (evecs) {
        note_launch();
        k_output<<<grid_for((size_t)n * k), 256, 0, st>>>(X, mass, n, p.n_pad, k, evecs);
    }
    MCS_CUDA(cudaGetLastError());
    MCS_CUDA(cudaStreamSynchronize(st));
    if (stats) {
        stats->iterations = iters;
        stats->converged = converged;
        stats->block = m;
        stats->tc_products = gemms;
        stats->upper_bound = ub;
        stats->max_residual = 0.0;
        for (int j = 0; j < k; j++) stats->max_residual = std::max(stats->max_residual, res[j]);
        stats->device_error = err;
        stats->product = c.sparse ? 2 : 1;
        stats->nnz = nnz;
        MCS_CUDA(cudaMemcpy(&stats->jacobi_sweeps, c.w.sweeps, sizeof(int), cudaMemcpyDeviceToHost));
    }
    if (err & kErrTimeout) {
        set_error("mcs_steklov_modes: a tensor-core pipeline wait timed out");
        return MCS_ERR_DEVICE;
    }
    if (converged < k) {
        set_error("mcs_steklov_modes: not converged within max_iters");
        return MCS_WARN_NOT_CONVERGED;
    }
    return MCS_OK;
}

// test hook: Zt = (A X)^T for symmetric A (n x n FP64, row-major) and
// Xt (m x n FP64), through the same tensor-core product
mcs_status mcs_tc_symm_product(const double *A, const double *Xt_in, int n, int m_in, double *Zt_out, void *workspace,
                               size_t workspace_bytes, void *stream_) {
    MCS_ARG(A && Xt_in && Zt_out, "mcs_tc_symm_product: NULL pointer");
    MCS_ARG(n >= 16 && m_in >= 16 && m_in <= 160 && m_in % 16 == 0, "mcs_tc_symm_product: need m in {16,...,160}, m % 16 == 0");
    Ctx c;
    c.p = plan_for(n, m_in - 32 > 0 ? m_in - 32 : 1, 32);
    c.p.m = m_in;
    const int stage = 2 * BM * 128 + 2 * m_in * 128;
    c.p.stages = std::max(2, std::min(4, (220 * 1024) / stage));
    c.p.smem = c.p.stages * stage + 1024;
    c.p.tmem_cols = 32;
    while (c.p.tmem_cols < (uint32_t)m_in) c.p.tmem_cols <<= 1;
    c.p.idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(m_in >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    c.st = as_stream(stream_);
    c.w = ws_layout(c.p, (char *)workspace);
    MCS_ARG(workspace && workspace_bytes >= c.w.total, "mcs_tc_symm_product: workspace too small");
    const Plan &p = c.p;
    if (!make_map(&c.mAh, c.w.Ahi, p.n_pad, p.n_pad, BM) || !make_map(&c.mAl, c.w.Alo, p.n_pad, p.n_pad, BM) ||
        !make_map(&c.mBh[0], c.w.vh[0], p.n_pad, p.m, p.m) || !make_map(&c.mBl[0], c.w.vl[0], p.n_pad, p.m, p.m)) {
        set_error("mcs_tc_symm_product: tensor map failed");
        return MCS_ERR_CUDA;
    }
    MCS_CUDA(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem));
    cudaStream_t st = c.st;
    MCS_CUDA(cudaMemsetAsync(c.w.err, 0, sizeof(int), st));
    // unit mass: A itself
    double *ones = c.w.rowabs;  // n doubles
    std::vector<double> h1(n, 1.0);
    MCS_CUDA(cudaMemcpyAsync(ones, h1.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    note_launch();
    k_inv_sqrt<<<(n + 255) / 256, 256, 0, st>>>(ones, n, c.w.sinv);
    note_launch();
    k_prep_A<<<p.n_pad, 256, 0, st>>>(A, c.w.sinv, n, p.n_pad, c.w.Ahi, c.w.Alo, c.w.Zt);
    const size_t mv = (size_t)p.m * p.n_pad;
    MCS_CUDA(cudaMemsetAsync(c.w.Xt, 0, mv * sizeof(double), st));
    MCS_CUDA(cudaMemcpy2DAsync(c.w.Xt, p.n_pad * sizeof(double), Xt_in, n * sizeof(double), n * sizeof(double), p.m,
                               cudaMemcpyDeviceToDevice, st));
    note_launch();
    k_split<<<grid_for(mv), 256, 0, st>>>(c.w.Xt, mv, c.w.vh[0], c.w.vl[0]);
    MCS_CUDA(tc_product(c, 0));
    note_launch();
    k_combine<<<grid_for(mv), 256, 0, st>>>(c.w.P, p.splits, p.m, n, p.n_pad, 1.0, 0.0, 0.0, nullptr, nullptr, nullptr,
                                           nullptr, nullptr, nullptr, c.w.Zt);
    MCS_CUDA(cudaMemcpy2DAsync(Zt_out, n * sizeof(double), c.w.Zt, p.n_pad * sizeof(double), n * sizeof(double), p.m,
                               cudaMemcpyDeviceToDevice, st));
    int err = 0;
    MCS_CUDA(cudaMemcpyAsync(&err, c.w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MCS_CUDA(cudaStreamSynchronize(st));
    if (err) {
        set_error("mcs_tc_symm_product: device error (pipeline timeout)");
        return MCS_ERR_DEVICE;
    }
    return MCS_OK;
}

size_t mcs_tc_symm_product_workspace_size(int n, int m) {
    Plan p = plan_for(n, std::max(1, m - 32), 32);
    p.m = m;
    return ws_layout(p, nullptr).total;
}

void mcs_default_eig_params(mcs_eig_params *p) {
    if (!p) return;
    // degree 0: chosen by the product (see mcs_steklov_modes).  For the dense
    // tf32-split product 48 (measured, k = 64: two-sphere exterior n = 5124:
    // degree 48 34.5 ms, 64 57.7 ms, 80 48.7 ms; icosphere s3 interior n = 642:
    // 13.9, 25.1, 31.5 ms): higher degrees spread the wanted components over
    // more magnitudes than those products keep, stall, and pay for the
    // halving; 24 needs more FP64 orthogonalisations and Rayleigh-Ritz steps
    // per converged block
    p->degree = 0;
    p->max_iters = 60;
    p->tol = 1e-5;
    p->product = 0;
}

}  // extern "C"
